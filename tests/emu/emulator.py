"""Run recorded libvbe launches on the CPU (test infrastructure).

A context created with VBE_RECORD keeps its bases in host memory and
records each launch (kernel source, entry, grid, block, parameter words)
instead of running it. This module compiles each generated source with
``vbe_emu.h`` into a small shared library and executes the launches in
order on the host, with every memory access checked against the context's
allocations. It lets the host test suite check the code generator's index
arithmetic and results without a GPU.
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os
import re
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
EMU_H = os.path.join(HERE, "vbe_emu.h")
# the soft float64 headers that generated kernels include
CSRC = os.path.join(os.path.dirname(os.path.dirname(HERE)), "paper_1210_7774_b300", "csrc")

_GLOBALS = """
thread_local dim3 threadIdx, blockIdx;
dim3 blockDim, gridDim;
std::vector<EmuRange> g_ranges;
std::atomic<long long> g_bad{0};
char g_bad_msg[256];
std::barrier<>* g_block_bar = nullptr;
std::vector<std::unique_ptr<std::barrier<>>> g_warp_bar;
unsigned long long g_xchg[1024];
int g_emu_drop = 0;
extern "C" void emu_set_drop(int d) { g_emu_drop = d; }
"""

_WRAP_COMMON = """
extern "C" void emu_set_ranges(const unsigned long long* lohi, int n) {
  g_ranges.clear();
  for (int i = 0; i < n; ++i) g_ranges.push_back({(uintptr_t)lohi[2 * i], (uintptr_t)lohi[2 * i + 1]});
}
extern "C" const char* emu_msg() { return g_bad_msg; }
static int emu_check_words(int nw) { return nw == (int)(sizeof(P) / 8) ? 0 : -1; }
template <class F> struct emu_arg;
template <class T> struct emu_arg<void(T)> { typedef std::remove_cv_t<T> type; };
"""

_WRAP_TILE = """
extern "C" long long emu_tile(int U, const long long* w, int nw, unsigned grid, unsigned block) {
  if (emu_check_words(nw)) return -1;
  P p;
  memcpy(&p, w, sizeof(P));
  g_bad = 0;
  emu_grid(grid, block, [&]() { if (U == 1) @P@_u1(p); else if (U == 2) @P@_u2(p); else @P@_u4(p); });
  return g_bad.load();
}
"""

_WRAP_PACK = """
extern "C" long long emu_pack(int U, long long descs, long long prefix, int ninst, long long total,
                              long long chunk, long long work, unsigned grid, unsigned block) {
  g_bad = 0;
  emu_grid(grid, block, [&]() {
    if (U == 1) @P@_pack_u1((const P*)descs, (const i64*)prefix, ninst, total, chunk, (unsigned*)work);
    else @P@_pack_u4((const P*)descs, (const i64*)prefix, ninst, total, chunk, (unsigned*)work);
  });
  return g_bad.load();
}
"""

_WRAP_BULK = """
extern "C" long long emu_bulk(const long long* w, int nw, unsigned grid, unsigned block) {
  if (emu_check_words(nw)) return -1;
  P p;
  memcpy(&p, w, sizeof(P));
  g_bad = 0;
  emu_grid(grid, block, [&]() { @P@_bulk(p); });
  return g_bad.load();
}
"""

_WRAP_ENTRY = """
extern "C" long long emu_@E@(const long long* w, int nw, unsigned grid, unsigned block) {
  typedef emu_arg<decltype(@E@)>::type A;  // P, or the tensor-map block of a tensor-copy kernel
  if (nw != (int)(sizeof(A) / 8)) return -1;
  A p;
  memcpy(&p, w, sizeof(A));
  g_bad = 0;
  emu_grid(grid, block, [&]() { @E@(p); });
  return g_bad.load();
}
"""

_WRAP_AXIS = """
extern "C" long long emu_axis(const long long* w, int nw, unsigned grid, unsigned block) {
  if (emu_check_words(nw)) return -1;
  P p;
  memcpy(&p, w, sizeof(P));
  g_bad = 0;
  emu_grid(grid, block, [&]() { @P@_axis(p); });
  return g_bad.load();
}
"""


# bump when build() changes how it finds entries or picks wrappers
_WRAPPER_RULES = "entries: launch bounds with an optional minimum of blocks; group forms sg ss tm rs"


class EmulationError(AssertionError):
    pass


class Emulator:
    def __init__(self, workdir: str | None = None):
        self.dir = workdir or os.path.join(tempfile.gettempdir(), "vbe_emu_cache")
        os.makedirs(self.dir, exist_ok=True)
        self.mods = {}
        self.launches = 0

    def _key(self, src: str) -> str:
        # the source names the soft float64 headers' hash; the emulation
        # header, the wrappers and the rules that pick the wrappers are part
        # of every module too
        return hashlib.sha1((src + self._emu_h + _GLOBALS + _WRAP_COMMON + _WRAPPER_RULES).encode()).hexdigest()[:20]

    @property
    def _emu_h(self) -> str:
        if not hasattr(self, "_emu_text"):
            self._emu_text = open(EMU_H).read()
        return self._emu_text

    def prebuild(self, sources) -> None:
        """Compile many sources at once (in parallel processes)."""
        from concurrent.futures import ThreadPoolExecutor
        todo = {self._key(s): s for s in sources}
        todo = [s for h, s in todo.items() if not os.path.exists(os.path.join(self.dir, f"emu_{h}.so"))]
        with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as pool:
            list(pool.map(self.build, todo))

    def module(self, src: str):
        h = self._key(src)
        if h in self.mods:
            return self.mods[h]
        so = self.build(src)
        return self._load(h, so)

    def build(self, src: str) -> str:
        h = self._key(src)
        so = os.path.join(self.dir, f"emu_{h}.so")
        if not os.path.exists(so):
            parts = [f'#include "{EMU_H}"', "#include <type_traits>", _GLOBALS, src, _WRAP_COMMON]
            names = re.findall(r"__global__ void __launch_bounds__\(\d+(?:, \d+)?\) (\w+)\(", src)
            prefix = names[0].rsplit("_", 1)[0] if names else "vbe"
            if prefix.endswith("_pack"):
                prefix = prefix[:-5]
            if prefix + "_u1" in names:
                parts.append(_WRAP_TILE.replace("@P@", prefix))
            if prefix + "_pack_u1" in names:
                parts.append(_WRAP_PACK.replace("@P@", prefix))
            if prefix + "_axis" in names:
                parts.append(_WRAP_AXIS.replace("@P@", prefix))
            if prefix + "_bulk" in names:
                parts.append(_WRAP_BULK.replace("@P@", prefix))
            for name in names:  # tile-fused groups: one kernel per tile shape
                if re.search(r"_(s[gs]|tm|rs)\d+x\d+$", name):
                    parts.append(_WRAP_ENTRY.replace("@E@", name))
            cpp = os.path.join(self.dir, f"emu_{h}.cpp")
            with open(cpp, "w") as f:
                f.write("\n".join(parts))
            tmp = so + f".{os.getpid()}.tmp"
            r = subprocess.run(["g++", "-std=c++20", "-O0", "-fPIC", "-shared", "-pthread", "-w", "-I", CSRC, cpp,
                                "-o", tmp],
                               stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
            if r.returncode != 0:
                raise EmulationError("emulation build failed:\n" + r.stdout.decode()[-4000:])
            os.replace(tmp, so)
        return so

    def _load(self, h: str, so: str):
        lib = ctypes.CDLL(so)
        lib.emu_set_ranges.argtypes = [ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_int]
        lib.emu_msg.restype = ctypes.c_char_p
        if hasattr(lib, "emu_tile"):
            lib.emu_tile.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int, ctypes.c_uint,
                                     ctypes.c_uint]
            lib.emu_tile.restype = ctypes.c_longlong
        if hasattr(lib, "emu_bulk"):
            lib.emu_bulk.argtypes = [ctypes.POINTER(ctypes.c_longlong), ctypes.c_int, ctypes.c_uint, ctypes.c_uint]
            lib.emu_bulk.restype = ctypes.c_longlong
        if hasattr(lib, "emu_axis"):
            lib.emu_axis.argtypes = [ctypes.POINTER(ctypes.c_longlong), ctypes.c_int, ctypes.c_uint, ctypes.c_uint]
            lib.emu_axis.restype = ctypes.c_longlong
        if hasattr(lib, "emu_pack"):
            lib.emu_pack.argtypes = [ctypes.c_int] + [ctypes.c_longlong] * 2 + [ctypes.c_int] + \
                [ctypes.c_longlong] * 3 + [ctypes.c_uint, ctypes.c_uint]
            lib.emu_pack.restype = ctypes.c_longlong
        self.mods[h] = lib
        return lib

    def run(self, record_json: str, drop_copies: bool = False) -> int:
        """Execute the recorded launches in order; ``drop_copies``: bulk and
        tensor copies never land (every wait on them runs out)."""
        js = json.loads(record_json)
        flat = []
        for addr, nbytes in js["allocs"]:
            flat += [addr, addr + nbytes]
        ranges = (ctypes.c_ulonglong * max(1, len(flat)))(*flat)
        for L in js["launches"]:
            if L.get("copy"):
                # a host <-> device copy in stream order (device memory is host
                # memory on a recording context)
                ctypes.memmove(L["dst"], L["src"], L["bytes"])
                continue
            lib = self.module(js["sources"][L["key"]])
            lib.emu_set_ranges(ranges, len(flat) // 2)
            lib.emu_set_drop(1 if drop_copies else 0)
            entry = L["entry"]
            if L.get("packed"):
                ctypes.c_uint.from_address(L["work"]).value = 0
                bad = lib.emu_pack(int(entry.rsplit("u", 1)[1]), L["descs"], L["prefix"], L["ninst"], L["total"],
                                   L["chunk"], L["work"], L["grid"], L["block"])
            else:
                w = (ctypes.c_longlong * len(L["words"]))(*L["words"])
                if re.search(r"_(s[gs]|tm|rs)\d+x\d+$", entry):
                    fn = getattr(lib, "emu_" + entry)
                    fn.argtypes = [ctypes.POINTER(ctypes.c_longlong), ctypes.c_int, ctypes.c_uint, ctypes.c_uint]
                    fn.restype = ctypes.c_longlong
                    bad = fn(w, len(L["words"]), L["grid"], L["block"])
                elif entry.endswith("_bulk"):
                    bad = lib.emu_bulk(w, len(L["words"]), L["grid"], L["block"])
                elif entry.endswith("_axis"):
                    bad = lib.emu_axis(w, len(L["words"]), L["grid"], L["block"])
                else:
                    bad = lib.emu_tile(int(entry.rsplit("_u", 1)[1]), w, len(L["words"]), L["grid"], L["block"])
            if bad:
                raise EmulationError(f"{entry} (grid {L['grid']}, block {L['block']}): "
                                     f"{'parameter block size mismatch' if bad < 0 else lib.emu_msg().decode()}")
            self.launches += 1
        return len(js["launches"])
