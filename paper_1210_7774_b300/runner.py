"""Marshal a bytecode program (``workloads.Program``) onto a libvbe context.

Bases become library handles (created lazily, or filled from host data, or
wrapping caller-owned device memory), each distinct view becomes one view
handle, and the instructions become ``vbe_instr`` arrays, one per batch.
All execution happens in libvbe; this module only translates.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from workloads.program import NP_DTYPE, Const, Program, View

from . import vbe as V

# the dtype a constant operand takes (vbe.h, vbe_instr.const_slot)
_SELECT = "SELECT"


def opcode_of(ctx, program: Program, op: str) -> int:
    """The opcode of a mnemonic; ``"USER:<name>"`` registers the program's
    user-defined operation of that name with the library."""
    if op.startswith("USER:"):
        u = program.user_ops[op[5:]]
        return V.vbe_op_register(ctx, u.name, u.body, u.nin, V.DTYPE_CODE[u.dtype])
    return V.OPCODES[op]


def _const_dtype(instr, k: int, dtypes: dict) -> str:
    if instr.op == _SELECT:
        return "bool" if k == 0 else dtypes[instr.out.base]
    if instr.op == "COPY":
        return dtypes[instr.out.base]
    for x in instr.ins:
        if isinstance(x, View):
            return dtypes[x.base]
    return dtypes[instr.out.base]


class Loaded:
    """A program's handles on one context."""

    def __init__(self, ex: "Executor", program: Program):
        self.ex = ex
        self.program = program
        self.base = {}  # program base id -> handle
        self.view = {}  # View -> handle
        self.batches = []  # (ctypes array, n)
        self.keep = []  # host buffers that must outlive uploads


class Executor:
    """One libvbe context plus program marshalling."""

    def __init__(self, flags: int = V.VBE_FUSE | V.VBE_GRAPHS | V.VBE_AUTOTUNE | V.VBE_PACK, device: int = 0,
                 stream: Optional[int] = None, cache_dir: Optional[str] = None, mem_cap_bytes: int = 0):
        self.flags = flags
        self.ctx = V.vbe_init(device, flags, mem_cap_bytes, stream, cache_dir)

    def close(self) -> None:
        if self.ctx:
            V.vbe_finalize(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------ loading
    def load(self, program: Program, device_ptrs: Optional[dict] = None, upload: bool = True) -> Loaded:
        """Create handles for ``program``. Bases with host data are uploaded
        (or, when ``device_ptrs`` maps their id to a device address holding
        the data, registered without a copy)."""
        L = Loaded(self, program)
        device_ptrs = device_ptrs or {}
        for bid, b in program.bases.items():
            code = V.DTYPE_CODE[b.dtype]
            if bid in device_ptrs:
                L.base[bid] = V.vbe_base_register(self.ctx, code, b.nelem, device_ptrs[bid])
            else:
                L.base[bid] = V.vbe_base_create(self.ctx, code, b.nelem)
                if b.init is not None and upload:
                    arr = np.ascontiguousarray(b.init)
                    V.vbe_base_upload(self.ctx, L.base[bid], arr.ctypes.data, arr.nbytes)
        ranges = program.meta.get("batches") or [(0, len(program.instrs))]
        for (a, z) in ranges:
            L.batches.append(self.encode(L, program.instrs[a:z]))
        return L

    def view_handle(self, L: Loaded, v: View) -> int:
        h = L.view.get(v)
        if h is None:
            h = V.vbe_view_create(self.ctx, L.base[v.base], v.offset, v.shape, v.strides)
            L.view[v] = h
        return h

    def encode(self, L: Loaded, instrs) -> tuple:
        dtypes = {bid: b.dtype for bid, b in L.program.bases.items()}
        arr = (V.vbe_instr * max(1, len(instrs)))()
        codes = {}
        for i, ins in enumerate(instrs):
            e = arr[i]
            if ins.op not in codes:
                codes[ins.op] = opcode_of(self.ctx, L.program, ins.op)
            e.op = codes[ins.op]
            e.const_slot = -1
            e.out = self.view_handle(L, ins.out) if ins.out is not None else 0
            for k, x in enumerate(ins.ins):
                if isinstance(x, Const):
                    e.const_slot = k
                    cd = _const_dtype(ins, k, dtypes)
                    if cd in ("float32", "float64"):
                        e.konst.f64 = float(x.value)
                    else:
                        e.konst.i64 = int(x.value)
                    e.in_[k] = 0
                else:
                    e.in_[k] = self.view_handle(L, x)
            e.axis = ins.axis
            e.seed = ins.seed & ((1 << 64) - 1)
            e.key = ins.key & ((1 << 64) - 1)
            e.step = ins.step
        return (arr, len(instrs))

    # ---------------------------------------------------------- execution
    def submit(self, L: Loaded, batch: int) -> int:
        arr, n = L.batches[batch]
        return V.vbe_submit(self.ctx, arr, n)

    def run(self, L: Loaded) -> None:
        for k in range(len(L.batches)):
            self.submit(L, k)

    def read(self, L: Loaded, bid: int) -> np.ndarray:
        b = L.program.bases[bid]
        out = np.empty(b.nelem, dtype=NP_DTYPE[b.dtype])
        V.vbe_sync(self.ctx, L.base[bid], out.ctypes.data, out.nbytes)
        return out

    def plan(self, L: Loaded, batch: int = 0, source: bool = False) -> str:
        arr, n = L.batches[batch]
        return V.vbe_plan(self.ctx, arr, n, source)

    def stats(self) -> dict:
        return V.vbe_get_stats(self.ctx)

    def release(self, L: Loaded) -> None:
        for h in L.base.values():
            try:
                V.vbe_free(self.ctx, h)
            except V.VbeError:
                pass  # already released by a FREE instruction
        L.base.clear()
        L.view.clear()


class Request:
    """A program packed as a ``vbe_request`` for the serving loop. The
    ctypes arrays and the result buffers live as long as this object."""

    def __init__(self, program: Program, results=None):
        self.program = program
        ids = list(program.bases)
        index = {bid: i for i, bid in enumerate(ids)}
        self.results = {}
        self.bases = (V.vbe_req_base * max(1, len(ids)))()
        self._keep = []
        want = program.outputs if results is None else results
        for i, bid in enumerate(ids):
            b = program.bases[bid]
            rb = self.bases[i]
            rb.dtype = V.DTYPE_CODE[b.dtype]
            rb.nelem = b.nelem
            if b.init is not None:
                arr = np.ascontiguousarray(b.init)
                self._keep.append(arr)
                rb.init = arr.ctypes.data
            if bid in want:
                out = np.empty(b.nelem, dtype=NP_DTYPE[b.dtype])
                self.results[bid] = out
                rb.result = out.ctypes.data
        views = {}
        for ins in program.instrs:
            for v in (ins.out, *ins.ins):
                if isinstance(v, View) and v not in views:
                    views[v] = len(views) + 1
        self.views = (V.vbe_req_view * max(1, len(views)))()
        for v, k in views.items():
            rv = self.views[k - 1]
            rv.base = index[v.base]
            rv.ndim = v.ndim
            rv.offset = v.offset
            for d in range(v.ndim):
                rv.shape[d] = v.shape[d]
                rv.strides[d] = v.strides[d]
        dtypes = {bid: b.dtype for bid, b in program.bases.items()}
        n = len(program.instrs)
        self.instrs = (V.vbe_instr * max(1, n))()
        for i, ins in enumerate(program.instrs):
            e = self.instrs[i]
            e.op = V.OPCODES[ins.op]
            e.const_slot = -1
            e.out = views[ins.out] if ins.out is not None else 0
            for k, x in enumerate(ins.ins):
                if isinstance(x, Const):
                    e.const_slot = k
                    if _const_dtype(ins, k, dtypes) in ("float32", "float64"):
                        e.konst.f64 = float(x.value)
                    else:
                        e.konst.i64 = int(x.value)
                else:
                    e.in_[k] = views[x]
            e.axis = ins.axis
            e.seed = ins.seed & ((1 << 64) - 1)
            e.key = ins.key & ((1 << 64) - 1)
            e.step = ins.step
        self.req = V.vbe_request(self.bases, len(ids), len(views), self.views, self.instrs, n)
        self._ids = ids

    def result_bytes(self) -> int:
        """Bytes of all result buffers, each rounded up to 64 bytes."""
        return sum((a.nbytes + 63) // 64 * 64 for a in self.results.values())

    def bind_results(self, arena: np.ndarray) -> None:
        """Point the request's result buffers into ``arena`` (a uint8 array of
        at least result_bytes(); e.g. page-locked memory, which the server
        then fills straight from the device). ``results`` become views of it."""
        off = 0
        for i, bid in enumerate(self._ids):
            if bid not in self.results:
                continue
            a = self.results[bid]
            view = arena[off:off + a.nbytes].view(a.dtype)
            self.results[bid] = view
            self.bases[i].result = view.ctypes.data
            off += (a.nbytes + 63) // 64 * 64


def run_program(program: Program, flags: int = V.VBE_FUSE | V.VBE_GRAPHS | V.VBE_AUTOTUNE | V.VBE_PACK,
                outputs=None, device: int = 0) -> dict:
    """Execute ``program`` on the GPU and return ``{base id: flat array}``
    for its outputs."""
    with Executor(flags, device) as ex:
        L = ex.load(program)
        ex.run(L)
        return {bid: ex.read(L, bid) for bid in (outputs or program.outputs)}
