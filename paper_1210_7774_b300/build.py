"""Build libvbe.so in-tree with nvcc for sm_103a.

The library's host code (analysis, code generation, runtime, server) is
C++ compiled by nvcc's host compiler; its kernels are generated per run and
compiled at run time by NVRTC for sm_103a. ``python -m
paper_1210_7774_b300.build`` or ``build()`` rebuilds when a source is newer
than the library.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libvbe.so")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cpp")) + glob.glob(os.path.join(CSRC, "*.cu")))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def embed_device_sources() -> None:
    """Write _embed_sf64.inc: the device-side soft float64 code (tables and
    functions) as two C++ raw strings, which the runtime hands to NVRTC as
    the headers "sf64_tables.h" and "sf64.cuh" of the kernels that need them."""
    parts = []
    for var, name in (("kSf64Tables", "sf64_tables.h"), ("kSf64Code", "sf64.cuh")):
        text = open(os.path.join(CSRC, name)).read()
        assert ")VBESF64" not in text
        parts.append(f'static const char* const {var} = R"VBESF64({text})VBESF64";\n')
    out = os.path.join(CSRC, "_embed_sf64.inc")
    body = "".join(parts)
    if not os.path.exists(out) or open(out).read() != body:
        with open(out, "w") as f:
            f.write(body)


def build(force: bool = False, verbose: bool = False) -> str:
    embed_device_sources()
    if not force and not _stale():
        return LIB
    nvcc = os.path.join(CUDA, "bin", "nvcc")
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    objs = []
    procs = []
    for src in sources():
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, "-lineinfo", "-O2", "-std=c++17", "-Xcompiler", "-fPIC,-Wall",
               "-I", INCLUDE, "-c", src, "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    for cmd, p in procs:
        out = p.communicate()[0].decode()
        if p.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + out)
        if verbose and out.strip():
            print(out)
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-L", os.path.join(CUDA, "lib64"), "-lnvrtc",
           "-Xlinker", "-rpath," + os.path.join(CUDA, "lib64")]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + " ".join(cmd) + "\n" + r.stdout.decode())
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
