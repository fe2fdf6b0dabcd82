"""mcore: the paper's multi-core blocked Vector Engine, restated in C++ as a
CPU baseline (``mcore.cpp``): kernels formed by the blockable rule, each run
block by block over a pool of worker threads, with the number of data
blocks chosen by the user (section "Vector Engine" of the implementation;
the "mcore" engine of section "Performance Study").

A baseline for the benchmark, not an execution path of the GPU library:
nothing in the library calls it. ``run(program)`` executes a
``workloads.Program`` on host copies of its bases and returns
``{base id: flat array}`` like the reference interpreter.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from workloads.program import NP_DTYPE, Const, View

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mcore.cpp")
LIB = os.path.join(HERE, "libmcore.so")

OPCODES = {
    "ADD": 1, "SUBTRACT": 2, "MULTIPLY": 3, "DIVIDE": 4, "MAXIMUM": 5, "MINIMUM": 6, "SQRT": 7, "EXP": 8,
    "LOG": 9, "ABSOLUTE": 10, "NEGATIVE": 11, "LESS": 12, "LESS_EQUAL": 13, "GREATER": 14,
    "GREATER_EQUAL": 15, "EQUAL": 16, "NOT_EQUAL": 17, "SELECT": 18, "CAST": 19, "COPY": 20, "RANDOM": 21,
    "ADD_REDUCE": 22, "MIN_REDUCE": 23, "MAX_REDUCE": 24, "SYNC": 25, "DISCARD": 26, "FREE": 27,
    "ARGMIN_REDUCE": 28, "ARGMAX_REDUCE": 29,
}
DTYPE = {"bool": 0, "int64": 1, "float32": 2, "float64": 3}


class mc_base(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("pad", ctypes.c_int32), ("nelem", ctypes.c_int64),
                ("data", ctypes.c_void_p)]


class mc_view(ctypes.Structure):
    _fields_ = [("base", ctypes.c_int32), ("ndim", ctypes.c_int32), ("offset", ctypes.c_int64),
                ("shape", ctypes.c_int64 * 8), ("strides", ctypes.c_int64 * 8)]


class mc_instr(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("const_slot", ctypes.c_int32), ("out", ctypes.c_int32),
                ("in_", ctypes.c_int32 * 3), ("axis", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("kf", ctypes.c_double), ("ki", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("key", ctypes.c_uint64), ("step", ctypes.c_int64)]


def build(force: bool = False) -> str:
    """Compile libmcore.so with g++ (plain -O3, no host-specific flags)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = f"{LIB}.{os.getpid()}.tmp"  # concurrent builders each write their own
        subprocess.run(["g++", "-O3", "-std=c++17", "-fPIC", "-shared", "-Wall", "-o", tmp, SRC, "-lpthread"],
                       check=True)
        os.replace(tmp, LIB)
    return LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.mcore_run.argtypes = [ctypes.POINTER(mc_base), ctypes.c_int32, ctypes.POINTER(mc_view),
                                   ctypes.c_int32, ctypes.POINTER(mc_instr), ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
        _lib.mcore_run.restype = ctypes.c_int32
    return _lib


class McoreError(RuntimeError):
    pass


def cores() -> int:
    return len(os.sched_getaffinity(0))


class Prepared:
    """A program marshalled once (host copies of its bases, views and
    instructions), so that it can be run several times for timing."""

    def __init__(self, program, instrs=None):
        self.program = program
        ids = list(program.bases)
        index = {bid: i for i, bid in enumerate(ids)}
        self.arrays = {}
        self.bases = (mc_base * max(1, len(ids)))()
        for i, bid in enumerate(ids):
            b = program.bases[bid]
            arr = np.array(b.init, dtype=NP_DTYPE[b.dtype]).reshape(-1) if b.init is not None else \
                np.zeros(b.nelem, dtype=NP_DTYPE[b.dtype])
            self.arrays[bid] = arr
            self.bases[i].dtype = DTYPE[b.dtype]
            self.bases[i].nelem = b.nelem
            self.bases[i].data = arr.ctypes.data
        instrs = program.instrs if instrs is None else instrs
        views = {}
        for ins in instrs:
            for v in (ins.out, *ins.ins):
                if isinstance(v, View) and v not in views:
                    views[v] = len(views)
        self.views = (mc_view * max(1, len(views)))()
        for v, k in views.items():
            mv = self.views[k]
            mv.base = index[v.base]
            mv.ndim = v.ndim
            mv.offset = v.offset
            for d in range(v.ndim):
                mv.shape[d] = v.shape[d]
                mv.strides[d] = v.strides[d]
        self.nviews = len(views)
        self.instrs = (mc_instr * max(1, len(instrs)))()
        for i, ins in enumerate(instrs):
            if ins.op not in OPCODES:
                raise McoreError(f"mcore does not run {ins.op}")
            e = self.instrs[i]
            e.op = OPCODES[ins.op]
            e.const_slot = -1
            e.out = views[ins.out] if ins.out is not None else -1
            for k in range(3):
                e.in_[k] = -1
            for k, x in enumerate(ins.ins):
                if isinstance(x, Const):
                    e.const_slot = k
                    e.kf = float(x.value)
                    e.ki = int(x.value) if float(x.value).is_integer() else 0
                else:
                    e.in_[k] = views[x]
            e.axis = ins.axis
            e.seed = ins.seed & ((1 << 64) - 1)
            e.key = ins.key & ((1 << 64) - 1)
            e.step = ins.step
        self.ninstrs = len(instrs)
        self.kernels = 0

    def run(self, threads: int | None = None, blocks: int | None = None, inline_below: int = 1 << 15) -> dict:
        """Execute on ``threads`` workers (default: every usable core) with
        ``blocks`` data blocks per kernel (default: 64 per worker); kernels
        of fewer than ``inline_below`` element-operations run on the calling
        thread alone."""
        threads = threads or cores()
        blocks = blocks or 64 * threads
        nk = ctypes.c_int64(0)
        rc = _load().mcore_run(self.bases, len(self.arrays), self.views, self.nviews, self.instrs, self.ninstrs,
                               threads, blocks, inline_below, ctypes.byref(nk))
        if rc != 0:
            raise McoreError(f"mcore_run failed ({rc})")
        self.kernels = nk.value
        return self.arrays


def run(program, threads: int | None = None, blocks: int | None = None, instrs=None,
        inline_below: int = 1 << 15) -> dict:
    return Prepared(program, instrs).run(threads, blocks, inline_below)
