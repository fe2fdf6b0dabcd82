"""Data model for vector-bytecode programs and a small builder.

A program is what the paper's Bridge hands to the Vector Engine Manager: a
batch of vector bytecodes (section "Bytecode": an assembly-like instruction
``op $d, $a, $b`` whose operands are multidimensional arrays) over
array-views of array-bases (section "Numerical Python": a base is a
contiguous allocation, a view selects and re-orders its elements).

This module only describes programs and their seeded inputs. It performs
none of the arithmetic that a bytecode stands for: the oracle and the CUDA
executor each give the mnemonics their meaning in code of their own.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Union

import numpy as np

DTYPES = ("bool", "int64", "float32", "float64")
NP_DTYPE = {
    "bool": np.dtype(np.bool_),
    "int64": np.dtype(np.int64),
    "float32": np.dtype(np.float32),
    "float64": np.dtype(np.float64),
}
ITEMSIZE = {k: v.itemsize for k, v in NP_DTYPE.items()}


@dataclass(frozen=True)
class View:
    """An array-view: ``base[offset + sum_k i_k * strides[k]]`` for
    ``0 <= i_k < shape[k]``. Offset and strides count elements; a stride may
    be 0 (broadcast) or negative (reversed)."""

    base: int
    offset: int
    shape: tuple
    strides: tuple

    @property
    def ndim(self) -> int:
        return len(self.shape)

    @property
    def size(self) -> int:
        n = 1
        for s in self.shape:
            n *= s
        return n


@dataclass(frozen=True)
class Const:
    """A scalar operand in place of one input view. Its value is converted
    to the dtype of the instruction's other inputs."""

    value: Union[int, float, bool]


Operand = Union[View, Const]


@dataclass(frozen=True)
class Instr:
    """One vector bytecode. ``op`` is the mnemonic (e.g. ``"ADD"``).

    ``axis`` is used by the reductions, ``seed``/``key``/``step`` by RANDOM.
    SYNC, DISCARD and FREE take one operand, ``out``, whose base they act on.
    """

    op: str
    out: Optional[View]
    ins: tuple = ()
    axis: int = 0
    seed: int = 0
    key: int = 0
    step: int = 1


@dataclass
class Base:
    dtype: str
    nelem: int
    init: Optional[np.ndarray] = None  # flat host data uploaded before the run
    shape: tuple = ()  # logical shape used by ``whole()``; product == nelem


@dataclass(frozen=True)
class UserOp:
    """A user-defined elementwise operation: ``body`` is the CUDA device
    function body the executor compiles (arguments ``a``, ``b``, ``c``);
    ``fn`` is the same operation written for NumPy arrays of ``dtype``,
    which the oracle runs. The two are written independently."""

    name: str
    body: str
    nin: int
    dtype: str
    fn: object = None


@dataclass
class Program:
    name: str
    bases: dict = field(default_factory=dict)  # id -> Base
    instrs: list = field(default_factory=list)
    outputs: list = field(default_factory=list)  # base ids holding the result
    meta: dict = field(default_factory=dict)
    # user-defined operations used as ``"USER:<name>"``: name -> UserOp
    user_ops: dict = field(default_factory=dict)

    def compulsory_bytes(self) -> int:
        """Live-in bytes read plus live-out bytes written, each once: the
        inputs (bases with host data) plus the declared outputs."""
        nbytes = 0
        for bid, b in self.bases.items():
            if b.init is not None:
                nbytes += b.nelem * ITEMSIZE[b.dtype]
        for bid in self.outputs:
            b = self.bases[bid]
            nbytes += b.nelem * ITEMSIZE[b.dtype]
        return nbytes


def c_strides(shape) -> tuple:
    st = []
    acc = 1
    for s in reversed(shape):
        st.append(acc)
        acc *= s
    return tuple(reversed(st))


class ProgramBuilder:
    """Builds a :class:`Program` with fresh base ids."""

    def __init__(self, name: str):
        self.p = Program(name)
        self._next = 1

    def base(self, dtype: str, shape, init: Optional[np.ndarray] = None) -> int:
        if isinstance(shape, int):
            shape = (shape,)
        shape = tuple(int(s) for s in shape)
        nelem = 1
        for s in shape:
            nelem *= s
        if dtype not in DTYPES:
            raise ValueError(f"unknown dtype {dtype}")
        if init is not None:
            init = np.ascontiguousarray(init, dtype=NP_DTYPE[dtype]).reshape(-1)
            if init.size != nelem:
                raise ValueError("init size does not match base size")
        bid = self._next
        self._next += 1
        self.p.bases[bid] = Base(dtype, nelem, init, shape)
        return bid

    def whole(self, bid: int) -> View:
        b = self.p.bases[bid]
        return View(bid, 0, b.shape, c_strides(b.shape))

    def view(self, bid: int, offset: int, shape, strides) -> View:
        return View(bid, int(offset), tuple(int(s) for s in shape), tuple(int(s) for s in strides))

    def sub2d(self, bid: int, r0: int, r1: int, c0: int, c1: int) -> View:
        """The slice ``base2d[r0:r1, c0:c1]`` of a 2-D base (row-major)."""
        b = self.p.bases[bid]
        rows, cols = b.shape
        assert 0 <= r0 <= r1 <= rows and 0 <= c0 <= c1 <= cols
        return View(bid, r0 * cols + c0, (r1 - r0, c1 - c0), (cols, 1))

    def emit(self, op: str, out: Optional[View], *ins: Operand, axis: int = 0,
             seed: int = 0, key: int = 0, step: int = 1) -> None:
        self.p.instrs.append(Instr(op, out, tuple(ins), axis, seed, key, step))

    def user_op(self, name: str, body: str, nin: int, dtype: str, fn) -> str:
        """Declare a user-defined operation; returns its mnemonic for emit()."""
        self.p.user_ops[name] = UserOp(name, body, nin, dtype, fn)
        return "USER:" + name

    def discard(self, *bids: int) -> None:
        for bid in bids:
            self.emit("DISCARD", self.whole(bid))

    def free(self, *bids: int) -> None:
        for bid in bids:
            self.emit("FREE", self.whole(bid))

    def sync(self, *bids: int) -> None:
        for bid in bids:
            self.emit("SYNC", self.whole(bid))

    def build(self, outputs) -> Program:
        self.p.outputs = list(outputs)
        return self.p
