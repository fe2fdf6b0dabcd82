"""Reference interpreter: executes a bytecode program one instruction at a
time, in order, on NumPy arrays in the host's memory.

Test infrastructure only (see the package docstring).

Semantics followed, by section of the paper:

* "Bytecode": one opcode per mnemonic; the opcode fixes the operand count;
  operands are multidimensional array-views.
* "Numerical Python": a view is ``base[offset + sum_k i_k * strides[k]]``
  over a contiguous array-base; here it is built with ``as_strided`` on the
  base buffer.
* "Vector Engine" (design): instructions obey their serialisation order, so
  the interpreter simply runs them in order.
* "Vector Engine Manager": SYNC, DISCARD and FREE manage ownership. Here
  SYNC is a no-op (host memory is the only copy), DISCARD marks the
  contents of a base undefined (filled with a sentinel so that a later read
  shows up), FREE removes the base.

Readings where the paper is silent (each listed in the design notes):

* an instruction whose output view partially overlaps an input view reads
  its inputs as if they had been copied first;
* float32 transcendental functions are evaluated in float64 and rounded
  once to float32; float32 reductions accumulate in float64 and round once;
* integer arithmetic wraps modulo 2^64;
* a float -> int64 CAST truncates toward zero (values outside int64 are not
  defined);
* MAXIMUM(a, b) is ``a`` if ``a > b`` or ``a`` is NaN, else ``b`` (NumPy's
  ``maximum``: NaN propagates, a tie of signed zeros gives ``b``); MINIMUM
  likewise with ``<``; MIN/MAX_REDUCE fold the same rule, except that when
  the extreme is a zero present with both signs the sign of the result
  depends on the combining order (NumPy's reduction of a contiguous axis
  does not combine sequentially), so it is not part of the result.
"""
from __future__ import annotations

import warnings

import numpy as np
from numpy.lib.stride_tricks import as_strided

from workloads.program import NP_DTYPE, Const, Program, View

from .splitmix import random_u01

ARITH = {"ADD", "SUBTRACT", "MULTIPLY", "MAXIMUM", "MINIMUM"}
FLOAT_BINARY = {"DIVIDE"}
FLOAT_UNARY = {"SQRT", "EXP", "LOG"}
SIGNED_UNARY = {"ABSOLUTE", "NEGATIVE"}
COMPARE = {"LESS", "LESS_EQUAL", "GREATER", "GREATER_EQUAL", "EQUAL", "NOT_EQUAL"}
REDUCE = {"ADD_REDUCE", "MIN_REDUCE", "MAX_REDUCE", "ARGMIN_REDUCE", "ARGMAX_REDUCE"}
CONTROL = {"SYNC", "DISCARD", "FREE"}

NUMERIC = {"int64", "float32", "float64"}
FLOATS = {"float32", "float64"}


class OracleError(ValueError):
    pass


def _sentinel(dtype: np.dtype):
    if dtype.kind == "f":
        return np.nan
    if dtype.kind == "b":
        return True
    return np.iinfo(np.int64).min + 12345


class Memory:
    """Base arrays of a program, held as flat NumPy buffers."""

    def __init__(self, program: Program):
        self.dtype = {}
        self.buf = {}
        self.user_ops = getattr(program, "user_ops", {})
        for bid, b in program.bases.items():
            dt = NP_DTYPE[b.dtype]
            self.dtype[bid] = dt
            if b.init is not None:
                self.buf[bid] = np.array(b.init, dtype=dt, copy=True).reshape(-1)
            else:
                self.buf[bid] = np.full(b.nelem, _sentinel(dt), dtype=dt)

    def view(self, v: View) -> np.ndarray:
        """``as_strided`` view of base ``v.base`` after checking that every
        element it reaches lies inside the base."""
        if v.base not in self.buf:
            raise OracleError(f"base {v.base} is not live")
        buf = self.buf[v.base]
        if len(v.shape) != len(v.strides):
            raise OracleError("shape and strides differ in length")
        if any(s < 0 for s in v.shape):
            raise OracleError("negative extent")
        if min(v.shape, default=1) > 0:
            lo = v.offset + sum(min(0, (n - 1) * s) for n, s in zip(v.shape, v.strides))
            hi = v.offset + sum(max(0, (n - 1) * s) for n, s in zip(v.shape, v.strides))
            if lo < 0 or hi >= buf.size:
                raise OracleError(f"view reaches [{lo}, {hi}] outside base of {buf.size}")
            start = buf[v.offset:]
        else:
            start = buf[: 0]
        isz = buf.itemsize
        return as_strided(start, shape=v.shape, strides=tuple(s * isz for s in v.strides),
                          writeable=True)


def _self_overlapping(v: View) -> bool:
    """True if two distinct indices of ``v`` can reach the same element,
    decided by the sufficient condition that, with dimensions sorted by
    |stride|, each |stride| exceeds the span of the smaller ones."""
    if v.size <= 1:
        return False
    dims = sorted((abs(s), n) for n, s in zip(v.shape, v.strides) if n > 1)
    span = 0
    for s, n in dims:
        if s <= span:
            return True
        span += s * (n - 1)
    return False


def _operand(mem: Memory, x, dtype: np.dtype) -> np.ndarray:
    if isinstance(x, Const):
        if dtype.kind == "b":
            return np.array(bool(x.value))
        if dtype.kind == "i":
            return np.array(int(x.value), dtype=dtype)
        return np.array(float(x.value), dtype=np.float64).astype(dtype)
    # a private copy: the instruction reads its inputs as if copied first
    return np.array(mem.view(x), copy=True)


def _in_dtype(mem: Memory, ins, default):
    for x in ins:
        if isinstance(x, View):
            return mem.dtype[x.base]
    return default


def execute(mem: Memory, ins_) -> None:
    """Execute one bytecode on ``mem``."""
    op, out = ins_.op, ins_.out
    if op in CONTROL:
        if out is None:
            raise OracleError(f"{op} needs a base")
        bid = out.base
        if bid not in mem.buf:
            raise OracleError(f"{op} of a base that is not live")
        if op == "DISCARD":
            mem.buf[bid][...] = _sentinel(mem.dtype[bid])
        elif op == "FREE":
            del mem.buf[bid]
        return
    if out is None:
        raise OracleError(f"{op} needs an output")
    if _self_overlapping(out):
        raise OracleError("output view overlaps itself")
    o = mem.view(out)
    odt = mem.dtype[out.base]
    ins = ins_.ins
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        if op == "RANDOM":
            if odt != np.float64 or ins:
                raise OracleError("RANDOM writes float64 and has no inputs")
            m = np.arange(out.size, dtype=np.uint64).reshape(out.shape)
            o[...] = random_u01(ins_.seed, ins_.key, ins_.step, m)
            return
        if op in REDUCE:
            (x,) = ins
            if not isinstance(x, View):
                raise OracleError("reduction input must be a view")
            a = _operand(mem, x, mem.dtype[x.base])
            ax = ins_.axis
            if not (0 <= ax < a.ndim):
                raise OracleError("reduction axis out of range")
            if op in ("ARGMIN_REDUCE", "ARGMAX_REDUCE"):
                # NumPy's argmin/argmax: the first occurrence of the minimum
                # (maximum); a NaN counts as the minimum (maximum), so the
                # first NaN wins
                if odt != np.int64 or a.dtype.kind not in "if":
                    raise OracleError("argmin/argmax reads a number and writes int64")
                if tuple(np.delete(np.array(a.shape, dtype=np.int64), ax)) != tuple(out.shape):
                    raise OracleError("reduction output shape")
                if a.shape[ax] == 0:
                    raise OracleError("argmin/argmax over an empty axis")
                f = np.argmin if op == "ARGMIN_REDUCE" else np.argmax
                o[...] = f(a, axis=ax).astype(np.int64)
                return
            if a.dtype != odt or odt.kind not in "if":
                raise OracleError("reduction dtype")
            if tuple(np.delete(np.array(a.shape, dtype=np.int64), ax)) != tuple(out.shape):
                raise OracleError("reduction output shape")
            if op == "ADD_REDUCE":
                if odt == np.float32:
                    r = np.add.reduce(a.astype(np.float64), axis=ax).astype(np.float32)
                else:
                    r = np.add.reduce(a, axis=ax, dtype=odt)
            else:
                if a.shape[ax] == 0:
                    raise OracleError("min/max reduction over an empty axis")
                f = np.minimum if op == "MIN_REDUCE" else np.maximum
                r = f.reduce(a, axis=ax)
            o[...] = r
            return
        idt = _in_dtype(mem, ins, odt)
        if op in ("CAST",):
            (x,) = ins
            a = _operand(mem, x, idt)
            if odt.kind == "b":
                o[...] = a != 0
            else:
                o[...] = a.astype(odt)
            return
        args = []
        for k, x in enumerate(ins):
            if op == "SELECT" and k == 0:
                args.append(_operand(mem, x, np.dtype(np.bool_)))
            elif op == "SELECT":
                args.append(_operand(mem, x, odt))
            else:
                args.append(_operand(mem, x, idt))
        for a in args:
            if a.ndim and tuple(a.shape) != tuple(out.shape):
                raise OracleError(f"{op}: input shape {a.shape} != output shape {out.shape}")
        if op == "COPY":
            if idt != odt:
                raise OracleError("COPY keeps the dtype")
            o[...] = args[0]
        elif op == "SELECT":
            if args[0].dtype != np.bool_:
                raise OracleError("SELECT condition must be bool")
            o[...] = np.where(args[0], args[1], args[2])
        elif op in COMPARE:
            if odt.kind != "b":
                raise OracleError("comparisons write bool")
            f = {"LESS": np.less, "LESS_EQUAL": np.less_equal, "GREATER": np.greater,
                 "GREATER_EQUAL": np.greater_equal, "EQUAL": np.equal,
                 "NOT_EQUAL": np.not_equal}[op]
            o[...] = f(args[0], args[1])
        elif op in ARITH or op in FLOAT_BINARY:
            if idt != odt or odt.name not in NUMERIC:
                raise OracleError(f"{op} dtype")
            if op in FLOAT_BINARY and odt.name not in FLOATS:
                raise OracleError("DIVIDE needs a float dtype")
            f = {"ADD": np.add, "SUBTRACT": np.subtract, "MULTIPLY": np.multiply,
                 "DIVIDE": np.divide, "MAXIMUM": np.maximum, "MINIMUM": np.minimum}[op]
            o[...] = f(args[0], args[1], dtype=odt)
        elif op in FLOAT_UNARY:
            if idt != odt or odt.name not in FLOATS:
                raise OracleError(f"{op} needs a float dtype")
            f = {"SQRT": np.sqrt, "EXP": np.exp, "LOG": np.log}[op]
            if odt == np.float32 and op != "SQRT":
                o[...] = f(args[0].astype(np.float64)).astype(np.float32)
            else:
                o[...] = f(args[0])
        elif op in SIGNED_UNARY:
            if idt != odt or odt.name not in NUMERIC:
                raise OracleError(f"{op} dtype")
            o[...] = (np.absolute if op == "ABSOLUTE" else np.negative)(args[0])
        elif op.startswith("USER:"):
            # section "Interface": a registered user-defined operation,
            # run through its NumPy definition
            u = mem.user_ops.get(op[5:])
            if u is None:
                raise OracleError(f"unknown user operation {op}")
            if len(args) != u.nin or any(a.dtype != np.dtype(u.dtype) for a in args) or odt != np.dtype(u.dtype):
                raise OracleError(f"{op}: operands must be {u.nin} x {u.dtype}")
            r = np.asarray(u.fn(*args))
            if r.dtype != odt:
                raise OracleError(f"{op}: the NumPy definition returned {r.dtype}, not {odt}")
            o[...] = r
        else:
            raise OracleError(f"unknown opcode {op}")


def run(program: Program, instrs=None) -> dict:
    """Run ``program`` (or the instruction list ``instrs`` over its bases)
    and return ``{base id: flat array}`` for the bases still live."""
    mem = Memory(program)
    for ins_ in (program.instrs if instrs is None else instrs):
        execute(mem, ins_)
    return mem.buf
