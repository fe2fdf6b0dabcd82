"""Parity cases shared by the CPU-emulation tests and the GPU tests: each
case is a seeded bytecode program plus the rule its outputs must satisfy
against the oracle (bit-exact, ulp-bounded, or bounded by rtol * sum|x|
for reordered sums)."""
from __future__ import annotations

import math

import numpy as np

import oracle
from workloads import (Const, ProgramBuilder, blackscholes, bs_inputs, gray_scott, jacobi, knn, montecarlo_pi,
                       shallow_water)

F64_REDUCE_RTOL = 1e-12
F32_REDUCE_RTOL = 1e-5
ULP_TRANSCENDENTAL = 4


def special(dt, n, rng):
    if dt == "float64" or dt == "float32":
        x = rng.standard_normal(n) * np.exp2(rng.integers(-20, 20, n))
        sp = [0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, 5e-324 if dt == "float64" else 1e-45]
        x[: len(sp)] = sp
        return x.astype(dt)
    if dt == "int64":
        x = rng.integers(-(2**62), 2**62, n, dtype=np.int64)
        x[:4] = [0, -1, np.iinfo(np.int64).min, np.iinfo(np.int64).max]
        return x
    return rng.random(n) < 0.5


def positive(dt, n, rng):
    return (np.exp(rng.uniform(-30, 30, n))).astype(dt)


def _ordered(x, dt):
    """Float bit patterns mapped onto a monotone integer line (sign and
    magnitude -> signed integer; both zeros map to 0)."""
    it = np.int64 if dt == "float64" else np.int32
    i = np.asarray(x, dtype=dt).view(it).astype(np.int64)
    mag = i & np.int64((1 << (63 if dt == "float64" else 31)) - 1)
    return np.where(i < 0, -mag, mag)


def ulp_diff(a, b, dt):
    return np.abs(_ordered(a, dt) - _ordered(b, dt))


def assert_exact(got, want, what=""):
    got = np.asarray(got)
    want = np.asarray(want)
    if got.dtype.kind == "f":
        # equal values with equal signs (so signed zeros must match), or both
        # NaN (the sign and payload of a NaN carry no meaning and are not
        # compared: GPU arithmetic returns its canonical NaN)
        same = ((got == want) & (np.signbit(got) == np.signbit(want))) | (np.isnan(got) & np.isnan(want))
    else:
        same = got == want
    if not np.all(same):
        i = int(np.argmin(same))
        raise AssertionError(f"{what}: {np.sum(~same)} mismatches, first at {i}: got {got[i]!r} want {want[i]!r}")


def assert_ulp(got, want, dt, ulps, what=""):
    both_nan = np.isnan(got) & np.isnan(want)
    d = ulp_diff(got, want, dt)
    d[both_nan] = 0
    if np.any(d > ulps):
        i = int(np.argmax(d))
        raise AssertionError(f"{what}: {int(d[i])} ulp at {i}: got {got[i]!r} want {want[i]!r}")


def assert_close_sum(got, want, scale, rtol, what=""):
    err = np.abs(got.astype(np.float64) - want.astype(np.float64))
    bound = rtol * np.maximum(scale, np.finfo(np.float64).tiny)
    bad = ~(err <= bound) & ~(np.isnan(got) & np.isnan(want))
    if np.any(bad):
        i = int(np.argmax(bad))
        raise AssertionError(f"{what}: |{got[i]} - {want[i]}| > {rtol} * {scale[i]}")


# ------------------------------------------------------------------ cases

class Case:
    def __init__(self, name, program, check):
        self.name = name
        self.program = program
        self.check = check  # check(got: dict, want: dict)

    def __repr__(self):
        return self.name


def _exact_check(p):
    def check(got, want):
        for bid in p.outputs:
            assert_exact(got[bid], want[bid], f"{p.name} base {bid}")
    return check


def elementwise_cases(n=1037, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    binary = ["ADD", "SUBTRACT", "MULTIPLY", "MAXIMUM", "MINIMUM"]
    for dt in ("float64", "float32", "int64"):
        for op in binary + (["DIVIDE"] if dt != "int64" else []):
            b = ProgramBuilder(f"{op}_{dt}")
            x = b.base(dt, n, special(dt, n, rng))
            y = b.base(dt, n, special(dt, n, rng)[::-1].copy())
            o = b.base(dt, n)
            b.emit(op, b.whole(o), b.whole(x), b.whole(y))
            p = b.build([o])
            out.append(Case(p.name, p, _exact_check(p)))
        for op in ["ABSOLUTE", "NEGATIVE"]:
            b = ProgramBuilder(f"{op}_{dt}")
            x = b.base(dt, n, special(dt, n, rng))
            o = b.base(dt, n)
            b.emit(op, b.whole(o), b.whole(x))
            p = b.build([o])
            out.append(Case(p.name, p, _exact_check(p)))
        for op in ["LESS", "LESS_EQUAL", "GREATER", "GREATER_EQUAL", "EQUAL", "NOT_EQUAL"]:
            b = ProgramBuilder(f"{op}_{dt}")
            x = b.base(dt, n, special(dt, n, rng))
            y = b.base(dt, n, np.where(rng.random(n) < 0.3, special(dt, n, rng), special(dt, n, rng)[::-1]))
            o = b.base("bool", n)
            b.emit(op, b.whole(o), b.whole(x), b.whole(y))
            p = b.build([o])
            out.append(Case(p.name, p, _exact_check(p)))
    for dt in ("float64", "float32"):
        b = ProgramBuilder(f"SQRT_{dt}")
        x = b.base(dt, n, np.abs(special(dt, n, rng)))
        o = b.base(dt, n)
        b.emit("SQRT", b.whole(o), b.whole(x))
        p = b.build([o])
        out.append(Case(p.name, p, _exact_check(p)))
        for op, gen in (("EXP", lambda: rng.uniform(-80, 80, n)), ("LOG", lambda: positive(dt, n, rng))):
            b = ProgramBuilder(f"{op}_{dt}")
            data = np.asarray(gen(), dtype=dt)
            data[:3] = [0.0, np.inf, np.nan] if op == "EXP" else [1.0, np.inf, 0.0]
            x = b.base(dt, n, data)
            o = b.base(dt, n)
            b.emit(op, b.whole(o), b.whole(x))
            p = b.build([o])

            def chk(got, want, p=p, o=o, dt=dt):
                assert_ulp(got[o], want[o], dt, ULP_TRANSCENDENTAL, p.name)
            out.append(Case(p.name, p, chk))
    # SELECT, CAST, COPY/fill with constants
    for dt in ("float64", "float32", "int64", "bool"):
        b = ProgramBuilder(f"SELECT_{dt}")
        c = b.base("bool", n, rng.random(n) < 0.5)
        x = b.base(dt, n, special(dt, n, rng))
        y = b.base(dt, n, special(dt, n, rng))
        o = b.base(dt, n)
        o2 = b.base(dt, n)
        b.emit("SELECT", b.whole(o), b.whole(c), b.whole(x), b.whole(y))
        b.emit("SELECT", b.whole(o2), b.whole(c), Const(True if dt == "bool" else 3), b.whole(y))
        p = b.build([o, o2])
        out.append(Case(p.name, p, _exact_check(p)))
        for dt2 in ("float64", "float32", "int64", "bool"):
            b = ProgramBuilder(f"CAST_{dt}_{dt2}")
            src = special(dt, n, rng)
            if dt in ("float64", "float32") and dt2 == "int64":
                src = (rng.standard_normal(n) * 1e6).astype(dt)  # inside int64
            x = b.base(dt, n, src)
            o = b.base(dt2, n)
            b.emit("CAST", b.whole(o), b.whole(x))
            p = b.build([o])
            out.append(Case(p.name, p, _exact_check(p)))
        b = ProgramBuilder(f"FILL_{dt}")
        o = b.base(dt, n)
        b.emit("COPY", b.whole(o), Const(1 if dt != "bool" else True))
        p = b.build([o])
        out.append(Case(p.name, p, _exact_check(p)))
    # RANDOM
    b = ProgramBuilder("RANDOM")
    o = b.base("float64", (7, n))
    b.emit("RANDOM", b.whole(o), seed=12345, key=(3 << 32) | 1, step=2)
    p = b.build([o])
    out.append(Case(p.name, p, _exact_check(p)))
    return out


def view_cases(seed=1):
    rng = np.random.default_rng(seed)
    out = []
    N = 67
    data = rng.standard_normal(N * N)
    # shifted, reversed, strided, broadcast, 3-D views into one grid
    b = ProgramBuilder("views2d")
    g = b.base("float64", (N, N), data)
    o1 = b.base("float64", (N - 2, N - 2))
    o2 = b.base("float64", (N, N))
    o3 = b.base("float64", (30, 20))
    o4 = b.base("float64", (5, 7, 9))
    b.emit("ADD", b.whole(o1), b.sub2d(g, 0, N - 2, 1, N - 1), b.sub2d(g, 2, N, 1, N - 1))
    b.emit("SUBTRACT", b.whole(o1), b.whole(o1), b.view(g, N * N - 1, (N - 2, N - 2), (-N, -1)))
    b.emit("MULTIPLY", b.whole(o2), b.whole(g), b.view(g, 3, (N, N), (0, 1)))
    b.emit("COPY", b.whole(o3), b.view(g, 5, (30, 20), (2 * N, 3)))
    b.emit("ADD", b.whole(o4), b.view(g, 11, (5, 7, 9), (N * 9, 1, N)), b.view(g, 0, (5, 7, 9), (0, N, 0)))
    p = b.build([o1, o2, o3, o4])
    out.append(Case(p.name, p, _exact_check(p)))
    # in-place update through identical views, then a partial overlap (staged)
    b = ProgramBuilder("inplace_and_staged")
    a = b.base("float64", 1000, rng.standard_normal(1000))
    b.emit("MULTIPLY", b.whole(a), b.whole(a), Const(2.0))
    b.emit("ADD", b.view(a, 1, (999,), (1,)), b.view(a, 0, (999,), (1,)), Const(1.0))
    b.emit("COPY", b.whole(a), b.view(a, 999, (1000,), (-1,)))
    p = b.build([a])
    out.append(Case(p.name, p, _exact_check(p)))
    # empty views
    b = ProgramBuilder("empty")
    a = b.base("float64", 10, np.arange(10.0))
    o = b.base("float64", 10, np.zeros(10))
    s = b.base("float64", 3)
    b.emit("ADD", b.view(o, 0, (0,), (1,)), b.view(a, 0, (0,), (1,)), Const(1.0))
    b.emit("ADD_REDUCE", b.whole(s), b.view(a, 0, (0, 3), (1, 1)), axis=0)
    p = b.build([o, s])
    out.append(Case(p.name, p, _exact_check(p)))
    # misaligned one-dimensional views (no vector path) and ragged tails
    b = ProgramBuilder("misaligned")
    a = b.base("float32", 4099, rng.standard_normal(4099).astype(np.float32))
    o = b.base("float32", 4099)
    b.emit("ADD", b.view(o, 3, (4093,), (1,)), b.view(a, 1, (4093,), (1,)), b.view(a, 5, (4093,), (1,)))
    b.emit("COPY", b.view(o, 0, (3,), (1,)), Const(0.0))
    b.emit("COPY", b.view(o, 4096, (3,), (1,)), Const(0.0))
    p = b.build([o])
    out.append(Case(p.name, p, _exact_check(p)))
    out += tile_group_cases(seed + 10)
    out += user_op_cases(seed + 20)
    return out


def user_op_cases(seed=21, n=1537):
    """User-defined operations (section "Interface"), fused with ordinary
    bytecodes: one to three inputs, float64 / float32 / int64, a constant
    operand, and use inside a stencil chain."""
    rng = np.random.default_rng(seed)
    out = []
    b = ProgramBuilder("user_ops_mixed")
    x = b.base("float64", n, rng.standard_normal(n))
    y = b.base("float64", n, rng.standard_normal(n))
    z = b.base("float64", n, rng.random(n) + 0.5)
    xf = b.base("float32", n, rng.standard_normal(n).astype(np.float32))
    xi = b.base("int64", n, rng.integers(-1000, 1000, n))
    o1, o2, o3 = b.base("float64", n), b.base("float32", n), b.base("int64", n)
    fma3 = b.user_op("axpy_div", "return (a * b + c) / c;", 3, "float64", lambda a, bb, c: (a * bb + c) / c)
    sq = b.user_op("sq_plus_one", "return a * a + 1.0f;", 1, "float32",
                   lambda a: a * a + np.float32(1.0))
    tri = b.user_op("tri", "return a * (a - 1) / 2 + b;", 2, "int64", lambda a, bb: a * (a - 1) // 2 + bb)
    b.emit(fma3, b.whole(o1), b.whole(x), b.whole(y), b.whole(z))
    b.emit("MULTIPLY", b.whole(o1), b.whole(o1), Const(0.5))
    b.emit(sq, b.whole(o2), b.whole(xf))
    b.emit("ADD", b.whole(o2), b.whole(o2), Const(2.0))
    b.emit(tri, b.whole(o3), b.whole(xi), Const(7))
    p = b.build([o1, o2, o3])
    out.append(Case(p.name, p, _exact_check(p)))
    return out


def tile_group_cases(seed=11, N=37, M=45):
    """Chains of two-dimensional runs handing temporaries to each other at
    small shifts (tile-fused into one kernel): an in-place anchor that each
    point reads only through its own view (no renaming), with RANDOM and
    constants in the producer; a three-run chain with shifts in both
    dimensions writing a separate base; int64 and bool temporaries read
    diagonally; divides with special operands. Sizes are ragged for every
    tile."""
    rng = np.random.default_rng(seed)
    out = []
    b = ProgramBuilder("tile_group_inplace")
    a = b.base("float64", (N, M), rng.standard_normal(N * M))
    c = b.base("float64", (N, M), rng.standard_normal(N * M))
    t = b.base("float64", (N, M - 1))
    r = b.base("float64", (N, M - 1))
    b.emit("SUBTRACT", b.whole(t), b.sub2d(a, 0, N, 1, M), b.sub2d(a, 0, N, 0, M - 1))
    b.emit("RANDOM", b.whole(r), seed=5, key=3)
    b.emit("MULTIPLY", b.whole(t), b.whole(t), b.whole(r))
    b.emit("MULTIPLY", b.whole(t), b.whole(t), Const(0.5))
    cc = b.sub2d(c, 0, N, 1, M - 1)
    b.emit("ADD", cc, cc, b.sub2d(t, 0, N, 1, M - 1))
    b.emit("SUBTRACT", cc, cc, b.sub2d(t, 0, N, 0, M - 2))
    b.discard(t, r)
    p = b.build([c])
    out.append(Case(p.name, p, _exact_check(p)))
    b = ProgramBuilder("tile_group_chain3_float32")
    a = b.base("float32", (N, M), rng.standard_normal(N * M).astype(np.float32))
    o = b.base("float32", (N, M), np.zeros(N * M, np.float32))
    t1 = b.base("float32", (N - 1, M))
    t2 = b.base("float32", (N - 1, M - 1))
    b.emit("ADD", b.whole(t1), b.sub2d(a, 0, N - 1, 0, M), b.sub2d(a, 1, N, 0, M))
    b.emit("MULTIPLY", b.whole(t2), b.sub2d(t1, 0, N - 1, 0, M - 1), b.sub2d(t1, 0, N - 1, 1, M))
    b.emit("SUBTRACT", b.sub2d(o, 0, N - 2, 0, M - 2), b.sub2d(t2, 1, N - 1, 1, M - 1),
           b.sub2d(t2, 0, N - 2, 0, M - 2))
    b.free(t1, t2)
    p = b.build([o])
    out.append(Case(p.name, p, _exact_check(p)))
    # int64 and bool temporaries handed on at row and column shifts (a mask
    # and a SELECT reading them diagonally)
    b = ProgramBuilder("tile_group_int64_bool")
    a = b.base("int64", (N, M), rng.integers(-1000, 1000, N * M))
    o = b.base("int64", (N, M), np.zeros(N * M, np.int64))
    t = b.base("int64", (N - 1, M - 1))
    msk = b.base("bool", (N - 1, M - 1))
    b.emit("ADD", b.whole(t), b.sub2d(a, 0, N - 1, 0, M - 1), b.sub2d(a, 1, N, 1, M))
    b.emit("GREATER", b.whole(msk), b.whole(t), Const(0))
    b.emit("SELECT", b.sub2d(o, 0, N - 2, 0, M - 2), b.sub2d(msk, 1, N - 1, 0, M - 2), b.sub2d(t, 0, N - 2, 1, M - 1),
           b.sub2d(t, 1, N - 1, 1, M - 1))
    b.discard(t, msk)
    p = b.build([o])
    out.append(Case(p.name, p, _exact_check(p)))
    # a producer read 3 rows and 5 columns away (deep histories in the
    # row-sweep form), a stencil input with a 10-column spread, a transposed
    # view and a broadcast row read directly from memory
    b = ProgramBuilder("tile_group_deep_shifts")
    a = b.base("float64", (N, M), rng.standard_normal(N * M))
    bt = b.base("float64", (M, N), rng.standard_normal(N * M))
    row = b.base("float64", (M,), rng.standard_normal(M))
    o = b.base("float64", (N, M), np.zeros(N * M))
    t = b.base("float64", (N - 3, M - 5))
    b.emit("MULTIPLY", b.whole(t), b.sub2d(a, 0, N - 3, 0, M - 5), b.sub2d(a, 3, N, 5, M))
    b.emit("ADD", b.whole(t), b.whole(t), b.view(bt, 0, (N - 3, M - 5), (1, N)))
    ov = b.sub2d(o, 0, N - 6, 0, M - 10)
    b.emit("SUBTRACT", ov, b.sub2d(t, 0, N - 6, 0, M - 10), b.sub2d(t, 3, N - 3, 5, M - 5))
    b.emit("ADD", ov, ov, b.view(row, 0, (N - 6, M - 10), (0, 1)))
    b.discard(t)
    p = b.build([o])
    out.append(Case(p.name, p, _exact_check(p)))
    # divisions with zero numerators and special divisors (zero, subnormal,
    # huge, infinite, NaN) inside a tile-fused group
    for dt in ("float32", "float64"):
        info = np.finfo(dt)
        sp = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, info.tiny / 8, -info.tiny / 1024, info.max / 2, 1.5,
                       -3.0, 2.0 ** -60, -(2.0 ** -61), 2.0 ** 70, 2.0 ** 40], dt)
        num = rng.standard_normal(N * M).astype(dt)
        num[rng.random(N * M) < 0.6] = 0.0
        num[rng.random(N * M) < 0.1] = -0.0
        # tiny numerators, log-uniform from the smallest subnormal to 2^-56
        # (the float32 divide scales those below 2^-60)
        lo = np.log2(info.smallest_subnormal)
        pick = rng.random(N * M) < 0.15
        num[pick] = (np.exp2(rng.uniform(lo, -56.0, pick.sum())) * rng.choice([-1.0, 1.0], pick.sum())).astype(dt)
        den = rng.standard_normal(N * M).astype(dt)
        pick = rng.random(N * M) < 0.3
        den[pick] = sp[rng.integers(0, len(sp), pick.sum())]
        b = ProgramBuilder(f"tile_group_div_{dt}")
        a = b.base(dt, (N, M), num)
        d = b.base(dt, (N, M), den)
        o = b.base(dt, (N, M), np.zeros(N * M, dt))
        t = b.base(dt, (N, M - 1))
        b.emit("DIVIDE", b.whole(t), b.sub2d(a, 0, N, 1, M), b.sub2d(d, 0, N, 0, M - 1))
        b.emit("DIVIDE", b.sub2d(o, 0, N, 0, M - 2), b.sub2d(t, 0, N, 1, M - 1), b.sub2d(d, 0, N, 2, M))
        b.emit("ADD", b.sub2d(o, 0, N, 0, M - 2), b.sub2d(o, 0, N, 0, M - 2), b.sub2d(t, 0, N, 0, M - 2))
        b.discard(t)
        p = b.build([o])
        out.append(Case(p.name, p, _exact_check(p)))
    return out


def _abs_sum(x, axis):
    return np.add.reduce(np.abs(x.astype(np.float64)), axis=axis)


def reduction_cases(shape=(9, 33, 70), seed=2):
    rng = np.random.default_rng(seed)
    out = []
    for dt in ("float64", "float32", "int64"):
        x = special(dt, int(np.prod(shape)), rng) if dt == "int64" else \
            rng.standard_normal(int(np.prod(shape))).astype(dt)
        if dt == "int64":
            x = (x >> 20)
        for op in ("ADD_REDUCE", "MIN_REDUCE", "MAX_REDUCE"):
            for ax in range(3):
                b = ProgramBuilder(f"{op}_{dt}_ax{ax}")
                xb = b.base(dt, shape, x)
                oshape = tuple(s for k, s in enumerate(shape) if k != ax)
                o = b.base(dt, oshape)
                b.emit(op, b.whole(o), b.whole(xb), axis=ax)
                p = b.build([o])
                if op == "ADD_REDUCE" and dt != "int64":
                    scale = _abs_sum(x.reshape(shape), ax).reshape(-1)
                    rtol = F64_REDUCE_RTOL if dt == "float64" else F32_REDUCE_RTOL

                    def chk(got, want, o=o, scale=scale, rtol=rtol, p=p):
                        assert_close_sum(got[o], want[o], scale, rtol, p.name)
                else:
                    chk = _exact_check(p)
                out.append(Case(p.name, p, chk))
    # ARGMIN / ARGMAX: ties (values drawn from a few levels), NaNs and
    # infinities, every axis, a 1-D input (whole-array index) and a long axis
    lv = np.array([0.0, -0.0, 1.0, -1.0, 2.5, np.inf, -np.inf, np.nan])
    for dt in ("float64", "float32", "int64"):
        x = rng.integers(-3, 4, int(np.prod(shape))).astype(dt)
        if dt != "int64":
            sp = rng.random(x.size) < 0.05
            x[sp] = lv[rng.integers(0, len(lv), int(sp.sum()))].astype(dt)
        for op in ("ARGMIN_REDUCE", "ARGMAX_REDUCE"):
            for ax in range(3):
                b = ProgramBuilder(f"{op}_{dt}_ax{ax}")
                xb = b.base(dt, shape, x)
                o = b.base("int64", tuple(s for k, s in enumerate(shape) if k != ax))
                b.emit(op, b.whole(o), b.whole(xb), axis=ax)
                p = b.build([o])
                out.append(Case(p.name, p, _exact_check(p)))
            b = ProgramBuilder(f"{op}_{dt}_1d")
            n1 = 100_003
            xb = b.base(dt, n1, rng.integers(-50, 50, n1).astype(dt))
            o = b.base("int64", 1)
            b.emit(op, b.view(o, 0, (), ()), b.whole(xb), axis=0)
            p = b.build([o])
            out.append(Case(p.name, p, _exact_check(p)))
    # a long reduced axis, inner and outer: a block per output with several
    # elements of each thread in flight at once, ties, NaNs and infinities
    for dt in ("float64", "float32", "int64"):
        rows, cols = 7, 3001
        x = rng.integers(-3, 4, rows * cols).astype(dt)
        if dt != "int64":
            sp = rng.random(x.size) < 0.02
            x[sp] = lv[rng.integers(0, len(lv), int(sp.sum()))].astype(dt)
        for op in ("ARGMIN_REDUCE", "ARGMAX_REDUCE", "MIN_REDUCE", "MAX_REDUCE"):
            for ax, shp in ((1, (rows, cols)), (0, (cols, rows))):
                b = ProgramBuilder(f"{op}_{dt}_long{ax}")
                xb = b.base(dt, shp, x)
                odt = "int64" if op.startswith("ARG") else dt
                o = b.base(odt, rows)
                b.emit(op, b.whole(o), b.whole(xb), axis=ax)
                p = b.build([o])
                out.append(Case(p.name, p, _exact_check(p)))
    # MIN_REDUCE (MAX_REDUCE) followed by ARGMIN_REDUCE (ARGMAX_REDUCE) of the
    # same view over the same axis, run as one pass: ties, NaNs, infinities
    # and zeros of both signs; thread and block per output (rows of 8: a
    # thread per output with 16-byte vector loads). Indices bit-exact;
    # the minimum's value exact, except the sign of a zero minimum where
    # zeros of both signs tie: either zero is the minimum, and which one a
    # fold returns depends on its combining order (the oracle's NumPy
    # reduction included), so that sign is not compared
    for dt in ("float64", "float32", "int64"):
        for shp, ax in (((7, 3001), 1), ((3001, 7), 0), ((9, 33, 70), 2), ((9, 33, 70), 0), ((600, 8), 1)):
            n = int(np.prod(shp))
            x = rng.integers(-2, 3, n).astype(dt)
            if dt != "int64":
                x[rng.random(n) < 0.3] = -0.0
                sp = rng.random(n) < 0.01
                x[sp] = lv[rng.integers(0, len(lv), int(sp.sum()))].astype(dt)
            oshape = tuple(s_ for k, s_ in enumerate(shp) if k != ax)
            for mop, aop in (("MIN_REDUCE", "ARGMIN_REDUCE"), ("MAX_REDUCE", "ARGMAX_REDUCE")):
                b = ProgramBuilder(f"{mop}_{aop}_{dt}_{'x'.join(map(str, shp))}_ax{ax}")
                xb = b.base(dt, shp, x)
                mv = b.base(dt, oshape)
                ix = b.base("int64", oshape)
                b.emit(mop, b.whole(mv), b.whole(xb), axis=ax)
                b.emit(aop, b.whole(ix), b.whole(xb), axis=ax)
                p = b.build([mv, ix])

                def pchk(got, want, mv=mv, ix=ix, p=p):
                    assert_exact(got[ix], want[ix], p.name + " indices")
                    g, w = got[mv], want[mv]
                    same = (g == w) | (np.isnan(g) & np.isnan(w)) if g.dtype.kind == "f" else g == w
                    assert np.all(same), f"{p.name} values: {np.sum(~same)} mismatches"
                out.append(Case(p.name, p, pchk))
    # float32 axis sums at the switch between plain sums (at most 128 terms
    # per output) and compensated ones (129 and more), on data that makes
    # every addition round the same way: 1.0 first, then terms just under
    # half an ulp of 1.0, so a plain sum in order loses each of them. The
    # bound for any order of n - 1 additions is (n - 1) * 2^-24 * sum|x|
    # (about 7.6e-6 at n = 128), inside the 1e-5 tolerance
    tiny = np.float32(np.float64(2.0 ** -24) * (1 - 2.0 ** -10))
    for nred in (128, 129):
        for ax in (1, 0):
            rows = 67
            blk = np.full((rows, nred), tiny, dtype=np.float32)
            blk[:, 0] = 1.0
            blk[1::2, 0] = tiny
            blk[1::2, -1] = 1.0  # odd rows: the large term last
            x = blk if ax == 1 else np.ascontiguousarray(blk.T)
            b = ProgramBuilder(f"ADD_REDUCE_float32_round_{nred}_ax{ax}")
            xb = b.base("float32", x.shape, x)
            o = b.base("float32", rows)
            b.emit("ADD_REDUCE", b.whole(o), b.whole(xb), axis=ax)
            p = b.build([o])
            scale = _abs_sum(x, ax).reshape(-1)

            def rchk(got, want, o=o, scale=scale, p=p):
                assert_close_sum(got[o], want[o], scale, F32_REDUCE_RTOL, p.name)
            out.append(Case(p.name, p, rchk))
    # a MIN_REDUCE (MAX_REDUCE) written into its own input's first column,
    # then the ARGMIN_REDUCE (ARGMAX_REDUCE) of that input: in program order
    # the index is taken over the updated rows (the first element now holds
    # each row's extreme, so the index is 0 unless an earlier tie or NaN)
    for dt in ("float64", "int64"):
        for mop, aop in (("MIN_REDUCE", "ARGMIN_REDUCE"), ("MAX_REDUCE", "ARGMAX_REDUCE")):
            b = ProgramBuilder(f"{mop}_into_input_then_{aop}_{dt}")
            rows, cols = 37, 301
            xb = b.base(dt, (rows, cols), rng.integers(-1000, 1000, rows * cols).astype(dt))
            ix = b.base("int64", rows)
            b.emit(mop, b.view(xb, 0, (rows,), (cols,)), b.whole(xb), axis=1)
            b.emit(aop, b.whole(ix), b.whole(xb), axis=1)
            p = b.build([xb, ix])
            out.append(Case(p.name, p, _exact_check(p)))
    # fused chain with a full reduction and with an axis reduction, plus stores
    for dt in ("float64", "float32"):
        b = ProgramBuilder(f"chain_full_{dt}")
        n = 50_001
        xv = rng.standard_normal(n).astype(dt)
        yv = rng.standard_normal(n).astype(dt)
        x = b.base(dt, n, xv)
        y = b.base(dt, n, yv)
        t = b.base(dt, n)
        s = b.base(dt, 1)
        b.emit("MULTIPLY", b.whole(t), b.whole(x), b.whole(x))
        b.emit("ADD", b.whole(t), b.whole(t), b.whole(y))
        b.emit("ADD_REDUCE", b.view(s, 0, (), ()), b.whole(t), axis=0)
        p = b.build([t, s])
        scale = np.array([np.sum(np.abs(xv.astype(np.float64) ** 2 + yv))])
        rtol = F64_REDUCE_RTOL if dt == "float64" else F32_REDUCE_RTOL

        def chk(got, want, t=t, s=s, scale=scale, rtol=rtol, p=p):
            assert_exact(got[t], want[t], p.name)
            assert_close_sum(got[s], want[s], scale, rtol, p.name)
        out.append(Case(p.name, p, chk))
        b = ProgramBuilder(f"chain_axis_{dt}")
        m = 300
        xv = rng.standard_normal((m, 41)).astype(dt)
        x = b.base(dt, (m, 41), xv)
        t = b.base(dt, (m, 41))
        r0 = b.base(dt, 41)
        b.emit("ABSOLUTE", b.whole(t), b.whole(x))
        b.emit("ADD_REDUCE", b.whole(r0), b.whole(t), axis=0)
        p = b.build([t, r0])
        scale = np.sum(np.abs(xv.astype(np.float64)), axis=0)

        def chk2(got, want, t=t, r0=r0, scale=scale, rtol=rtol, p=p):
            assert_exact(got[t], want[t], p.name)
            assert_close_sum(got[r0], want[r0], scale, rtol, p.name)
        out.append(Case(p.name, p, chk2))
    return out


def knn_check(p, rows=None):
    """kNN results: distances within the reduction tolerance (the squared
    distances are sums of D squares, summed in another order than the
    oracle's); an index may differ from the oracle's only at a near tie,
    i.e. where both points' distances (float64, from the inputs) agree
    within that tolerance; every row's indices are distinct. ``rows``: the
    query rows the oracle computed (a sample of a larger run)."""
    rtol = F64_REDUCE_RTOL if p.meta["dtype"] == "float64" else F32_REDUCE_RTOL
    X = p.bases[p.meta["X"]].init.reshape(p.meta["N"], p.meta["D"]).astype(np.float64)
    Q = p.bases[p.meta["Q"]].init.reshape(p.meta["M"], p.meta["D"]).astype(np.float64)
    k = p.meta["k"]

    def check(got, want):
        """``want``: the oracle's outputs for all rows, or (with ``rows``)
        for a program over the sampled queries only, keyed like ``got``."""
        gd = got[p.meta["dist"]].reshape(-1, k)
        gi = got[p.meta["idx"]].reshape(-1, k)
        sel = np.arange(gd.shape[0]) if rows is None else np.asarray(rows)
        wd = want[p.meta["dist"]].reshape(-1, k)
        wi = want[p.meta["idx"]].reshape(-1, k)
        gd, gi = gd[sel], gi[sel]
        assert_close_sum(gd.reshape(-1), wd.reshape(-1).astype(gd.dtype), np.abs(wd.reshape(-1)).astype(np.float64) + 1e-300,
                         rtol, p.name + " dist")
        for r in range(len(sel)):
            assert len(set(gi[r].tolist())) == k, (p.name, r)
            for j in range(k):
                if gi[r, j] != wi[r, j]:
                    q = Q[sel[r]]
                    da = np.sum((q - X[gi[r, j]]) ** 2)
                    db = np.sum((q - X[wi[r, j]]) ** 2)
                    assert abs(da - db) <= 4 * rtol * max(da, db), (p.name, r, j, gi[r, j], wi[r, j], da, db)
    return check


def jacobi_case(n, iters, one_batch=False):
    """Jacobi on an n x n grid: the grid bit-exact, the deltas within the
    reduction tolerance (with ``one_batch``: every iteration in one batch)."""
    p = jacobi(n, iters, one_batch=one_batch)
    if one_batch:
        p.name += "_one_batch"

    def jchk(got, want, p=p):
        assert_exact(got[p.meta["grid"]], want[p.meta["grid"]], "jacobi grid")
        g0 = p.bases[p.meta["grid"]].init.reshape(n, n)
        assert_close_sum(got[p.meta["deltas"]], want[p.meta["deltas"]],
                         np.full(want[p.meta["deltas"]].size, np.sum(np.abs(g0)) * 2), F64_REDUCE_RTOL, "jacobi deltas")
    return Case(p.name, p, jchk)


def workload_cases(scale="small"):
    out = []
    n = 24 if scale == "small" else 256
    out.append(jacobi_case(n, 3 if scale == "small" else 10))
    out.append(jacobi_case(n, 3 if scale == "small" else 10, one_batch=True))  # the program as one batch
    nb = 3000 if scale == "small" else 100_000
    for dt, rtol in (("float64", 1e-12), ("float32", 1e-5)):
        p = blackscholes(nb, dt, seed=11)
        inp = bs_inputs(nb, "float64", seed=11)
        mx = np.maximum(inp["S"], inp["K"])

        def bchk(got, want, p=p, mx=mx, rtol=rtol):
            for bid in (p.meta["call"], p.meta["put"]):
                err = np.abs(got[bid].astype(np.float64) - want[bid].astype(np.float64))
                assert np.all(err <= rtol * mx), f"{p.name}: max err/max(S,K) {np.max(err / mx)}"
        out.append(Case(p.name, p, bchk))
    N = 18 if scale == "small" else 130
    for dt in ("float64", "float32"):
        p = shallow_water(N, 3 if scale == "small" else 10, dt)
        out.append(Case(p.name, p, _exact_check(p)))
    for dt in ("float64", "float32"):
        # D = 5: rows too short for vector loads; D = 8: 16-byte vector loads
        for p in ([knn(211, 37, 5, 3, dt), knn(97, 29, 8, 2, dt)] if scale == "small"
                  else [knn(2000, 300, 16, 4, dt)]):
            out.append(Case(p.name, p, knn_check(p)))
    R, C = (20, 24) if scale == "small" else (130, 70)
    for dt in ("float64", "float32"):
        p = gray_scott(R, C, 3 if scale == "small" else 10, dt)
        out.append(Case(p.name, p, _exact_check(p)))
    sizes = [1, 37, 1000, 4096, 333] if scale == "small" else \
        np.floor(np.exp2(10 + 8 * np.random.default_rng(3).random(64))).astype(int).tolist()
    p = montecarlo_pi(seed=99, sizes=sizes)
    out.append(Case(p.name, p, _exact_check(p)))
    return out


def all_small_cases():
    return elementwise_cases() + view_cases() + reduction_cases() + workload_cases("small")


def oracle_outputs(program):
    mem = oracle.run(program)
    return {bid: mem[bid] for bid in program.outputs}
