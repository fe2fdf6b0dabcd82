"""Pins for the oracle's per-bytecode semantics against values fixed by
mathematics, not by the oracle itself: exact rationals for IEEE correct
rounding, mpmath for transcendentals, explicit index loops for views and
reductions, Python integers for wrap-around, a textbook sequential
splitmix64 and its published outputs for RANDOM."""
import math
import os
import struct
from fractions import Fraction

import mpmath
import numpy as np
import pytest

import oracle
from workloads import Const, ProgramBuilder, View

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def run1(op, out_dtype, out_shape, ins, **kw):
    """Run one bytecode; ``ins`` are (dtype, array) pairs or Const."""
    b = ProgramBuilder("one")
    views = []
    for x in ins:
        if isinstance(x, Const):
            views.append(x)
        else:
            dt, arr = x
            arr = np.asarray(arr)
            bid = b.base(dt, arr.shape if arr.ndim else (1,), arr.reshape(-1))
            views.append(b.whole(bid) if arr.ndim else b.view(bid, 0, (), ()))
    ob = b.base(out_dtype, out_shape if out_shape else (1,))
    ov = b.whole(ob) if out_shape else b.view(ob, 0, (), ())
    b.emit(op, ov, *views, **kw)
    p = b.build([ob])
    mem = oracle.run(p)
    return mem[ob].reshape(out_shape)


def rand_doubles(rng, n):
    mant = rng.uniform(-2, 2, n)
    expo = rng.integers(-60, 60, n)
    return np.ldexp(mant, expo)


# ---------------------------------------------------------------- IEEE +-*/

@pytest.mark.parametrize("op,f", [("ADD", lambda a, b: a + b), ("SUBTRACT", lambda a, b: a - b),
                                  ("MULTIPLY", lambda a, b: a * b), ("DIVIDE", lambda a, b: a / b)])
def test_f64_basic_ops_correctly_rounded(op, f):
    rng = np.random.default_rng(1)
    a, b = rand_doubles(rng, 300), rand_doubles(rng, 300)
    got = run1(op, "float64", (300,), [("float64", a), ("float64", b)])
    for x, y, r in zip(a.tolist(), b.tolist(), got.tolist()):
        exact = f(Fraction(x), Fraction(y))
        assert r == float(exact)  # Fraction -> float rounds to nearest, ties to even


def _f32(x: float) -> float:
    return struct.unpack("f", struct.pack("f", x))[0]


@pytest.mark.parametrize("op,f", [("ADD", lambda a, b: a + b), ("SUBTRACT", lambda a, b: a - b),
                                  ("MULTIPLY", lambda a, b: a * b), ("DIVIDE", lambda a, b: a / b)])
def test_f32_basic_ops_correctly_rounded(op, f):
    rng = np.random.default_rng(2)
    a = rand_doubles(rng, 300).astype(np.float32)
    b = rand_doubles(rng, 300).astype(np.float32)
    got = run1(op, "float32", (300,), [("float32", a), ("float32", b)])
    for x, y, r in zip(a.tolist(), b.tolist(), got.tolist()):
        # the exact result rounded once to binary32 (via a Fraction -> double
        # -> float chain; the double step is exact enough for +-*/ of floats,
        # checked here by comparing with the two float32 neighbours)
        exact = f(Fraction(x), Fraction(y))
        cand = np.float32(float(exact))
        lo = np.nextafter(cand, np.float32(-np.inf))
        hi = np.nextafter(cand, np.float32(np.inf))
        err = abs(Fraction(float(cand)) - exact)
        assert err <= abs(Fraction(float(lo)) - exact) and err <= abs(Fraction(float(hi)) - exact)
        assert r == float(cand)


def _is_correct_sqrt(x: float, r: float, dtype) -> bool:
    below = float(np.nextafter(dtype(r), dtype(-np.inf)))
    above = float(np.nextafter(dtype(r), dtype(np.inf)))
    lo = (Fraction(below) + Fraction(r)) / 2
    hi = (Fraction(r) + Fraction(above)) / 2
    X = Fraction(x)
    return lo * lo < X < hi * hi or (X == Fraction(r) ** 2)


@pytest.mark.parametrize("dt", ["float64", "float32"])
def test_sqrt_correctly_rounded(dt):
    rng = np.random.default_rng(3)
    npdt = np.dtype(dt).type
    a = np.abs(rand_doubles(rng, 300)).astype(dt)
    got = run1("SQRT", dt, (300,), [(dt, a)])
    for x, r in zip(a.tolist(), got.tolist()):
        assert _is_correct_sqrt(x, r, npdt)


def test_sqrt_special_values():
    a = np.array([0.0, -0.0, np.inf, -1.0, np.nan, 4.0])
    got = run1("SQRT", "float64", (6,), [("float64", a)])
    assert got[0] == 0.0 and math.copysign(1, got[1]) == -1.0 and got[2] == np.inf
    assert np.isnan(got[3]) and np.isnan(got[4]) and got[5] == 2.0


# ---------------------------------------------------------------- exp, log

def _ulp_err(r, exact_mp, dtype):
    r = dtype(r)
    ulp = float(np.spacing(np.abs(r))) if r != 0 else float(np.finfo(dtype).tiny)
    return abs(mpmath.mpf(float(r)) - exact_mp) / ulp


@pytest.mark.parametrize("dt,tol", [("float64", 1.0), ("float32", 0.51)])
def test_exp_log_within_ulp(dt, tol):
    mpmath.mp.dps = 50
    rng = np.random.default_rng(4)
    npdt = np.dtype(dt).type
    xe = rng.uniform(-30, 30, 400).astype(dt)
    xl = np.exp(rng.uniform(-40, 40, 400)).astype(dt)
    ge = run1("EXP", dt, (400,), [(dt, xe)])
    gl = run1("LOG", dt, (400,), [(dt, xl)])
    for x, r in zip(xe.tolist(), ge.tolist()):
        assert _ulp_err(r, mpmath.exp(mpmath.mpf(x)), npdt) <= tol
    for x, r in zip(xl.tolist(), gl.tolist()):
        assert _ulp_err(r, mpmath.log(mpmath.mpf(x)), npdt) <= tol


def test_exp_log_special_values():
    ge = run1("EXP", "float64", (4,), [("float64", np.array([0.0, -np.inf, np.inf, 1000.0]))])
    assert ge.tolist() == [1.0, 0.0, np.inf, np.inf]
    gl = run1("LOG", "float64", (4,), [("float64", np.array([1.0, 0.0, np.inf, -1.0]))])
    assert gl[0] == 0.0 and gl[1] == -np.inf and gl[2] == np.inf and np.isnan(gl[3])


# ---------------------------------------------------------------- others

def test_compare_ieee_with_nan():
    a = np.array([1.0, 2.0, np.nan, 3.0, -0.0])
    b = np.array([2.0, 2.0, 1.0, np.nan, 0.0])
    py = {"LESS": lambda x, y: x < y, "LESS_EQUAL": lambda x, y: x <= y,
          "GREATER": lambda x, y: x > y, "GREATER_EQUAL": lambda x, y: x >= y,
          "EQUAL": lambda x, y: x == y, "NOT_EQUAL": lambda x, y: x != y}
    for op, f in py.items():
        got = run1(op, "bool", (5,), [("float64", a), ("float64", b)])
        assert got.tolist() == [f(x, y) for x, y in zip(a.tolist(), b.tolist())], op


def test_maximum_minimum_nan_and_zero():
    a = np.array([1.0, np.nan, 2.0, -0.0, 0.0])
    b = np.array([2.0, 1.0, np.nan, 0.0, -0.0])
    mx = run1("MAXIMUM", "float64", (5,), [("float64", a), ("float64", b)])
    mn = run1("MINIMUM", "float64", (5,), [("float64", a), ("float64", b)])
    assert mx[0] == 2.0 and np.isnan(mx[1]) and np.isnan(mx[2])
    assert mn[0] == 1.0 and np.isnan(mn[1]) and np.isnan(mn[2])
    # reading: MAXIMUM(a, b) = a if (a > b or a is NaN) else b, so a tie
    # between signed zeros yields the second operand (likewise MINIMUM)
    assert math.copysign(1, mx[3]) == 1 and math.copysign(1, mx[4]) == -1
    assert math.copysign(1, mn[3]) == 1 and math.copysign(1, mn[4]) == -1


def test_select_and_const_operands():
    c = np.array([True, False, True, False])
    a = np.array([1.0, 2.0, 3.0, 4.0])
    got = run1("SELECT", "float64", (4,), [("bool", c), ("float64", a), Const(-1.5)])
    assert got.tolist() == [1.0, -1.5, 3.0, -1.5]
    got = run1("SUBTRACT", "float64", (4,), [Const(1.0), ("float64", a)])
    assert got.tolist() == [0.0, -1.0, -2.0, -3.0]
    # a float32 constant is the float64 literal rounded once to float32
    got = run1("MULTIPLY", "float32", (1,), [("float32", np.array([1.0], np.float32)), Const(0.1)])
    assert got[0] == _f32(0.1)


def test_cast_rules():
    d = np.array([1.9, -1.9, 0.0, 2.5, -0.0, 1e10])
    assert run1("CAST", "int64", (6,), [("float64", d)]).tolist() == [math.trunc(x) for x in d]
    assert run1("CAST", "bool", (6,), [("float64", d)]).tolist() == [x != 0 for x in d]
    bo = np.array([True, False, True])
    assert run1("CAST", "int64", (3,), [("bool", bo)]).tolist() == [1, 0, 1]
    big = np.array([2**53 + 1, -(2**62) - 1, 3], dtype=np.int64)
    assert run1("CAST", "float64", (3,), [("int64", big)]).tolist() == [float(int(x)) for x in big]
    rng = np.random.default_rng(5)
    x = rand_doubles(rng, 200)
    assert run1("CAST", "float32", (200,), [("float64", x)]).tolist() == [_f32(v) for v in x]


def test_int64_wraps():
    M = 1 << 64

    def wrap(v):
        v %= M
        return v - M if v >= 1 << 63 else v

    a = np.array([2**62, -(2**63), 7, 2**40 + 3], dtype=np.int64)
    b = np.array([2**62, -1, -9, 2**40 + 5], dtype=np.int64)
    for op, f in (("ADD", lambda x, y: x + y), ("SUBTRACT", lambda x, y: x - y),
                  ("MULTIPLY", lambda x, y: x * y)):
        got = run1(op, "int64", (4,), [("int64", a), ("int64", b)])
        assert got.tolist() == [wrap(f(int(x), int(y))) for x, y in zip(a, b)], op
    got = run1("NEGATIVE", "int64", (4,), [("int64", a)])
    assert got.tolist() == [wrap(-int(x)) for x in a]
    got = run1("ABSOLUTE", "int64", (4,), [("int64", a)])
    assert got.tolist() == [wrap(abs(int(x))) for x in a]


def test_dtype_rules_rejected():
    with pytest.raises(oracle.OracleError):
        run1("DIVIDE", "int64", (2,), [("int64", np.array([1, 2])), ("int64", np.array([1, 2]))])
    with pytest.raises(oracle.OracleError):
        run1("EXP", "int64", (2,), [("int64", np.array([1, 2]))])
    with pytest.raises(oracle.OracleError):
        run1("ADD", "float64", (2,), [("float32", np.array([1, 2], np.float32)),
                                       ("float32", np.array([1, 2], np.float32))])


# ---------------------------------------------------------------- views

def _brute_view(base, v: View):
    out = np.empty(v.shape, dtype=base.dtype)
    for idx in np.ndindex(*v.shape):
        out[idx] = base[v.offset + sum(i * s for i, s in zip(idx, v.strides))]
    return out


def test_views_match_index_loops():
    rng = np.random.default_rng(6)
    data = rng.random(400)
    cases = [View(1, 0, (20, 20), (20, 1)), View(1, 21, (18, 18), (20, 1)),
             View(1, 399, (10, 10), (-20, -1)), View(1, 5, (4, 7), (0, 3)),
             View(1, 50, (3, 4, 5), (60, 1, 11)), View(1, 7, (), ()), View(1, 0, (0, 5), (5, 1))]
    for v in cases:
        b = ProgramBuilder("v")
        bid = b.base("float64", 400, data)
        assert bid == 1
        ob = b.base("float64", max(v.size, 1))
        ov = b.view(ob, 0, v.shape, tuple(int(s) for s in np.cumprod((1,) + v.shape[:0:-1])[::-1])
                    if v.shape else ())
        b.emit("COPY", ov, v)
        got = oracle.run(b.build([ob]))[ob][: v.size].reshape(v.shape)
        assert np.array_equal(got, _brute_view(data, v)), v


def test_view_out_of_bounds_rejected():
    b = ProgramBuilder("oob")
    a = b.base("float64", 10, np.zeros(10))
    o = b.base("float64", 10)
    b.emit("COPY", b.whole(o), b.view(a, 1, (10,), (1,)))
    with pytest.raises(oracle.OracleError):
        oracle.run(b.build([o]))
    b = ProgramBuilder("oob2")
    a = b.base("float64", 10, np.zeros(10))
    o = b.base("float64", 10)
    b.emit("COPY", b.view(o, 0, (5,), (1,)), b.view(a, 3, (5,), (-1,)))
    with pytest.raises(oracle.OracleError):
        oracle.run(b.build([o]))


def test_self_overlapping_output_rejected():
    b = ProgramBuilder("ovl")
    a = b.base("float64", 10, np.zeros(10))
    b.emit("COPY", b.view(a, 0, (5,), (0,)), Const(1.0))
    with pytest.raises(oracle.OracleError):
        oracle.run(b.build([a]))


def test_partial_overlap_reads_inputs_first():
    # a[1:] = a[:-1] + 1 reads the old a, as if copied first
    data = np.arange(10, dtype=np.float64)
    b = ProgramBuilder("shift")
    a = b.base("float64", 10, data)
    b.emit("ADD", b.view(a, 1, (9,), (1,)), b.view(a, 0, (9,), (1,)), Const(1.0))
    got = oracle.run(b.build([a]))[a]
    want = list(data)
    snap = list(data)
    for i in range(1, 10):
        want[i] = snap[i - 1] + 1
    assert got.tolist() == want
    # reversed in place: a = a[::-1]
    b = ProgramBuilder("rev")
    a = b.base("float64", 10, data)
    b.emit("COPY", b.whole(a), b.view(a, 9, (10,), (-1,)))
    assert oracle.run(b.build([a]))[a].tolist() == data[::-1].tolist()


def test_broadcast_view_is_repetition():
    row = np.array([1.0, 2.0, 3.0])
    b = ProgramBuilder("bc")
    r = b.base("float64", 3, row)
    m = b.base("float64", (4, 3), np.arange(12.0))
    o = b.base("float64", (4, 3))
    b.emit("ADD", b.whole(o), b.whole(m), b.view(r, 0, (4, 3), (0, 1)))
    got = oracle.run(b.build([o]))[o].reshape(4, 3)
    for i in range(4):
        for j in range(3):
            assert got[i, j] == 3 * i + j + row[j]


# ---------------------------------------------------------------- reductions

def test_add_reduce_f64_against_fsum():
    rng = np.random.default_rng(7)
    x = rng.standard_normal((13, 17, 11))
    for ax in range(3):
        shp = tuple(s for k, s in enumerate(x.shape) if k != ax)
        got = run1("ADD_REDUCE", "float64", shp, [("float64", x)], axis=ax)
        want = np.moveaxis(x, ax, -1)
        for idx in np.ndindex(*shp):
            vals = want[idx].tolist()
            assert abs(got[idx] - math.fsum(vals)) <= 1e-14 * math.fsum(abs(v) for v in vals)


def test_add_reduce_f32_accumulates_wide():
    x = np.full(1 << 20, 0.1, dtype=np.float32)
    got = run1("ADD_REDUCE", "float32", (), [("float32", x)], axis=0)
    exact = Fraction(float(np.float32(0.1))) * (1 << 20)
    assert float(got) == _f32(float(exact))


def test_add_reduce_int_wraps_and_min_max():
    a = np.array([[2**62, 2**62, 5], [-3, 4, -(2**63)]], dtype=np.int64)
    got = run1("ADD_REDUCE", "int64", (3,), [("int64", a)], axis=0)
    M = 1 << 64
    for j in range(3):
        s = (int(a[0, j]) + int(a[1, j])) % M
        assert int(got[j]) == (s - M if s >= 1 << 63 else s)
    got = run1("ADD_REDUCE", "int64", (2,), [("int64", a)], axis=1)
    for i in range(2):
        s = sum(int(v) for v in a[i]) % M
        assert int(got[i]) == (s - M if s >= 1 << 63 else s)
    f = np.array([[3.0, -1.0, 7.0], [2.0, np.nan, 0.5]])
    mx = run1("MAX_REDUCE", "float64", (2,), [("float64", f)], axis=1)
    mn = run1("MIN_REDUCE", "float64", (3,), [("float64", f)], axis=0)
    assert mx[0] == 7.0 and np.isnan(mx[1])
    assert mn[0] == 2.0 and np.isnan(mn[1]) and mn[2] == 0.5


def test_reduce_empty_axis():
    z = np.zeros((0, 3))
    got = run1("ADD_REDUCE", "float64", (3,), [("float64", z)], axis=0)
    assert got.tolist() == [0.0, 0.0, 0.0]
    with pytest.raises(oracle.OracleError):
        run1("MAX_REDUCE", "float64", (3,), [("float64", z)], axis=0)


# ---------------------------------------------------------------- RANDOM

def _seq_splitmix(seed, count):
    M = (1 << 64) - 1
    s = seed & M
    out = []
    for _ in range(count):
        s = (s + 0x9E3779B97F4A7C15) & M
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        out.append(z ^ (z >> 31))
    return out


def test_splitmix_published_values():
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        want = [int(line, 16) for line in f if line.strip() and not line.startswith("#")]
    got = oracle.mix64(np.array([(k + 1) * oracle.GAMMA % (1 << 64) for k in range(4)],
                                dtype=np.uint64))
    assert [int(v) for v in got] == want
    assert _seq_splitmix(0, 4) == want


def test_random_is_sequential_stream_interleaved():
    seed = 987654321
    seq = _seq_splitmix(seed, 40)
    x = run1("RANDOM", "float64", (20,), [], seed=seed, key=0, step=2)
    y = run1("RANDOM", "float64", (20,), [], seed=seed, key=1, step=2)
    assert x.tolist() == [(seq[2 * m] >> 11) * 2.0**-53 for m in range(20)]
    assert y.tolist() == [(seq[2 * m + 1] >> 11) * 2.0**-53 for m in range(20)]
    # a 2-D output numbers its elements in row-major order
    z = run1("RANDOM", "float64", (4, 5), [], seed=seed, key=0, step=1)
    assert z.reshape(-1).tolist() == [(seq[m] >> 11) * 2.0**-53 for m in range(20)]


def test_user_operation_dispatch():
    """A user-defined operation runs its NumPy definition on the views, with
    the arithmetic rules' dtype checks: compared with a per-element loop."""
    from workloads import ProgramBuilder
    rng = np.random.default_rng(9)
    b = ProgramBuilder("user")
    x = b.base("float64", (6, 5), rng.standard_normal(30))
    y = b.base("float64", (6, 5), rng.standard_normal(30))
    o = b.base("float64", (6, 5))
    op = b.user_op("hyp", "return a * a + b * b;", 2, "float64", lambda a, c: a * a + c * c)
    b.emit(op, b.whole(o), b.view(x, 29, (6, 5), (-5, -1)), b.whole(y))
    p = b.build([o])
    got = oracle.run(p)[o]
    xs, ys = p.bases[x].init, p.bases[y].init
    want = [xs[29 - k] * xs[29 - k] + ys[k] * ys[k] for k in range(30)]
    assert got.tolist() == want
    bad = b.base("float32", (6, 5), np.zeros(30, np.float32))
    b.emit(op, b.whole(o), b.whole(bad), b.whole(y))
    with pytest.raises(oracle.OracleError):
        oracle.run(b.build([o]))


def _arg_loop(row, maxi):
    """Index of the first best element of a list, a NaN being best."""
    best = None
    for j, x in enumerate(row):
        if best is None:
            best = j
            continue
        v = row[best]
        if math.isnan(v):
            continue
        if math.isnan(x) or (x > v if maxi else x < v):
            best = j
    return best


@pytest.mark.parametrize("op", ["ARGMIN_REDUCE", "ARGMAX_REDUCE"])
def test_argmin_argmax_first_occurrence_and_nan(op):
    """Brute force over rows with ties, NaNs and infinities, along each axis
    of a 2-D view and of a reversed view."""
    from workloads import ProgramBuilder
    rng = np.random.default_rng(4)
    vals = np.array([0.0, -0.0, 1.0, -1.0, 2.0, np.inf, -np.inf, np.nan])
    data = vals[rng.integers(0, len(vals), 7 * 9)]
    for axis in (0, 1):
        b = ProgramBuilder("arg")
        x = b.base("float64", (7, 9), data)
        o = b.base("int64", 9 if axis == 0 else 7)
        b.emit(op, b.whole(o), b.view(x, 62, (7, 9), (-9, -1)), axis=axis)
        p = b.build([o])
        got = oracle.run(p)[o].tolist()
        m = data.reshape(7, 9)[::-1, ::-1]
        rows = [list(m[:, j]) for j in range(9)] if axis == 0 else [list(m[i, :]) for i in range(7)]
        assert got == [_arg_loop(r, op == "ARGMAX_REDUCE") for r in rows]


# ------------------------------------------------- SYNC / DISCARD / FREE
#
# Section "Vector Engine Manager": sync asks for read access, so the copy the
# host reads must be the most recent one (the oracle's host memory is the
# only copy: the values stay as they are); discard declares every other copy
# invalid (the oracle's base has no defined contents until it is written
# again, which it shows as a sentinel: NaN for floats, a fixed int64, True
# for bool); release (FREE) ends the base (any later use is an error).

def _ctl_program(ctl, dtype="float64", via_subview=False):
    b = ProgramBuilder("ctl")
    init = np.arange(12, dtype=np.float64).reshape(3, 4) * 1.5 - 4.0
    if dtype == "int64":
        init = np.arange(12, dtype=np.int64).reshape(3, 4) * 7 - 30
    x = b.base(dtype, (3, 4), init)
    y = b.base(dtype, (3, 4))
    b.emit("ADD", b.whole(y), b.whole(x), b.whole(x))
    # the control instruction names its base through any view of it
    cv = b.view(y, 5, (2, 2), (4, 1)) if via_subview else b.whole(y)
    b.emit(ctl, cv)
    return b, x, y, init


@pytest.mark.parametrize("via_subview", [False, True])
@pytest.mark.parametrize("dtype", ["float64", "int64"])
def test_sync_leaves_values_unchanged(dtype, via_subview):
    b, x, y, init = _ctl_program("SYNC", dtype, via_subview)
    z = b.base(dtype, (3, 4))
    b.emit("COPY", b.whole(z), b.whole(y))
    mem = oracle.run(b.build([y, z]))
    want = [v + v for v in init.reshape(-1).tolist()]
    assert mem[y].tolist() == want and mem[z].tolist() == want
    assert mem[x].tolist() == init.reshape(-1).tolist()


@pytest.mark.parametrize("via_subview", [False, True])
def test_discard_makes_every_element_undefined(via_subview):
    """A read after DISCARD sees no stale value: every element of the base,
    including those outside the naming view, reads as the sentinel."""
    b, x, y, init = _ctl_program("DISCARD", "float64", via_subview)
    z = b.base("float64", (3, 4))
    b.emit("COPY", b.whole(z), b.whole(y))
    mem = oracle.run(b.build([y, z]))
    assert all(math.isnan(v) for v in mem[z].tolist())
    assert all(math.isnan(v) for v in mem[y].tolist())
    assert mem[x].tolist() == init.reshape(-1).tolist()  # other bases untouched


def test_discard_int_and_bool_sentinels():
    b, x, y, init = _ctl_program("DISCARD", "int64")
    mem = oracle.run(b.build([y]))
    assert mem[y].tolist() == [-(2**63) + 12345] * 12
    b = ProgramBuilder("ctlb")
    f = b.base("float64", (5,), np.array([1.0, -1.0, 0.0, 2.0, -3.0]))
    m = b.base("bool", (5,))
    b.emit("GREATER", b.whole(m), b.whole(f), Const(0.0))
    b.emit("DISCARD", b.whole(m))
    assert oracle.run(b.build([m]))[m].tolist() == [True] * 5


def test_write_after_discard_is_live_again():
    b, x, y, init = _ctl_program("DISCARD")
    b.emit("MULTIPLY", b.whole(y), b.whole(x), Const(3.0))
    mem = oracle.run(b.build([y]))
    assert mem[y].tolist() == [v * 3.0 for v in init.reshape(-1).tolist()]


@pytest.mark.parametrize("use", ["read", "write", "SYNC", "DISCARD", "FREE"])
def test_any_use_after_free_raises(use):
    b, x, y, init = _ctl_program("FREE")
    z = b.base("float64", (3, 4))
    if use == "read":
        b.emit("COPY", b.whole(z), b.whole(y))
    elif use == "write":
        b.emit("COPY", b.whole(y), b.whole(x))
    else:
        b.emit(use, b.whole(y))
    with pytest.raises(oracle.OracleError):
        oracle.run(b.build([z]))


def test_free_removes_only_its_base():
    b, x, y, init = _ctl_program("FREE")
    mem = oracle.run(b.build([x]))
    assert y not in mem
    assert mem[x].tolist() == init.reshape(-1).tolist()


def test_control_of_a_base_never_created_raises():
    b = ProgramBuilder("ctl0")
    x = b.base("float64", (4,), np.zeros(4))
    for op in ("SYNC", "DISCARD", "FREE"):
        p = b.build([x])
        p.instrs = [oracle_instr(op, 999)]
        with pytest.raises(oracle.OracleError):
            oracle.run(p)


def oracle_instr(op, bid):
    from workloads.program import Instr
    return Instr(op, View(bid, 0, (4,), (1,)))
