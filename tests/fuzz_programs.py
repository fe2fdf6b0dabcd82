"""Seeded random bytecode programs for differential testing against the oracle.

A program works on a few small 9 x 11 bases (float64, int64, bool) through
random views of them: sub-blocks, rows or columns reversed (negative
strides), transposed (column stride 1, row stride 11), every other row,
broadcast rows (zero stride, inputs only), so consecutive instructions
overlap, alias in place, partially overlap their own inputs and depend on
each other through every kind of view; this is what the paper's blockable
rule and the library's fusion breaks, staging and pairing have to get
right. The bytecodes are the exact ones (add, subtract, multiply, divide,
maximum, minimum, negative, absolute, square root, compares, select, copy,
cast of small integers, min/max/argmin/argmax reductions over either axis,
int64 sums), so every result must equal the oracle's bit for bit; the one
documented relaxation is the sign of a zero chosen by a MIN/MAX reduction
from tied signed zeros. Reductions write bases that no later instruction
reads, so no reordering tolerance is needed anywhere.

The other generators: ``random_stencil_program`` makes random stencil
chains that the library turns into tile-fused groups, to be run in every
group form (optionally ending in MIN/MAX reductions, as a Jacobi sweep
does); ``random_reduce_chain_program`` makes programs whose later
instructions read reduction results back through broadcasts;
``random_nd_program`` works on views of rank 1 to 5. ``random_program``
also draws float32 programs (``fdt``).
"""
from __future__ import annotations

import numpy as np

from parity_cases import Case, assert_exact
from workloads import Const, ProgramBuilder

R, C = 9, 11
SHAPES = [(3, 4), (4, 7), (5, 5), (9, 2), (2, 11), (1, 6), (6, 1), (9, 11), (7, 9)]


def _view(b, rng, bid, h, w, broadcast_ok):
    """A random view of shape (h, w) of the R x C base ``bid``."""
    for _ in range(50):
        kind = int(rng.integers(0, 6 if broadcast_ok else 5))
        if kind == 0 and h <= R and w <= C:  # sub-block
            r0, c0 = rng.integers(0, R - h + 1), rng.integers(0, C - w + 1)
            return b.view(bid, r0 * C + c0, (h, w), (C, 1))
        if kind == 1 and h <= R and w <= C:  # columns reversed
            r0, c0 = rng.integers(0, R - h + 1), rng.integers(0, C - w + 1)
            return b.view(bid, r0 * C + c0 + w - 1, (h, w), (C, -1))
        if kind == 2 and h <= R and w <= C:  # rows reversed
            r0, c0 = rng.integers(0, R - h + 1), rng.integers(0, C - w + 1)
            return b.view(bid, (r0 + h - 1) * C + c0, (h, w), (-C, 1))
        if kind == 3 and h <= C and w <= R:  # transposed: (i, j) -> base[r0 + j, c0 + i]
            r0, c0 = rng.integers(0, R - w + 1), rng.integers(0, C - h + 1)
            return b.view(bid, r0 * C + c0, (h, w), (1, C))
        if kind == 4 and 2 * (h - 1) < R and w <= C:  # every other row
            r0, c0 = rng.integers(0, R - 2 * (h - 1)), rng.integers(0, C - w + 1)
            return b.view(bid, r0 * C + c0, (h, w), (2 * C, 1))
        if kind == 5 and w <= C:  # one row, broadcast down
            r0, c0 = rng.integers(0, R), rng.integers(0, C - w + 1)
            return b.view(bid, r0 * C + c0, (h, w), (0, 1))
    raise AssertionError("no view fits")


def random_program(seed: int, fdt: str = "float64"):
    """``fdt`` is the floating type of the float bases (float32 programs
    draw the same instructions; their divides and square roots are
    correctly rounded in float32, so they too are exact)."""
    rng = np.random.default_rng(1000 + seed)
    b = ProgramBuilder(f"fuzz{seed}" + ("" if fdt == "float64" else "_f32"))
    n = R * C
    F = [b.base(fdt, (R, C), rng.standard_normal(n) * np.exp2(rng.integers(-3, 4, n))) for _ in range(3)]
    I = [b.base("int64", (R, C), rng.integers(-50, 50, n)) for _ in range(2)]
    B = b.base("bool", (R, C), rng.random(n) < 0.5)
    red = b.base(fdt, (64,), np.zeros(64))
    redi = b.base("int64", (64,), np.zeros(64, np.int64))

    def fv(h, w, bc=True):
        return _view(b, rng, F[rng.integers(0, 3)], h, w, bc)

    def iv(h, w, bc=True):
        return _view(b, rng, I[rng.integers(0, 2)], h, w, bc)

    def red_out(bid, m):
        return b.view(bid, int(rng.integers(0, 64 - m + 1)), (m,), (1,))

    for _ in range(int(rng.integers(8, 21))):
        h, w = SHAPES[rng.integers(0, len(SHAPES))]
        k = int(rng.integers(0, 10))
        if k <= 2:  # float binary
            op = ["ADD", "SUBTRACT", "MULTIPLY", "DIVIDE", "MAXIMUM", "MINIMUM"][rng.integers(0, 6)]
            y = Const(float(np.round(rng.standard_normal(), 3))) if rng.random() < 0.25 else fv(h, w)
            b.emit(op, fv(h, w, False), fv(h, w), y)
        elif k == 3:  # float unary
            op = ["NEGATIVE", "ABSOLUTE", "COPY"][rng.integers(0, 3)]
            b.emit(op, fv(h, w, False), fv(h, w))
        elif k == 4:  # square root of a magnitude, in place
            o = fv(h, w, False)
            b.emit("ABSOLUTE", o, fv(h, w))
            b.emit("SQRT", o, o)
        elif k == 5:  # int64
            op = ["ADD", "SUBTRACT", "MAXIMUM", "MINIMUM"][rng.integers(0, 4)]
            b.emit(op, iv(h, w, False), iv(h, w), iv(h, w) if rng.random() < 0.7 else Const(int(rng.integers(-9, 9))))
        elif k == 6:  # compare, then select
            cmpop = ["LESS", "GREATER", "LESS_EQUAL", "EQUAL"][rng.integers(0, 4)]
            m = _view(b, rng, B, h, w, False)
            b.emit(cmpop, m, fv(h, w), fv(h, w))
            b.emit("SELECT", fv(h, w, False), _view(b, rng, B, h, w, True), fv(h, w), fv(h, w))
        elif k == 7:  # casts of small integers both ways
            b.emit("CAST", fv(h, w, False), iv(h, w))
            if rng.random() < 0.5:
                b.emit("CAST", iv(h, w, False), _view(b, rng, B, h, w, True))
        elif k == 8:  # min/max/argmin/argmax reductions (sometimes a MIN then ARGMIN pair)
            ax = int(rng.integers(0, 2))
            m = (h, w)[1 - ax]
            x = fv(h, w)
            op = ["MIN_REDUCE", "MAX_REDUCE"][rng.integers(0, 2)]
            b.emit(op, red_out(red, m), x, axis=ax)
            if rng.random() < 0.6:
                b.emit("ARGMIN_REDUCE" if op == "MIN_REDUCE" else "ARGMAX_REDUCE", red_out(redi, m), x, axis=ax)
        else:  # int64 sums (exact)
            ax = int(rng.integers(0, 2))
            b.emit("ADD_REDUCE", red_out(redi, (h, w)[1 - ax]), iv(h, w), axis=ax)
    outs = F + I + [B, red, redi]
    p = b.build(outs)

    def check(got, want):
        for bid in outs:
            if bid == red:
                # MIN/MAX of tied signed zeros may return either zero (see
                # the readings of the paper): values compared, NaN as NaN
                g, wv = np.asarray(got[bid]), np.asarray(want[bid])
                same = (g == wv) | (np.isnan(g) & np.isnan(wv))
                assert np.all(same), f"{p.name} reductions: got {g[~same][:4]} want {wv[~same][:4]}"
            else:
                assert_exact(got[bid], want[bid], f"{p.name} base {bid}")
    return Case(p.name, p, check)


def fuzz_cases(seeds, fdt: str = "float64"):
    return [random_program(s, fdt) for s in seeds]


def random_reduce_chain_program(seed: int):
    """Random programs in which later instructions read what reductions
    wrote: int64 sums and ARGMIN/ARGMAX indices (exact in any combining
    order) land in a 64-element int64 base, and later int64 operations,
    compares, selects and casts read them through row or column broadcasts
    (stride 0 along one axis) of that base, then feed further reductions.
    Every reduction result read later is a dependency through a reduction,
    which fusion must break and packing must not put into one launch with
    its reader. MIN/MAX values go to a float64 base that nothing reads (the
    sign of a zero chosen from tied signed zeros is not fixed)."""
    rng = np.random.default_rng(9000 + seed)
    b = ProgramBuilder(f"fuzz_redchain{seed}")
    n = R * C
    F = [b.base("float64", (R, C), rng.standard_normal(n) * np.exp2(rng.integers(-3, 4, n))) for _ in range(2)]
    I = [b.base("int64", (R, C), rng.integers(-50, 50, n)) for _ in range(2)]
    B = b.base("bool", (R, C), rng.random(n) < 0.5)
    redi = b.base("int64", (64,), rng.integers(-20, 20, 64))
    redf = b.base("float64", (64,), np.zeros(64))

    def fv(h, w, bc=True):
        return _view(b, rng, F[rng.integers(0, 2)], h, w, bc)

    def iv(h, w, bc=True):
        return _view(b, rng, I[rng.integers(0, 2)], h, w, bc)

    def red_out(bid, m):
        return b.view(bid, int(rng.integers(0, 64 - m + 1)), (m,), (1,))

    def red_in(h, w):
        """redi read as an (h, w) array: a row repeated down, or a column
        repeated across"""
        if rng.random() < 0.5:
            return b.view(redi, int(rng.integers(0, 64 - w + 1)), (h, w), (0, 1))
        return b.view(redi, int(rng.integers(0, 64 - h + 1)), (h, w), (1, 0))

    for _ in range(int(rng.integers(10, 24))):
        h, w = SHAPES[rng.integers(0, len(SHAPES))]
        k = int(rng.integers(0, 8))
        if k <= 1:  # int64 sums over either axis into redi
            ax = int(rng.integers(0, 2))
            b.emit("ADD_REDUCE", red_out(redi, (h, w)[1 - ax]), iv(h, w), axis=ax)
        elif k == 2:  # argmin/argmax into redi, sometimes paired with its MIN/MAX
            ax = int(rng.integers(0, 2))
            m = (h, w)[1 - ax]
            x = fv(h, w)
            if rng.random() < 0.5:
                b.emit(["MIN_REDUCE", "MAX_REDUCE"][rng.integers(0, 2)], red_out(redf, m), x, axis=ax)
            b.emit(["ARGMIN_REDUCE", "ARGMAX_REDUCE"][rng.integers(0, 2)], red_out(redi, m), x, axis=ax)
        elif k <= 4:  # int64 arithmetic on reduction results
            op = ["ADD", "SUBTRACT", "MAXIMUM", "MINIMUM"][rng.integers(0, 4)]
            y = red_in(h, w) if rng.random() < 0.6 else iv(h, w)
            b.emit(op, iv(h, w, False), red_in(h, w) if rng.random() < 0.5 else iv(h, w), y)
        elif k == 5:  # compare with a reduction result, then select
            m = _view(b, rng, B, h, w, False)
            b.emit(["LESS", "GREATER_EQUAL", "EQUAL"][rng.integers(0, 3)], m, iv(h, w), red_in(h, w))
            b.emit("SELECT", iv(h, w, False), m, red_in(h, w), iv(h, w))
        elif k == 6:  # a reduction result into float64 arithmetic (exact: small integers)
            o = fv(h, w, False)
            b.emit("CAST", o, red_in(h, w))
            b.emit(["ADD", "MULTIPLY", "SUBTRACT"][rng.integers(0, 3)], o, o, fv(h, w))
        else:  # in place on redi itself: a slice updated from another slice
            m = int(rng.integers(1, 12))
            b.emit(["ADD", "SUBTRACT"][rng.integers(0, 2)], red_out(redi, m), red_out(redi, m), red_out(redi, m))
    outs = F + I + [B, redi, redf]
    p = b.build(outs)

    def check(got, want):
        for bid in outs:
            if bid == redf:
                g, wv = np.asarray(got[bid]), np.asarray(want[bid])
                same = (g == wv) | (np.isnan(g) & np.isnan(wv))
                assert np.all(same), f"{p.name} MIN/MAX values: got {g[~same][:4]} want {wv[~same][:4]}"
            else:
                assert_exact(got[bid], want[bid], f"{p.name} base {bid}")
    return Case(p.name, p, check)


def reduce_chain_cases(seeds):
    return [random_reduce_chain_program(s) for s in seeds]


LAYOUT = (3, 4, 5, 6)  # the n-D generator's bases, row-major
LSTR = (120, 30, 6, 1)


def _nd_view(b, rng, bid, shape, broadcast_ok):
    """A random view of the given shape (rank 1 to 5) of a LAYOUT base:
    each dimension walks a distinct base axis (in any order, forwards or
    backwards, every element or every other one when it fits) or, for
    inputs, repeats (stride 0); base axes left over sit at a random index."""
    for _ in range(200):
        axes = list(rng.permutation(4))
        off, strides, used = 0, [], []
        ok = True
        for n in shape:
            if broadcast_ok and rng.random() < 0.15:
                strides.append(0)
                continue
            cand = [a for a in axes if a not in used and LAYOUT[a] >= n]
            if not cand:
                ok = False
                break
            a = int(cand[rng.integers(0, len(cand))])
            used.append(a)
            step = 2 if (rng.random() < 0.3 and 2 * (n - 1) < LAYOUT[a]) else 1
            span = step * (n - 1)
            start = int(rng.integers(0, LAYOUT[a] - span))
            if rng.random() < 0.35:  # backwards
                off += (start + span) * LSTR[a]
                strides.append(-step * LSTR[a])
            else:
                off += start * LSTR[a]
                strides.append(step * LSTR[a])
        if not ok:
            continue
        for a in range(4):
            if a not in used:
                off += int(rng.integers(0, LAYOUT[a])) * LSTR[a]
        return b.view(bid, off, tuple(shape), tuple(strides))
    raise AssertionError("no view fits")


def random_nd_program(seed: int, fdt: str = "float64"):
    """Random exact programs over views of rank 1 to 5 of 3 x 4 x 5 x 6
    bases: dimensions in any order of the base axes, reversed, strided by
    two, broadcast (stride 0, inputs only), so the library's merging of
    dimensions, its general (non-vector) tile path and reductions over
    inner, middle and outer axes of such views are compared with the
    oracle bit for bit (int64 sums; MIN/MAX/ARGMIN/ARGMAX; a zero chosen
    from tied signed zeros by MIN/MAX compared by value)."""
    rng = np.random.default_rng(13000 + seed)
    b = ProgramBuilder(f"fuzz_nd{seed}" + ("" if fdt == "float64" else "_f32"))
    n = int(np.prod(LAYOUT))
    F = [b.base(fdt, LAYOUT, rng.standard_normal(n) * np.exp2(rng.integers(-3, 4, n))) for _ in range(2)]
    I = [b.base("int64", LAYOUT, rng.integers(-50, 50, n)) for _ in range(2)]
    B = b.base("bool", LAYOUT, rng.random(n) < 0.5)
    red = b.base(fdt, (256,), np.zeros(256))
    redi = b.base("int64", (256,), np.zeros(256, np.int64))

    def shape():
        r = int(rng.integers(1, 6))
        return tuple(int(rng.integers(1, 7)) for _ in range(r))

    def fv(S, bc=True):
        return _nd_view(b, rng, F[rng.integers(0, 2)], S, bc)

    def iv(S, bc=True):
        return _nd_view(b, rng, I[rng.integers(0, 2)], S, bc)

    def red_out(bid, S):
        """a contiguous (or, when there are two or more dims, transposed) view of S elements"""
        m = int(np.prod(S)) if S else 1
        if m > 256:
            raise AssertionError("result does not fit")
        off = int(rng.integers(0, 256 - m + 1))
        st = [0] * len(S)
        acc = 1
        order = list(range(len(S)))[::-1] if rng.random() < 0.7 else list(rng.permutation(len(S)))
        for k in order:
            st[k] = acc
            acc *= S[k]
        return b.view(bid, off, tuple(S) if S else (1,), tuple(st) if S else (1,))

    for _ in range(int(rng.integers(8, 18))):
        S = shape()
        k = int(rng.integers(0, 9))
        try:
            if k <= 2:
                op = ["ADD", "SUBTRACT", "MULTIPLY", "MAXIMUM", "MINIMUM", "DIVIDE"][rng.integers(0, 6)]
                y = Const(float(np.round(rng.standard_normal(), 3))) if rng.random() < 0.2 else fv(S)
                b.emit(op, fv(S, False), fv(S), y)
            elif k == 3:
                b.emit(["NEGATIVE", "ABSOLUTE", "COPY"][rng.integers(0, 3)], fv(S, False), fv(S))
            elif k == 4:
                op = ["ADD", "SUBTRACT", "MAXIMUM", "MINIMUM"][rng.integers(0, 4)]
                b.emit(op, iv(S, False), iv(S), iv(S))
            elif k == 5:
                m = _nd_view(b, rng, B, S, False)
                b.emit(["LESS", "GREATER", "EQUAL"][rng.integers(0, 3)], m, fv(S), fv(S))
                b.emit("SELECT", fv(S, False), _nd_view(b, rng, B, S, True), fv(S), fv(S))
            elif k == 6:
                b.emit("CAST", fv(S, False), iv(S))
            elif k == 7 and len(S) >= 2:  # min/max/argmin/argmax over any axis
                ax = int(rng.integers(0, len(S)))
                R_ = S[:ax] + S[ax + 1:]
                x = fv(S)
                op = ["MIN_REDUCE", "MAX_REDUCE"][rng.integers(0, 2)]
                b.emit(op, red_out(red, R_), x, axis=ax)
                if rng.random() < 0.6:
                    b.emit("ARGMIN_REDUCE" if op == "MIN_REDUCE" else "ARGMAX_REDUCE", red_out(redi, R_), x, axis=ax)
            elif len(S) >= 2:  # int64 sums over any axis
                ax = int(rng.integers(0, len(S)))
                b.emit("ADD_REDUCE", red_out(redi, S[:ax] + S[ax + 1:]), iv(S), axis=ax)
        except AssertionError:
            continue  # no view of that shape fits: draw another instruction
    outs = F + I + [B, red, redi]
    p = b.build(outs)

    def check(got, want):
        for bid in outs:
            if bid == red:
                g, wv = np.asarray(got[bid]), np.asarray(want[bid])
                same = (g == wv) | (np.isnan(g) & np.isnan(wv))
                assert np.all(same), f"{p.name} reductions: got {g[~same][:4]} want {wv[~same][:4]}"
            else:
                assert_exact(got[bid], want[bid], f"{p.name} base {bid}")
    return Case(p.name, p, check)


def nd_cases(seeds, fdt: str = "float64"):
    return [random_nd_program(s, fdt) for s in seeds]


def random_stencil_program(seed: int, reduce: bool = False):
    """A random stencil chain that the library fuses into one tile-fused
    group: 2 to 4 runs, each computing a temporary from the previous one
    (or the input) read at random row and column shifts of 0 to 3, with
    random exact operations and constants; later runs may read the input
    again at a shift; the last run writes a separate output or updates the
    input in place (renamed while the group reads it around). Temporaries
    are discarded, and the chain runs twice, so the second pass reads what
    the first renamed. Sizes are random (23 to 70), float64 or float32.

    With ``reduce`` each pass ends, as a Jacobi sweep does, with a MIN or
    MAX of one of its arrays along the rows and then of those results to a
    scalar (exact in any order; a zero chosen from tied signed zeros is
    compared by value). Those choices draw from a second generator, so the
    chains themselves are the same as without."""
    rng = np.random.default_rng(5000 + seed)
    rng2 = np.random.default_rng(7000 + seed)
    dt = ["float64", "float32"][rng.integers(0, 2)]
    R0, C0 = (int(x) for x in rng.integers(23, 71, 2))
    b = ProgramBuilder(f"fuzz_stencil{seed}_{dt}" + ("_red" if reduce else ""))
    A = b.base(dt, (R0, C0), (rng.standard_normal(R0 * C0) * 2.0).astype(dt))
    O = b.base(dt, (R0, C0), np.zeros(R0 * C0, dt))
    S = b.base(dt, (4,), np.zeros(4, dt)) if reduce else None
    nruns = int(rng.integers(2, 5))
    in_place = bool(rng.random() < 0.5)
    ops = ["ADD", "SUBTRACT", "MULTIPLY", "MAXIMUM", "MINIMUM", "DIVIDE"]
    plan = []  # per run: (shift range, ops, extra reads)
    for j in range(nruns):
        plan.append(dict(mdr=int(rng.integers(0, 4)), mdc=int(rng.integers(0, 4)),
                         op1=ops[rng.integers(0, 6)], op2=ops[rng.integers(0, 5)],
                         s3=(rng.random(), rng.random()), k=float(np.round(rng.uniform(0.5, 2.0), 2)),
                         second=int(rng.integers(0, 3)), reread=bool(rng.random() < 0.4),
                         ao=(rng.random(), rng.random())))
    for ps in range(2):
        prev, (pr, pc) = A, (R0, C0)
        temps = []
        arrays = []  # (view, rows) of every array the pass writes
        for j, q in enumerate(plan):
            Rj, Cj = pr - q["mdr"], pc - q["mdc"]
            last = j == nruns - 1
            if last:
                tgt = A if in_place else O
                a0 = int(q["ao"][0] * (R0 - Rj + 1))
                c0 = int(q["ao"][1] * (C0 - Cj + 1))
                out = b.sub2d(tgt, a0, a0 + Rj, c0, c0 + Cj)
            else:
                t = b.base(dt, (Rj, Cj))
                temps.append(t)
                out = b.whole(t)
            d3r = int(q["s3"][0] * (q["mdr"] + 1))
            d3c = int(q["s3"][1] * (q["mdc"] + 1))
            b.emit(q["op1"], out, b.sub2d(prev, 0, Rj, 0, Cj), b.sub2d(prev, q["mdr"], pr, q["mdc"], pc))
            if q["second"] == 1:
                b.emit(q["op2"], out, out, Const(q["k"]))
            elif q["second"] == 2:
                b.emit(q["op2"], out, out, b.sub2d(prev, d3r, d3r + Rj, d3c, d3c + Cj))
            if q["reread"] and j > 0:  # the input again, shifted
                b.emit("ADD", out, out, b.sub2d(A, d3r, d3r + Rj, d3c, d3c + Cj))
            arrays.append((out, Rj))
            prev, (pr, pc) = (t if not last else None), (Rj, Cj)
        if reduce:
            x, rows = arrays[int(rng2.integers(0, len(arrays)))]
            op = ["MIN_REDUCE", "MAX_REDUCE"][rng2.integers(0, 2)]
            rt = b.base(dt, (rows,))
            temps.append(rt)
            b.emit(op, b.whole(rt), x, axis=1)
            b.emit(op, b.view(S, ps, (), ()), b.whole(rt), axis=0)
        b.discard(*temps)
    p = b.build([A, O, S] if reduce else [A, O])
    exact = _exact_outputs(p)

    def check(got, want):
        if not reduce:
            return exact(got, want)
        for bid in (A, O):
            assert_exact(got[bid], want[bid], f"{p.name} base {bid}")
        g, wv = np.asarray(got[S]), np.asarray(want[S])
        same = (g == wv) | (np.isnan(g) & np.isnan(wv))
        assert np.all(same), f"{p.name} reductions: got {g} want {wv}"
    return Case(p.name, p, check)


def _exact_outputs(p):
    def check(got, want):
        for bid in p.outputs:
            assert_exact(got[bid], want[bid], f"{p.name} base {bid}")
    return check


def stencil_cases(seeds, reduce: bool = False):
    return [random_stencil_program(s, reduce) for s in seeds]
