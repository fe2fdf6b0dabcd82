"""Host-side tests of libvbe: the library loads and exports every entry
point the header declares; the analysis and the code generator work on a
host-only context (no GPU): fusion decisions, staging of partially
overlapping operands, validation errors, the overlap test against NumPy,
and NVRTC compilation of every kernel the workloads need."""
import ctypes
import json
import os
import re

import numpy as np
import pytest

from paper_1210_7774_b300 import build

build.build()

from paper_1210_7774_b300 import vbe as V  # noqa: E402
from paper_1210_7774_b300.runner import Executor  # noqa: E402
from workloads import (Const, ProgramBuilder, View, blackscholes, jacobi, montecarlo_pi,  # noqa: E402
                       shallow_water)
from parity_cases import tile_group_cases  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HOST = V.VBE_HOST_ONLY


def header_functions():
    txt = open(os.path.join(ROOT, "include", "vbe.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(vbe_\w+)\s*\(", txt, flags=re.M)))


def test_every_declared_function_is_exported():
    names = header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(V.lib, n), n
    assert set(names) == set(V.EXPORTED)


def test_strerror_and_errors_table():
    for code, name in V.ERRORS.items():
        assert V.vbe_strerror(code)
    assert V.vbe_strerror(-999) == "unknown error"


def runs_of(ex, L, batch=0):
    js = json.loads(ex.plan(L, batch))
    return [i["run"] for i in js["items"] if "run" in i], js


@pytest.fixture
def fused():
    ex = Executor(V.VBE_FUSE | V.VBE_PACK | HOST)
    yield ex
    ex.close()


@pytest.fixture
def plain():
    ex = Executor(HOST)
    yield ex
    ex.close()


def test_jacobi_iteration_is_one_tile_fused_kernel(fused):
    """The stencil run (with its merged reduction) and the copy back become
    one kernel: t stays in shared memory, the grid is renamed (the stencil
    reads it around every point), each point reduced exactly once."""
    p = jacobi(16, 2)
    L = fused.load(p, upload=False)
    js = json.loads(fused.plan(L, 0))
    groups = [i["group"] for i in js["items"] if "group" in i]
    assert len(groups) == 1 and not [i for i in js["items"] if "run" in i]
    g = groups[0]
    assert [r["box"] for r in g["runs"]] == [[0, 0, 0, 0], [0, 0, 0, 0]]
    assert g["renamed"] == [L.base[p.meta["grid"]]]


def test_jacobi_iteration_fuses_into_reduction_and_copy():
    p = jacobi(16, 2)
    fused = Executor(V.VBE_FUSE | V.VBE_PACK | V.VBE_NO_TILE_FUSION | HOST)
    L = fused.load(p, upload=False)
    runs, _ = runs_of(fused, L)
    assert [r["mode"] for r in runs] == ["full_reduce", "elementwise"]
    first = runs[0]
    assert first["ops"] == ["ADD", "ADD", "ADD", "MULTIPLY", "SUBTRACT", "ABSOLUTE"]
    assert first["reduce"]["axes"] == [0, 1]  # row sums then their sum
    t_id = list(p.bases)[1]  # bases: full grid, t, d, r, deltas
    assert first["stores"] == [L.base[t_id]]  # d and r stay in registers
    assert runs[1]["ops"] == ["COPY"]
    fused.close()


def test_plain_path_is_one_run_per_bytecode(plain):
    p = blackscholes(100)
    L = plain.load(p, upload=False)
    runs, _ = runs_of(plain, L)
    compute = [i for i in p.instrs if i.op not in ("SYNC", "DISCARD", "FREE")]
    assert len(runs) == len(compute)
    assert all(len(r["ops"]) == 1 for r in runs)


def test_blackscholes_is_one_kernel_with_two_stores(fused):
    p = blackscholes(1000)
    L = fused.load(p, upload=False)
    runs, _ = runs_of(fused, L)
    assert len(runs) == 1
    r = runs[0]
    assert len(r["loads"]) == 5 and len(r["stores"]) == 2
    assert r["vector"] is True


def test_shallow_water_step_runs():
    p = shallow_water(12, 1)
    with Executor(V.VBE_FUSE | V.VBE_PACK | V.VBE_NO_TILE_FUSION | HOST) as ex:
        L = ex.load(p, upload=False)
        runs, _ = runs_of(ex, L)
        # ghost columns, ghost rows, cell fluxes, x faces, y faces, update
        assert [len(r["ops"]) for r in runs] == [6, 6, 9, 21, 21, 18]
        # the in-place update reads and writes the same interior views
        assert sorted(set(runs[-1]["stores"])) == sorted(L.base[k] for k in (p.meta["H"], p.meta["U"], p.meta["V"]))


def test_shallow_water_step_is_one_tile_fused_group(fused):
    """Cell fluxes, both half steps and the update become one kernel: the
    fluxes and face values stay in shared memory (halo margins 2, 1, 1
    around the update's tile), only H, U, V are written, and they are
    renamed because the earlier runs read them around every point."""
    N = 12
    p = shallow_water(N, 1)
    L = fused.load(p, upload=False)
    js = json.loads(fused.plan(L, 0))
    kinds = ["group" if "group" in i else ("run" if "run" in i else "action") for i in js["items"]]
    assert kinds[:3] == ["run", "run", "group"] and set(kinds[3:]) == {"action"}
    g = js["items"][2]["group"]
    n = N - 2
    assert [r["shape"] for r in g["runs"]] == [[N, N], [n + 1, n], [n, n + 1], [n, n]]
    assert [r["box"] for r in g["runs"]] == [[0, 2, 0, 2], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 0, 0]]
    hv = sorted(L.base[k] for k in (p.meta["H"], p.meta["U"], p.meta["V"]))
    assert sorted(g["renamed"]) == hv
    assert all(s["shared"] for r in g["runs"][:-1] for s in r["stores"])
    assert sorted(s["base"] for s in g["runs"][-1]["stores"]) == hv
    # every value read from shared memory comes from an earlier run at a shift of at most one
    for k, r in enumerate(g["runs"]):
        for ld in r["loads"]:
            if ld["from"] >= 0:
                assert ld["from"] < k and all(0 <= d <= 1 for d in ld["shift"])


def test_tile_fusion_needs_dead_temporaries(fused):
    """A temporary that is still live after the chain (no DISCARD) must reach
    memory, so its producer stays a separate kernel."""
    def chain(discard):
        b = ProgramBuilder("live_temp")
        a = b.base("float64", (20, 20), np.zeros(400))
        t = b.base("float64", (19, 20))
        o = b.base("float64", (18, 20))
        b.emit("ADD", b.whole(t), b.sub2d(a, 0, 19, 0, 20), b.sub2d(a, 1, 20, 0, 20))
        b.emit("SUBTRACT", b.whole(o), b.sub2d(t, 1, 19, 0, 20), b.sub2d(t, 0, 18, 0, 20))
        if discard:
            b.discard(t)
        return b.build([o] if discard else [o, t])

    for discard, groups in ((False, 0), (True, 1)):
        L = fused.load(chain(discard), upload=False)
        js = json.loads(fused.plan(L, 0))
        assert sum("group" in i for i in js["items"]) == groups


def test_montecarlo_instances_keep_everything_in_registers(fused):
    p = montecarlo_pi(sizes=[100, 200, 300])
    L = fused.load(p, upload=False)
    runs, _ = runs_of(fused, L)
    assert len(runs) == 3
    for r in runs:
        assert r["loads"] == [] and r["stores"] == [] and r["mode"] == "full_reduce"


def test_partial_overlap_is_staged(fused):
    b = ProgramBuilder("shift")
    a = b.base("float64", 10, np.arange(10.0))
    b.emit("ADD", b.view(a, 1, (9,), (1,)), b.view(a, 0, (9,), (1,)), Const(1.0))
    p = b.build([a])
    L = fused.load(p, upload=False)
    runs, js = runs_of(fused, L)
    assert js["staged"] == 1
    assert runs[0]["ops"] == ["COPY"] and runs[1]["ops"] == ["ADD"]


def test_validation_errors(fused):
    ctx = fused.ctx
    f = V.vbe_base_create(ctx, V.VBE_FLOAT64, 10)
    i = V.vbe_base_create(ctx, V.VBE_INT64, 10)
    with pytest.raises(V.VbeError) as e:
        V.vbe_view_create(ctx, f, 5, (10,), (1,))
    assert e.value.code == -2
    vf = V.vbe_view_create(ctx, f, 0, (10,), (1,))
    vi = V.vbe_view_create(ctx, i, 0, (10,), (1,))
    vs = V.vbe_view_create(ctx, f, 0, (5,), (1,))
    vz = V.vbe_view_create(ctx, f, 0, (5,), (0,))

    def instr(op, out, *ins):
        arr = (V.vbe_instr * 1)()
        arr[0].op = V.OPCODES[op]
        arr[0].const_slot = -1
        arr[0].out = out
        for k, x in enumerate(ins):
            arr[0].in_[k] = x
        return arr

    cases = [(instr("ADD", vf, vf, vi), -3), (instr("DIVIDE", vi, vi, vi), -3), (instr("EXP", vi, vi), -3),
             (instr("ADD", vf, vf, vs), -4), (instr("COPY", vz, vs), -12), (instr("ADD", vf, vf, 999), -1)]
    for arr, code in cases:
        with pytest.raises(V.VbeError) as e:
            V.vbe_plan(ctx, arr, 1)
        assert e.value.code == code


def test_views_go_with_their_base(fused):
    """A base keeps the list of its views: freeing it (vbe_free, or a FREE
    bytecode in a recorded batch) makes exactly its views unknown; views of
    other bases keep working, and a destroyed view is gone."""
    ctx = fused.ctx
    f = V.vbe_base_create(ctx, V.VBE_FLOAT64, 10)
    g = V.vbe_base_create(ctx, V.VBE_FLOAT64, 10)
    vf = [V.vbe_view_create(ctx, f, k, (5,), (1,)) for k in range(3)]
    vg = V.vbe_view_create(ctx, g, 0, (5,), (1,))
    vg2 = V.vbe_view_create(ctx, g, 5, (5,), (1,))

    def instr(op, out, *ins):
        arr = (V.vbe_instr * 1)()
        arr[0].op = V.OPCODES[op]
        arr[0].const_slot = -1
        arr[0].out = out
        for k, x in enumerate(ins):
            arr[0].in_[k] = x
        return arr

    V.vbe_plan(ctx, instr("ADD", vf[0], vf[1], vg), 1)
    V.vbe_view_destroy(ctx, vg2)
    with pytest.raises(V.VbeError):
        V.vbe_view_destroy(ctx, vg2)  # already gone
    V.vbe_free(ctx, f)
    for v in vf:
        with pytest.raises(V.VbeError) as e:
            V.vbe_plan(ctx, instr("COPY", vg, v), 1)
        assert e.value.code == -1  # an unknown view
        with pytest.raises(V.VbeError):
            V.vbe_view_destroy(ctx, v)
    V.vbe_plan(ctx, instr("ADD", vg, vg, vg), 1)  # the other base's view is untouched
    h = V.vbe_view_create(ctx, g, 1, (9,), (1,))  # and the base takes new views
    V.vbe_plan(ctx, instr("COPY", vg, V.vbe_view_create(ctx, g, 2, (5,), (1,))), 1)
    V.vbe_view_destroy(ctx, h)


def _np_view(buf, v):
    return np.lib.stride_tricks.as_strided(buf[v.offset:], v.shape, tuple(8 * s for s in v.strides))


def test_overlap_test_is_sound_and_exact_on_grids(fused):
    """Random views of one base against np.shares_memory(max_work=None): a
    "disjoint" answer must never be wrong; for views whose strides form a
    divisibility chain (rows/columns/boxes of a grid) the answer is exact."""
    ctx = fused.ctx
    N = 24
    base = V.vbe_base_create(ctx, V.VBE_FLOAT64, N * N)
    buf = np.zeros(N * N)
    rng = np.random.default_rng(0)
    exact_checked = 0
    for _ in range(600):
        views = []
        for _ in range(2):
            kind = rng.integers(0, 3)
            if kind == 0:  # box
                r0, c0 = rng.integers(0, N, 2)
                nr, nc = rng.integers(1, N - r0 + 1), rng.integers(1, N - c0 + 1)
                views.append(View(1, int(r0 * N + c0), (int(nr), int(nc)), (N, 1)))
            elif kind == 1:  # strided row/column
                st = int(rng.choice([1, 2, 3, N, 2 * N]))
                off = int(rng.integers(0, N * N))
                n = int(rng.integers(1, max(2, (N * N - 1 - off) // st + 2)))
                n = min(n, (N * N - 1 - off) // st + 1)
                views.append(View(1, off, (n,), (st,)))
            else:  # reversed box
                r0, c0 = rng.integers(0, N, 2)
                nr, nc = rng.integers(1, r0 + 2), rng.integers(1, c0 + 2)
                views.append(View(1, int(r0 * N + c0), (int(nr), int(nc)), (-N, -1)))
        a, b = views
        ha = V.vbe_view_create(ctx, base, a.offset, a.shape, a.strides)
        hb = V.vbe_view_create(ctx, base, b.offset, b.shape, b.strides)
        got = V.vbe_views_may_overlap(ctx, ha, hb)
        truth = np.shares_memory(_np_view(buf, a), _np_view(buf, b), max_work=None)
        if truth:
            assert got, (a, b)
        chain = all(abs(s) in (1, N) for s in a.strides + b.strides)
        if chain:
            assert got == truth, (a, b)
            exact_checked += 1
    assert exact_checked > 200


@pytest.mark.parametrize("flags", [V.VBE_FUSE | V.VBE_PACK, 0])
def test_every_workload_kernel_compiles_for_sm103a(flags):
    with Executor(flags | HOST) as ex:
        for p in (jacobi(16, 1), blackscholes(1000), blackscholes(1000, "float32"),
                  montecarlo_pi(sizes=[10, 20]), shallow_water(12, 1), shallow_water(12, 1, "float32"),
                  *[c.program for c in tile_group_cases()]):
            L = ex.load(p, upload=False)
            assert V.vbe_plan_compile(ex.ctx, *L.batches[0]) >= 1


def test_generated_source_is_plain_cuda(fused):
    p = blackscholes(64, "float32")
    L = fused.load(p, upload=False)
    js = json.loads(fused.plan(L, 0, source=True))
    src = [i["run"]["source"] for i in js["items"] if "run" in i][0]
    assert "expf(" in src and "logf(" in src and "sqrtf(" in src
    assert "vbe_vload" in src  # 16-byte vector path
    assert "__fmaf" not in src and "fma(" not in src


def test_min_and_argmin_of_one_view_share_a_pass(fused):
    """kNN: each round's MIN_REDUCE and the ARGMIN_REDUCE of the same view
    and axis right after it are one run (one read of the distances), in the
    first round and after the masking; the plain path keeps them apart."""
    from workloads import knn
    p = knn(300, 20, 8, 3)
    L = fused.load(p, upload=False)
    runs, _ = runs_of(fused, L)
    paired = [r for r in runs if "reduce2" in r]
    assert len(paired) == 3
    assert all(r["reduce"]["op"] == "MIN_REDUCE" and r["reduce2"]["op"] == "ARGMIN_REDUCE" for r in paired)
    assert all(r["mode"].startswith("axis") for r in paired)
    # a MIN over one view and an ARGMIN over another are not paired
    b = ProgramBuilder("unpaired")
    x = b.base("float64", (4, 50), np.arange(200, dtype=np.float64))
    y = b.base("float64", (4, 50), np.arange(200, dtype=np.float64)[::-1].copy())
    m = b.base("float64", 4)
    i = b.base("int64", 4)
    b.emit("MIN_REDUCE", b.whole(m), b.whole(x), axis=1)
    b.emit("ARGMIN_REDUCE", b.whole(i), b.whole(y), axis=1)
    L = fused.load(b.build([m, i]), upload=False)
    runs, _ = runs_of(fused, L)
    assert not any("reduce2" in r for r in runs) and len(runs) == 2
    # a MIN written into its own input (x[:, 0]) changes the rows the ARGMIN
    # then reads: the two are not paired (the MIN reads a private copy of x)
    b = ProgramBuilder("min_into_input")
    x = b.base("float64", (4, 50), np.arange(200, dtype=np.float64))
    i = b.base("int64", 4)
    b.emit("MIN_REDUCE", b.view(x, 0, (4,), (50,)), b.whole(x), axis=1)
    b.emit("ARGMIN_REDUCE", b.whole(i), b.whole(x), axis=1)
    L = fused.load(b.build([x, i]), upload=False)
    runs, _ = runs_of(fused, L)
    assert not any("reduce2" in r for r in runs)


def test_group_sources_are_shared_by_identical_groups(fused):
    """A tile-fused group's generated source depends on its structure, not on
    which base handles it uses: two Jacobi programs of one size, the second
    loaded after unrelated bases (other handles), plan the same source; a
    different grid size may change it (sizes are part of the key)."""
    def group_source(p):
        L = fused.load(p, upload=False)
        js = json.loads(fused.plan(L, 0, source=True))
        srcs = [i["group"]["source"] for i in js["items"] if "group" in i]
        assert len(srcs) == 1
        return srcs[0]
    a = group_source(jacobi(64, 1))
    fused.load(blackscholes(100), upload=False)  # takes handles in between
    b = group_source(jacobi(64, 1))
    assert a == b
    assert "_tm32x32" in a  # the tensor-copy form with the whole-run reduction


def test_power_of_two_constants_get_their_own_kernel(fused):
    """Float64 products by a constant +-2^k are formed by moving the exponent
    field; whether a constant is such a power is part of the kernel's
    signature, so two runs that differ only there get different sources."""
    srcs = {}
    for c in (0.5, 0.3, -4.0, 2.0 ** -1030):
        b = ProgramBuilder(f"mulk_{c}")
        x = b.base("float64", 64, np.arange(64, dtype=np.float64))
        y = b.base("float64", 64)
        b.emit("MULTIPLY", b.whole(y), b.whole(x), Const(c))
        p = b.build([y])
        L = fused.load(p, upload=False)
        js = json.loads(fused.plan(L, 0, source=True))
        srcs[c] = [i["run"]["source"] for i in js["items"] if "run" in i][0]
    assert "vbe_dmul_k(" in srcs[0.5] and "vbe_dmul_k(" in srcs[-4.0]
    assert "vbe_dmul_k(" not in srcs[0.3]
    assert "vbe_dmul_k(" not in srcs[2.0 ** -1030]  # subnormal: not a normal power of two


def test_user_operation_registration(fused):
    """Section "Interface": registration of a user-defined operation. The
    body is compiled at registration; the same definition gets the same
    opcode (in any context); the operation fuses with ordinary bytecodes."""
    ctx = fused.ctx
    a = V.vbe_op_register(ctx, "hyp_test", "return a * a + b * b;", 2, V.VBE_FLOAT64)
    assert a >= V.VBE_OP_USER_BASE
    assert V.vbe_op_register(ctx, "hyp_test", "return a * a + b * b;", 2, V.VBE_FLOAT64) == a
    with Executor(V.VBE_HOST_ONLY) as other:
        assert V.vbe_op_register(other.ctx, "hyp_test", "return a * a + b * b;", 2, V.VBE_FLOAT64) == a
    bad = [("hyp_test", "return a;", 2, V.VBE_FLOAT64, -1),      # another definition under the name
           ("9bad", "return a;", 1, V.VBE_FLOAT64, -1),           # not an identifier
           ("ok_name", "return a;", 0, V.VBE_FLOAT64, -1),        # arity
           ("ok_name", "return a;", 1, V.VBE_BOOL, -1),           # dtype
           ("broken", "return a +;", 1, V.VBE_FLOAT32, -7)]       # does not compile
    for name, body, nin, dt, code in bad:
        with pytest.raises(V.VbeError) as e:
            V.vbe_op_register(ctx, name, body, nin, dt)
        assert e.value.code == code, (name, e.value)
    from parity_cases import user_op_cases
    case = user_op_cases()[0]
    L = fused.load(case.program, upload=False)
    runs, _ = runs_of(fused, L)
    # three independent chains of one shape: user op + ordinary op each, one kernel
    assert len(runs) == 1 and {"axpy_div", "sq_plus_one", "tri", "MULTIPLY", "ADD"} <= set(runs[0]["ops"])
    # dtype rules apply to user operations
    b = V.vbe_base_create(ctx, V.VBE_FLOAT32, 8)
    vb = V.vbe_view_create(ctx, b, 0, (8,), (1,))
    arr = (V.vbe_instr * 1)()
    arr[0].op = a
    arr[0].const_slot = -1
    arr[0].out = vb
    arr[0].in_[0] = vb
    arr[0].in_[1] = vb
    with pytest.raises(V.VbeError) as e:
        V.vbe_plan(ctx, arr, 1, False)
    assert e.value.code == -3


def test_caller_owned_state_is_never_renamed():
    """A base registered from the caller's memory keeps its address: when a
    shallow-water step would have to rename it, the chain stays separate
    kernels (the in-place update then happens in the caller's buffer)."""
    p = shallow_water(12, 1)
    with Executor(V.VBE_FUSE | V.VBE_PACK | HOST) as ex:
        fake = {p.meta["H"]: 0x10000}  # an address the host-only context never dereferences
        L = ex.load(p, device_ptrs=fake, upload=False)
        js = json.loads(ex.plan(L, 0))
        assert not any("group" in i for i in js["items"])
        assert [len(i["run"]["ops"]) for i in js["items"] if "run" in i] == [6, 6, 9, 21, 21, 18]


def test_fp64_rate_probe_rejects_bad_arguments():
    """vbe_measure_fp64_rate validates its arguments before touching a device."""
    for op, iters, scratch in ((3, 10, 16), (-1, 10, 16), (0, 0, 16), (0, 10, 0)):
        code = V.lib.vbe_measure_fp64_rate(op, iters, ctypes.byref(ctypes.c_double()), scratch or None, None)
        assert code == -1, (op, iters, scratch)
