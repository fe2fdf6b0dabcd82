"""GPU parity: the CUDA path (through the C ABI) against the oracle, element
by element, on seeded inputs; fused, plain (one launch per bytecode) and
graph-replayed execution; and the full-size configurations checked on
samples or properties that hold at any size."""
import os

import numpy as np
import pytest

from paper_1210_7774_b300 import build

build.build()

from paper_1210_7774_b300 import vbe as V  # noqa: E402
from paper_1210_7774_b300.runner import Executor  # noqa: E402

import oracle  # noqa: E402
from parity_cases import (F64_REDUCE_RTOL, Case, _exact_check, all_small_cases, assert_close_sum,  # noqa: E402
                          assert_exact, jacobi_case, oracle_outputs, tile_group_cases, workload_cases)
from workloads import (blackscholes, bs_inputs, gray_scott, jacobi, knn, knn_inputs, mc_sizes,  # noqa: E402
                       montecarlo_pi, shallow_water, sw_inputs)

pytestmark = pytest.mark.gpu
CACHE = os.environ.get("VBE_CACHE_DIR", "/tmp/vbe_kernel_cache")

FUSED = V.VBE_FUSE | V.VBE_PACK | V.VBE_AUTOTUNE
MODES = {"fused": FUSED, "plain": 0, "fused_graphs": FUSED | V.VBE_GRAPHS,
         # every eligible one-dimensional run staged through shared memory by
         # bulk copies, in chunks of 256 elements
         "fused_staged": FUSED | V.VBE_GRAPHS}
STAGING = {"fused_staged": 256}


def make_executor(flags, staging=0, **kw):
    """An executor; staging > 0 forces staged runs (the variable is read
    when the context is created, and restored right after)."""
    old = os.environ.pop("VBE_STAGING", None)
    if staging:
        os.environ["VBE_STAGING"] = str(staging)
    try:
        return Executor(flags, cache_dir=CACHE, **kw)
    finally:
        os.environ.pop("VBE_STAGING", None)
        if old is not None:
            os.environ["VBE_STAGING"] = old


def run_gpu(program, flags, repeat_batches=1, staging=0):
    with make_executor(flags, staging) as ex:
        L = ex.load(program)
        for _ in range(repeat_batches):
            ex.run(L)
        out = {bid: ex.read(L, bid) for bid in program.outputs}
        out["_stats"] = ex.stats()
        return out


SMALL = all_small_cases()


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("case", SMALL, ids=[c.name for c in SMALL])
def test_small_parity(case, mode):
    got = run_gpu(case.program, MODES[mode], staging=STAGING.get(mode, 0))
    case.check(got, oracle_outputs(case.program))


MEDIUM = workload_cases("medium")


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("case", MEDIUM, ids=[c.name for c in MEDIUM])
def test_medium_workload_parity(case, mode):
    got = run_gpu(case.program, MODES[mode], staging=STAGING.get(mode, 0))
    case.check(got, oracle_outputs(case.program))
    if mode == "fused_graphs" and case.name.startswith(("jacobi", "shallow")) and not case.name.endswith("one_batch"):
        # repeated iterations replay a graph (or, for a batch of one or two
        # launches, its cached launch list)
        assert got["_stats"]["graph_launches"] + got["_stats"]["list_replays"] > 0


def test_jacobi_config_full_size_graphs_and_plain_agree():
    """Config: 256x256 float64, 10 iterations, fused + graph replay; the grid
    is bit-exact with the oracle and with the plain path."""
    p = jacobi(256, 10)
    want = oracle_outputs(p)
    for flags in (FUSED | V.VBE_GRAPHS, 0):
        got = run_gpu(p, flags)
        assert_exact(got[p.meta["grid"]], want[p.meta["grid"]], "grid")
        g0 = p.bases[p.meta["grid"]].init
        assert_close_sum(got[p.meta["deltas"]], want[p.meta["deltas"]], np.full(1, 2 * np.abs(g0).sum()),
                         F64_REDUCE_RTOL, "deltas")


def test_synthetic_stencil_full_size():
    """10240 x 1024 Gray-Scott fields, float64 and float32: two steps
    bit-exact with the oracle (only + - * in a fixed order), tile-fused
    with both fields renamed."""
    for dt in ("float64", "float32"):
        p = gray_scott(10240, 1024, 2, dt)
        want = oracle_outputs(p)
        got = run_gpu(p, FUSED | V.VBE_GRAPHS)
        for q in ("U", "V"):
            assert_exact(got[p.meta[q]], want[p.meta[q]], q + " " + dt)


def test_knn_paper_size_sampled():
    """10,000 points, 1,000 queries (16-D, k = 4), float64 and float32: 64
    sampled queries recomputed by the oracle as a program of their own."""
    from parity_cases import knn_check
    for dt in ("float64", "float32"):
        inp = knn_inputs(10_000, 1_000, 16, dt)
        p = knn(10_000, 1_000, 16, 4, dt, inputs=inp)
        got = run_gpu(p, FUSED | V.VBE_GRAPHS)
        rows = np.sort(np.random.default_rng(5).choice(1_000, 64, replace=False))
        sub = knn(10_000, 64, 16, 4, dt, inputs={"X": inp["X"], "Q": inp["Q"][rows]})
        w = oracle_outputs(sub)
        want = {p.meta["dist"]: w[sub.meta["dist"]], p.meta["idx"]: w[sub.meta["idx"]]}
        knn_check(p, rows)(got, want)


def test_jacobi_paper_size_tile_fused():
    """The paper's Jacobi size (7168^2 float64, 4 iterations), each iteration
    one tile-fused kernel with the grid renamed: grid bit-exact with the
    oracle, deltas within the reduction tolerance."""
    p = jacobi(7168, 4)
    want = oracle_outputs(p)
    got = run_gpu(p, FUSED | V.VBE_GRAPHS)
    assert_exact(got[p.meta["grid"]], want[p.meta["grid"]], "grid")
    g0 = p.bases[p.meta["grid"]].init
    assert_close_sum(got[p.meta["deltas"]], want[p.meta["deltas"]], np.full(1, 2 * np.abs(g0).sum()),
                     F64_REDUCE_RTOL, "deltas")


@pytest.mark.parametrize("tile", ["t32x32", "t16x64", "s32x32", "32x32", "r24", "r64"])
def test_tile_group_forms_exact(tile):
    """Tile-fused groups forced into one tile shape and form (VBE_TILE, read
    when the context is created): inputs read through L1, staged through
    shared memory ("s"), prefetched by double-buffered tensor copies into
    persistent blocks that walk several tiles each ("t"), or swept down the
    rows by one warp per column strip, values in registers and handed
    across columns by warp shuffles ("r", strips of 24 or 64 rows).
    Bit-exact with the oracle on the synthetic chains (rows of 16-byte
    multiples, ragged against every tile), Jacobi 514^2 (a group with a
    whole-run reduction: deltas within the reduction tolerance; no row-sweep
    form), shallow water (state renamed every step) and Gray-Scott at
    2050 x 1032 (about 2,000 tiles), float64 and float32."""
    cases = tile_group_cases(seed=12, N=37, M=52) + [jacobi_case(514, 3)]
    for dt in ("float64", "float32"):
        for p in (shallow_water(256, 2, dt), gray_scott(2050, 1032, 2, dt)):
            cases.append(Case(p.name, p, _exact_check(p)))
    os.environ["VBE_TILE"] = tile
    try:
        for case in cases:
            got = run_gpu(case.program, V.VBE_FUSE | V.VBE_PACK)
            case.check(got, oracle_outputs(case.program))
            if tile.startswith("t"):
                assert got["_stats"]["tma_group_launches"] > 0, case.name
            if tile.startswith("r") and not case.name.startswith("jacobi"):
                assert got["_stats"]["sweep_group_launches"] > 0, case.name
    finally:
        os.environ.pop("VBE_TILE")


@pytest.mark.parametrize("staging", [0, 2048])
@pytest.mark.parametrize("dtype,rtol", [("float64", 1e-12), ("float32", 1e-5)])
def test_blackscholes_full_size_sampled(dtype, rtol, staging):
    """16M options, in the launch configuration the benchmark times (and
    with the inputs staged through shared memory in 2048-element chunks);
    20,000 sampled options recomputed by the oracle one program at a time."""
    n = 1 << 24
    inp = bs_inputs(n, dtype)
    p = blackscholes(n, dtype, inputs=inp)
    got = run_gpu(p, FUSED | V.VBE_GRAPHS, staging=staging)
    idx = np.sort(np.random.default_rng(7).choice(n, 20_000, replace=False))
    idx = np.concatenate([[0, 1, n - 2, n - 1], idx])
    sub = blackscholes(len(idx), dtype, inputs={k: v[idx] for k, v in inp.items()})
    want = oracle_outputs(sub)
    mx = np.maximum(inp["S"][idx], inp["K"][idx]).astype(np.float64)
    for full_id, sub_id in ((p.meta["call"], sub.meta["call"]), (p.meta["put"], sub.meta["put"])):
        err = np.abs(got[full_id][idx].astype(np.float64) - want[sub_id].astype(np.float64))
        assert np.all(err <= rtol * mx), np.max(err / mx)


def test_shallow_water_full_size_two_steps_exact_and_mass():
    """4096x4096 float64: two steps bit-exact with the oracle (the scheme uses
    only + - * /, so IEEE arithmetic fixes every bit; a step whose group
    renames the state writes the second buffer set, so two steps cover both
    address sets), in the launch configuration the benchmark times (fused,
    graph replay); five steps conserve mass to rounding and keep the
    droplet's mirror symmetry bitwise (negation, sums and products are
    exact under the mirror, so the scheme commutes with it bit for bit)."""
    N = 4096
    p = shallow_water(N, 2)
    want = oracle_outputs(p)
    got = run_gpu(p, FUSED | V.VBE_GRAPHS)
    for q in ("H", "U", "V"):
        assert_exact(got[p.meta[q]], want[p.meta[q]], q)
    inp = sw_inputs(N, centred=True)
    p5 = shallow_water(N, 5, inputs=inp)
    got = run_gpu(p5, FUSED | V.VBE_GRAPHS)
    H = got[p5.meta["H"]].reshape(N, N)[1:-1, 1:-1]
    H0 = inp["H"][1:-1, 1:-1]
    assert abs(H.sum(dtype=np.float64) - H0.sum(dtype=np.float64)) <= 1e-11 * H0.sum()
    assert np.array_equal(H, H[::-1, :])
    assert np.array_equal(H, H[:, ::-1])


def test_montecarlo_full_config_sampled_instances_exact():
    """All 256 instances (2^10..2^24 samples) in one packed launch (the
    packed-launch statistic says it ran); the smallest 24 instances (one
    chunk of the work queue each) and the four largest (about 16 M samples
    each: many chunks, whose partial counts the instance's last chunk
    combines) recomputed exactly by the oracle; every estimate within 6
    sigma of pi/4."""
    sizes = mc_sizes(256)
    p = montecarlo_pi(sizes=sizes)
    got = run_gpu(p, FUSED)
    assert got["_stats"]["packed_launches"] >= 1
    assert got["_stats"]["kernel_launches"] <= 4
    counts = got[p.meta["count"]]
    order = np.argsort(sizes)
    pick = np.concatenate([order[:24], order[-4:]])
    assert sizes[order[-4:]].min() > 1 << 23
    sub = montecarlo_pi(sizes=sizes[pick], keys=pick)
    want = oracle_outputs(sub)[sub.meta["count"]]
    assert counts[pick].tolist() == want.tolist()
    q = np.pi / 4
    sig = np.sqrt(q * (1 - q) / sizes)
    assert np.all(np.abs(counts / sizes - q) < 6 * sig)
    pp = montecarlo_pi(sizes=sizes[:32])
    plain = run_gpu(pp, 0)
    assert plain[pp.meta["count"]].tolist() == counts[:32].tolist()


def test_errors_on_device():
    with Executor(FUSED, cache_dir=CACHE) as ex:
        ctx = ex.ctx
        a = V.vbe_base_create(ctx, V.VBE_FLOAT64, 16)
        o = V.vbe_base_create(ctx, V.VBE_FLOAT64, 16)
        va = V.vbe_view_create(ctx, a, 0, (16,), (1,))
        vo = V.vbe_view_create(ctx, o, 0, (16,), (1,))
        arr = (V.vbe_instr * 1)()
        arr[0].op = V.OPCODES["SQRT"]
        arr[0].const_slot = -1
        arr[0].out = vo
        arr[0].in_[0] = va
        with pytest.raises(V.VbeError) as e:  # a was never written
            V.vbe_submit(ctx, arr, 1)
        assert e.value.code == -10
        host = np.arange(16.0)
        V.vbe_base_upload(ctx, a, host.ctypes.data, host.nbytes)
        t = V.vbe_submit(ctx, arr, 1)
        V.vbe_wait(ctx, t, 10_000_000_000)
        out = np.empty(16)
        V.vbe_sync(ctx, o, out.ctypes.data, out.nbytes)
        assert np.array_equal(out, np.sqrt(host))


def test_views_beyond_two_to_the_31_elements():
    """Maximum sizes: float32 views of 2^31 + 4099 elements (8.6 GB each,
    indices past every 32-bit boundary). x = a / 4 with a = i mod 1024 and
    y = b with b = (i div 3) mod 512, so z = x * y + x = a (b + 1) / 4 is
    exact in float32: z bit-exact at sampled indices (both sides of 2^31),
    the full ADD_REDUCE and the column sums of z viewed as
    (2^20 + 2) x 2048 (reduced dimension outer, 2^31 + 4096 elements)
    within the float32 reduction tolerance of exact integer sums."""
    torch = pytest.importorskip("torch")
    n = (1 << 31) + 4099
    R, C = n // 2048, 2048
    i = torch.arange(n, dtype=torch.int64, device="cuda")
    x = ((i % 1024).to(torch.float32) * 0.25)
    y = ((i // 3) % 512).to(torch.float32)
    del i
    z = torch.empty(n, dtype=torch.float32, device="cuda")
    s = torch.zeros(1, dtype=torch.float32, device="cuda")
    cs = torch.zeros(C, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    with Executor(FUSED, cache_dir=CACHE, stream=torch.cuda.current_stream().cuda_stream) as ex:
        ctx = ex.ctx
        f32 = V.DTYPE_CODE["float32"]
        bx, by, bz = (V.vbe_base_register(ctx, f32, n, t.data_ptr()) for t in (x, y, z))
        bs = V.vbe_base_register(ctx, f32, 1, s.data_ptr())
        bc = V.vbe_base_register(ctx, f32, C, cs.data_ptr())
        vx, vy, vz = (V.vbe_view_create(ctx, b, 0, (n,), (1,)) for b in (bx, by, bz))
        vs = V.vbe_view_create(ctx, bs, 0, (), ())
        vz2 = V.vbe_view_create(ctx, bz, 0, (R, C), (C, 1))
        vc = V.vbe_view_create(ctx, bc, 0, (C,), (1,))
        arr = (V.vbe_instr * 4)()
        for e, (op, out, ins, axis) in zip(arr, (("MULTIPLY", vz, (vx, vy), 0), ("ADD", vz, (vz, vx), 0),
                                                 ("ADD_REDUCE", vs, (vz,), 0), ("ADD_REDUCE", vc, (vz2,), 0))):
            e.op = V.OPCODES[op]
            e.const_slot = -1
            e.out = out
            for k, v in enumerate(ins):
                e.in_[k] = v
            e.axis = axis
        V.vbe_submit(ctx, arr, 4)
        torch.cuda.current_stream().synchronize()
    rng = np.random.default_rng(31)
    idx = np.unique(np.concatenate([[0, 1, (1 << 31) - 1, 1 << 31, (1 << 31) + 1, n - 1],
                                    rng.integers(0, n, 2000)]))
    a, b = idx % 1024, (idx // 3) % 512
    want = (a * (b + 1)).astype(np.float32) * np.float32(0.25)
    got = z[torch.from_numpy(idx).cuda()].cpu().numpy()
    assert_exact(got, want, "z at sampled indices")

    def exact_sum(lo, hi, step=1, start=0):
        # sum of a (b + 1) over i = start + step * k for lo <= k < hi, in int64
        tot = 0
        for c0 in range(lo, hi, 1 << 24):
            k = np.arange(c0, min(hi, c0 + (1 << 24)), dtype=np.int64)
            ii = start + step * k
            tot += int(np.sum((ii % 1024) * ((ii // 3) % 512 + 1)))
        return tot
    # a (b + 1) repeats with period lcm(1024, 3 * 512) = 3072
    q, rem = divmod(n, 3072)
    total = q * exact_sum(0, 3072) + exact_sum(0, rem)
    assert_close_sum(s.cpu().numpy(), np.array([total / 4.0]), np.array([total / 4.0]), 1e-5, "full sum")
    cols = rng.choice(C, 12, replace=False)
    col_want = np.array([exact_sum(0, R, C, int(c)) / 4.0 for c in cols])
    assert_close_sum(cs.cpu().numpy()[cols], col_want, col_want, 1e-5, "column sums")


def test_registered_device_memory():
    torch = pytest.importorskip("torch")
    x = torch.arange(1000, dtype=torch.float64, device="cuda")
    y = torch.empty(1000, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    with Executor(FUSED, cache_dir=CACHE, stream=torch.cuda.current_stream().cuda_stream) as ex:
        ctx = ex.ctx
        bx = V.vbe_base_register(ctx, V.VBE_FLOAT64, 1000, x.data_ptr())
        by = V.vbe_base_register(ctx, V.VBE_FLOAT64, 1000, y.data_ptr())
        vx = V.vbe_view_create(ctx, bx, 0, (1000,), (1,))
        vy = V.vbe_view_create(ctx, by, 0, (1000,), (1,))
        arr = (V.vbe_instr * 1)()
        arr[0].op = V.OPCODES["MULTIPLY"]
        arr[0].const_slot = 1
        arr[0].konst.f64 = 3.0
        arr[0].out = vy
        arr[0].in_[0] = vx
        V.vbe_submit(ctx, arr, 1)
        torch.cuda.current_stream().synchronize()
        assert torch.equal(y, x * 3.0)


def test_fp64_rate_probe_is_plausible():
    """The FP64 pipe's rate from the throughput kernel (median of three
    launches after a warm-up): the three operations agree within 5 %, and
    the rate lies between 1/128 and 1/32 of the FP32
    lanes' rate at the boost clock (B300's FP64 pipe: about 1/76)."""
    torch = pytest.importorskip("torch")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    scratch = torch.empty(2048 * sms, dtype=torch.float64, device="cuda")
    rates = []
    for op in ("dfma", "dadd", "dmul"):
        V.vbe_measure_fp64_rate(op, 512, scratch.data_ptr())  # warm-up launch
        rates.append(sorted(V.vbe_measure_fp64_rate(op, 2048, scratch.data_ptr()) for _ in range(3))[1])
    assert max(rates) <= 1.05 * min(rates), rates
    fp32 = sms * 128 * 2.032e9
    assert fp32 / 128 < rates[0] < fp32 / 32, rates
