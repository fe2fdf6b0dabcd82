"""Serving loop on the GPU: concurrent clients, continuous batching under a
memory cap, and each request's result identical alone and in the mix."""
import os
import threading

import numpy as np
import pytest

from paper_1210_7774_b300 import build

build.build()

from paper_1210_7774_b300 import vbe as V  # noqa: E402
from paper_1210_7774_b300.runner import Request  # noqa: E402

import oracle  # noqa: E402
from parity_cases import assert_close_sum, assert_exact  # noqa: E402
from workloads.serving import blackscholes_request, jacobi_request, request_mix, request_program  # noqa: E402

pytestmark = pytest.mark.gpu
CACHE = os.environ.get("VBE_CACHE_DIR", "/tmp/vbe_kernel_cache")
FLAGS = V.VBE_FUSE | V.VBE_PACK


def small_mix(n):
    """The request mix with sizes scaled down so the test stays short."""
    out = []
    for kind, prm in request_mix(n, seed=5):
        prm = dict(prm)
        if kind == "jacobi":
            prm["n"] = 32 + (prm["n"] // 16)
            prm["iters"] = min(prm["iters"], 6)
        else:
            prm["n"] = max(1, prm["n"] // 64)
        out.append((kind, prm))
    return out


def serve(programs, slots=4, cap=8 << 30, threads=8, workers=1):
    ctx = V.vbe_init(0, FLAGS, 0, None, CACHE)
    srv = V.vbe_server_create(ctx, slots, cap, FLAGS, workers=workers)
    reqs = [Request(p) for p in programs]
    results = [None] * len(reqs)

    def client(k):
        for i in range(k, len(reqs), threads):
            rid = V.vbe_server_submit(srv, reqs[i].req)
            results[i] = V.vbe_server_wait(srv, rid, 120_000_000_000)

    th = [threading.Thread(target=client, args=(k,)) for k in range(threads)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    V.vbe_server_destroy(srv)
    V.vbe_finalize(ctx)
    return reqs, results


@pytest.mark.parametrize("workers", [1, 3])
def test_requests_match_oracle_and_solo_results(workers):
    """With one scheduler thread, and with three (each with its own context
    and slots, planning in parallel)."""
    mix = small_mix(40)
    programs = [request_program(k, p) for k, p in mix]
    reqs, res = serve(programs, slots=6, workers=workers)
    assert all(r.status == 0 for r in res)
    assert all(r.t_arrive_ns <= r.t_admit_ns <= r.t_done_ns for r in res)
    # each result equals the same request run alone (bitwise: kernels and
    # launch shapes depend only on the request, never on co-tenants)
    solo_reqs, _ = serve(programs[:12], slots=1, threads=1)
    for a, b in zip(reqs[:12], solo_reqs):
        for bid in a.results:
            assert_exact(a.results[bid], b.results[bid], a.program.name)
    # and the oracle agrees
    for r in reqs[:10]:
        check_against_oracle(r)


def check_against_oracle(r):
    """One served request against the oracle: a Jacobi grid bit-exact and its
    last delta within the reduction tolerance (the delta is a sum of
    non-negative terms, so the sum of magnitudes is the delta itself); the
    Black-Scholes call and put per option within rtol * max(S, K), with S and
    K taken from the oracle's own run (their final DISCARD left out so that
    their values stay readable)."""
    p = r.program
    kind = p.meta["kind"]
    if kind == "jacobi":
        want = oracle.run(p)
        g, d = p.meta["grid"], p.meta["delta"]
        assert_exact(r.results[g], want[g], p.name)
        rtol = 1e-12 if want[d].dtype == np.float64 else 1e-5
        assert_close_sum(r.results[d], want[d], np.abs(want[d].astype(np.float64)), rtol, p.name + " delta")
        return
    keep = (p.meta["S"], p.meta["K"])
    want = oracle.run(p, [i for i in p.instrs if not (i.op == "DISCARD" and i.out.base in keep)])
    mx = np.maximum(want[keep[0]], want[keep[1]]).astype(np.float64)
    assert np.all((mx >= 10.0) & (mx < 100.0))
    for bid in p.outputs:
        got = r.results[bid]
        rtol = 1e-12 if got.dtype == np.float64 else 1e-5
        err = np.abs(got.astype(np.float64) - want[bid].astype(np.float64))
        assert np.all(err <= rtol * mx), (p.name, float(np.max(err / mx)))


def test_full_size_mix_matches_oracle():
    """The serving mix at its full sizes (Jacobi sides up to 2048, 1 to 20
    iterations; Black-Scholes up to 4M options; float32 and float64): the
    first 24 requests of the benchmark's mix plus the largest request of each
    kind, served by 16 slots under the 60 GB cap, every one against the
    oracle."""
    from workloads.serving import request_mix as mix_of
    mix = mix_of(24) + [("jacobi", dict(n=2048, iters=20, dtype="float64", seed=71)),
                        ("blackscholes", dict(n=4 << 20, dtype="float32", seed=72)),
                        ("blackscholes", dict(n=4 << 20, dtype="float64", seed=73))]
    programs = [request_program(k, p) for k, p in mix]
    reqs, res = serve(programs, slots=16, cap=60 << 30, threads=16, workers=4)
    assert all(x.status == 0 for x in res)
    for r in reqs:
        check_against_oracle(r)


def test_admission_respects_memory_cap_and_rejects_oversize():
    programs = [jacobi_request(64, 2, "float64", s) for s in range(6)]
    # the footprint counts every base, and once more each base the request
    # both reads and writes (the grid: it may get a second buffer)
    _, solo = serve(programs[:1], slots=1)
    foot = solo[0].footprint_bytes
    grid = 64 * 64 * 8
    assert foot == sum(b.nelem * 8 for b in programs[0].bases.values()) + grid
    # a cap that fits one request at a time: all complete, one by one, also
    # with several workers admitting from the one queue
    reqs, res = serve(programs, slots=4, cap=foot + 1024, threads=3, workers=2)
    assert all(r.status == 0 for r in res)
    spans = sorted((r.t_admit_ns, r.t_done_ns) for r in res)
    for (a0, d0), (a1, d1) in zip(spans, spans[1:]):
        assert a1 >= d0 - 1e6  # admitted only after the previous one finished
    ctx = V.vbe_init(0, FLAGS, 0, None, CACHE)
    srv = V.vbe_server_create(ctx, 2, foot // 2, FLAGS)
    big = Request(programs[0])
    with pytest.raises(V.VbeError) as e:
        V.vbe_server_submit(srv, big.req)
    assert e.value.code == -6
    V.vbe_server_destroy(srv)
    V.vbe_finalize(ctx)


def test_blackscholes_request_random_inputs_are_in_range():
    p = blackscholes_request(5000, "float64", 3)
    reqs, res = serve([p], slots=1, threads=1)
    call = reqs[0].results[p.outputs[0]]
    put = reqs[0].results[p.outputs[1]]
    assert np.all(call >= -1e-9) and np.all(put >= -1e-9) and np.all(call <= 100.0)


def test_pinned_result_buffers_filled_directly():
    """Result buffers in page-locked memory receive the device's copies
    directly (no staging); the results still match the oracle and the staged
    path bit for bit, with several workers and clients reusing their arenas."""
    torch = pytest.importorskip("torch")
    programs = [request_program(k, p) for k, p in small_mix(24)]
    staged, _ = serve(programs, slots=4, workers=2)
    reqs = [Request(p) for p in programs]
    nthreads = 4
    arenas = [torch.empty(max(r.result_bytes() for r in reqs), dtype=torch.uint8).pin_memory().numpy()
              for _ in range(nthreads)]
    got = [None] * len(reqs)
    ctx = V.vbe_init(0, FLAGS, 0, None, CACHE)
    srv = V.vbe_server_create(ctx, 4, 8 << 30, FLAGS, workers=2)

    def client(k):
        for i in range(k, len(reqs), nthreads):
            reqs[i].bind_results(arenas[k])
            r = V.vbe_server_wait(srv, V.vbe_server_submit(srv, reqs[i].req), 120_000_000_000)
            assert r.status == 0
            got[i] = {bid: a.copy() for bid, a in reqs[i].results.items()}

    th = [threading.Thread(target=client, args=(k,)) for k in range(nthreads)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    V.vbe_server_destroy(srv)
    V.vbe_finalize(ctx)
    for i, r in enumerate(staged):
        for bid in r.results:
            assert_exact(got[i][bid], r.results[bid], r.program.name)
    for i in range(0, len(reqs), 6):
        reqs[i].results = got[i]
        check_against_oracle(reqs[i])


def test_waits_out_of_order_and_timed_out_waits():
    """Each request wakes only its own waiter: one thread submits many
    requests and waits for them in reverse order; another waits with a wait
    limit too short for a large request (VBE_ERR_TIMEOUT, nothing taken),
    then waits again and gets the same results as a solo run."""
    progs = [request_program(k, p) for k, p in small_mix(24)]
    big = request_program("blackscholes", dict(n=1 << 22, dtype="float64", seed=7))
    ctx = V.vbe_init(0, FLAGS, 0, None, CACHE)
    srv = V.vbe_server_create(ctx, 4, 8 << 30, FLAGS, workers=2)
    try:
        reqs = [Request(p) for p in progs]
        ids = [V.vbe_server_submit(srv, r.req) for r in reqs]
        for i in reversed(range(len(ids))):
            assert V.vbe_server_wait(srv, ids[i], 120_000_000_000).status == 0
        rb = Request(big)
        rid = V.vbe_server_submit(srv, rb.req)
        with pytest.raises(V.VbeError) as e:
            V.vbe_server_wait(srv, rid, 1000)  # 1 us: the pricing of 4M options is still running
        assert e.value.code == -8  # VBE_ERR_TIMEOUT
        assert V.vbe_server_wait(srv, rid, 120_000_000_000).status == 0
    finally:
        V.vbe_server_destroy(srv)
        V.vbe_finalize(ctx)
    solo_reqs, solo = serve(progs, threads=1)
    for a, b in zip(reqs, solo_reqs):
        for bid in a.results:
            np.testing.assert_array_equal(a.results[bid], b.results[bid])
    big_solo_reqs, _ = serve([big], threads=1)
    for bid in rb.results:
        np.testing.assert_array_equal(rb.results[bid], big_solo_reqs[0].results[bid])
