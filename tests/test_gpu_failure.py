"""Failure detection on the GPU without a fault: the compute threads' waits
for staged data are limited to zero polls (vbe_debug_set_wait_polls), so
they run out at once while the producer and drain waits keep their full
limit and see every issued copy land. The kernel reports through the error
word, vbe_wait returns VBE_ERR_TIMEOUT (once), and the next ordinary batch
on the same context matches the oracle. Forms: one-dimensional runs staged
by bulk copies (Black-Scholes, 1M options) and a tile-fused group in the
tensor-copy form (Gray-Scott, 2050 x 1032). The same kernels ran this path
emulated on the CPU first (test_failure_host.py)."""
import numpy as np
import pytest

from paper_1210_7774_b300 import build

build.build()

from paper_1210_7774_b300 import vbe as V  # noqa: E402
from paper_1210_7774_b300.runner import Executor  # noqa: E402

from parity_cases import _exact_check, oracle_outputs  # noqa: E402
from test_gpu_parity import CACHE  # noqa: E402
from workloads import blackscholes, bs_inputs, gray_scott  # noqa: E402

pytestmark = pytest.mark.gpu
FLAGS = V.VBE_FUSE | V.VBE_PACK


def run_failing_then_ordinary(ex, p):
    L = ex.load(p)
    V.vbe_debug_set_wait_polls(ex.ctx, 0)
    t = 0
    for k in range(len(L.batches)):
        t = ex.submit(L, k)
    with pytest.raises(V.VbeError) as e:
        V.vbe_wait(ex.ctx, t, 30_000_000_000)
    assert e.value.code == -8  # VBE_ERR_TIMEOUT
    V.vbe_debug_set_wait_polls(ex.ctx, -1)  # reported once; normal kernels again
    L2 = ex.load(p)
    t = 0
    for k in range(len(L2.batches)):
        t = ex.submit(L2, k)
    V.vbe_wait(ex.ctx, t, 30_000_000_000)
    return {bid: ex.read(L2, bid) for bid in p.outputs}


def test_bulk_copy_wait_runs_out(monkeypatch):
    monkeypatch.setenv("VBE_STAGING", "256")  # every eligible run staged by bulk copies
    n = 1 << 20
    inp = bs_inputs(n, "float64")
    p = blackscholes(n, "float64", inputs=inp)
    with Executor(FLAGS, cache_dir=CACHE) as ex:
        got = run_failing_then_ordinary(ex, p)
    idx = np.sort(np.random.default_rng(3).choice(n, 4000, replace=False))
    sub = blackscholes(len(idx), "float64", inputs={k: v[idx] for k, v in inp.items()})
    want = oracle_outputs(sub)
    mx = np.maximum(inp["S"][idx], inp["K"][idx])
    for fb, sb in ((p.meta["call"], sub.meta["call"]), (p.meta["put"], sub.meta["put"])):
        assert np.all(np.abs(got[fb][idx] - want[sb]) <= 1e-12 * mx)


def test_tensor_copy_wait_runs_out(monkeypatch):
    monkeypatch.setenv("VBE_TILE", "t32x32")  # the tensor-copy form, read when the context is created
    p = gray_scott(2050, 1032, 1, "float32")
    with Executor(FLAGS, cache_dir=CACHE) as ex:
        got = run_failing_then_ordinary(ex, p)
        assert ex.stats()["tma_group_launches"] >= 2
    _exact_check(p)(got, oracle_outputs(p))
