"""The allocation-free sum entry point, for callers that must not let a
library allocate device memory on their hot path (work captured into a CUDA
graph by its caller, inference plugin enqueue functions, real-time loops).

Its result must agree with the regular executor's full ADD_REDUCE (reached
through vbe_submit) and with the oracle's ADD_REDUCE (the CPU reference
interpreter), within the reduction tolerance the parity tests use, on two
calls in a row (the second call reuses the fixed scratch the first one left
behind). This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1210_7774_b300 import build

build.build()

from paper_1210_7774_b300 import vbe as V  # noqa: E402
from paper_1210_7774_b300.runner import Executor  # noqa: E402
from workloads import ProgramBuilder  # noqa: E402

pytestmark = pytest.mark.gpu
RTOL = 1e-12  # float64 reductions: |got - want| <= RTOL * sum|x|


def sum_program(x: np.ndarray):
    b = ProgramBuilder("sum")
    xb = b.base("float64", x.size, x)
    s = b.base("float64", 1)
    b.emit("ADD_REDUCE", b.view(s, 0, (), ()), b.whole(xb), axis=0)
    return b.build([s]), s


def oracle_sum(x: np.ndarray) -> float:
    import oracle
    p, s = sum_program(x)
    return float(oracle.run(p)[s][0])


def executor_sum(x: np.ndarray) -> float:
    p, s = sum_program(x)
    with Executor(V.VBE_FUSE) as ex:
        L = ex.load(p)
        ex.run(L)
        return float(ex.read(L, s)[0])


@pytest.mark.parametrize("n", [10_000_019, 16384, 1, 0])
def test_noalloc_sum_matches_executor_twice(n):
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(n).standard_normal(n) * 3.0
    want = executor_sum(x) if n else 0.0
    ref = oracle_sum(x)
    dx = torch.from_numpy(x).cuda()
    out = torch.full((2,), np.nan, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    V.vbe_reduce_add_f64_noalloc(dx.data_ptr(), n, out.data_ptr(), stream)
    V.vbe_reduce_add_f64_noalloc(dx.data_ptr(), n, out.data_ptr() + 8, stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    bound = RTOL * max(np.abs(x).sum(), np.finfo(np.float64).tiny)
    for g in got:
        assert abs(g - want) <= bound, (g, want)  # the executor's ADD_REDUCE
        assert abs(g - ref) <= bound, (g, ref)    # the oracle's ADD_REDUCE
    assert got[0] == got[1]  # the order depends only on n


def test_noalloc_rejects_sizes_beyond_its_scratch():
    with pytest.raises(V.VbeError) as e:
        V.vbe_reduce_add_f64_noalloc(16, (1 << 30) + 1, 16, None)  # rejected before any launch
    assert e.value.code == -1
    with pytest.raises(V.VbeError):
        V.vbe_reduce_add_f64_noalloc(0, 10, 0, None)  # null pointers
