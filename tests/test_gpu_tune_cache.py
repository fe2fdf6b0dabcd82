"""Tuning choices persist in the cache directory: a second context (as a
second process would) on the same directory reuses them instead of timing
the candidates again, and computes the same results."""
import glob
import os

import numpy as np
import pytest

from paper_1210_7774_b300 import build

build.build()

from paper_1210_7774_b300 import vbe as V  # noqa: E402
from paper_1210_7774_b300.runner import Executor  # noqa: E402

from parity_cases import assert_exact, oracle_outputs  # noqa: E402
from workloads import blackscholes, bs_inputs, shallow_water  # noqa: E402

pytestmark = pytest.mark.gpu


def _run(program, cache):
    with Executor(V.VBE_FUSE | V.VBE_PACK | V.VBE_AUTOTUNE, cache_dir=cache) as ex:
        L = ex.load(program)
        ex.run(L)
        out = {bid: ex.read(L, bid) for bid in program.outputs}
        return out, ex.stats()["autotunes"]


def test_tuning_choices_reused_across_contexts(tmp_path):
    cache = str(tmp_path)
    n = 1 << 21  # above the size the tuner times
    bs = blackscholes(n, "float32", inputs=bs_inputs(n, "float32"))
    sw = shallow_water(520, 2, "float32")  # a tile-fused group (tile shape and form tuned)
    first = {p.name: _run(p, cache) for p in (bs, sw)}
    assert all(t > 0 for _, t in first.values())
    files = glob.glob(os.path.join(cache, "tune_*.txt"))
    assert len(files) == 1 and os.path.getsize(files[0]) > 0
    for p in (bs, sw):
        out, tunes = _run(p, cache)
        assert tunes == 0, p.name
        for bid in p.outputs:
            np.testing.assert_array_equal(out[bid], first[p.name][0][bid])
    want = oracle_outputs(sw)
    for bid in sw.outputs:
        assert_exact(first[sw.name][0][bid], want[bid], sw.name)


def test_tuning_choices_shared_by_contexts_of_a_process():
    """Contexts of one process (a server's scheduler threads) share their
    choices even without a cache directory: the second context tunes
    nothing and computes the same results."""
    n = (1 << 23) + 4096  # a size class no other test tunes in this process
    bs = blackscholes(n, "float64", inputs=bs_inputs(n, "float64"))
    first, tunes = _run(bs, None)
    assert tunes > 0
    second, tunes2 = _run(bs, None)
    assert tunes2 == 0
    for bid in bs.outputs:
        np.testing.assert_array_equal(first[bid], second[bid])
