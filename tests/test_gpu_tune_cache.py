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


def _unusual_chain(n):
    """An elementwise chain no other test builds (its own tuning key)."""
    from workloads import Const, ProgramBuilder
    rng = np.random.default_rng(77)
    b = ProgramBuilder("tune_damage")
    x = b.base("float32", (n,), rng.standard_normal(n).astype(np.float32))
    y = b.base("float32", (n,), rng.standard_normal(n).astype(np.float32))
    o = b.base("float32", (n,), np.zeros(n, np.float32))
    X, Y, O = b.whole(x), b.whole(y), b.whole(o)
    b.emit("MAXIMUM", O, X, Y)
    b.emit("SUBTRACT", O, O, X)
    b.emit("MULTIPLY", O, O, Const(0.375))
    b.emit("ABSOLUTE", O, O)
    b.emit("MINIMUM", O, O, Y)
    b.emit("ADD", O, O, X)
    b.emit("NEGATIVE", O, O)
    return b.build([o])


def test_damaged_tuning_lines_are_ignored(tmp_path):
    """Lines of the tuning file that do not parse, carry an extra field or
    hold values the tuner never writes (block 0, U 0, an unknown register
    cap, a negative chunk) are dropped when a context loads the file; the
    context falls back on the process's own choices and computes the same,
    exact results."""
    cache = str(tmp_path)
    p = _unusual_chain((1 << 21) + 96)
    first, tunes = _run(p, cache)
    assert tunes > 0
    (path,) = glob.glob(os.path.join(cache, "tune_*.txt"))
    keys = [ln.split()[0] for ln in open(path) if ln.strip()]
    assert keys
    with open(path, "w") as f:
        for k in keys:
            f.write(f"{k} 0 1 0 0 0\n")       # block 0
            f.write(f"{k} 256 0 0 0 0\n")     # U 0
            f.write(f"{k} 256 1 7 0 0\n")     # a register cap the tuner never uses
            f.write(f"{k} 256 1 0 -16 0\n")   # negative chunk
            f.write(f"{k} 256 1 0 0 0 9\n")   # an extra field
            f.write(f"{k} 256\n")             # cut short
            f.write(f"{k} 2x6 1 0 0 0\n")     # not a number
    second, tunes2 = _run(p, cache)
    assert tunes2 == 0
    np.testing.assert_array_equal(second[p.outputs[0]], first[p.outputs[0]])
    want = oracle_outputs(p)
    assert_exact(second[p.outputs[0]], want[p.outputs[0]], p.name)
