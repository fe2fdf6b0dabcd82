"""Failure detection of the bounded device waits, on the CPU: kernels that
stage their inputs by bulk copies (one-dimensional runs) or by tensor copies
(tile-fused groups in the tensor-copy form) are recorded and executed by the
emulator (1) with copies that never land and (2) with the compute threads'
wait limit set to zero polls (vbe_debug_set_wait_polls, the setting the GPU
test uses). Either way every wait ends, the kernel reports through the
context's error word, vbe_wait returns VBE_ERR_TIMEOUT, no mbarrier phase
ever receives a second copy (the emulator checks the phase accounting), and
the next ordinary batch on the same context matches the oracle."""
import json

import numpy as np
import pytest

from paper_1210_7774_b300 import build

build.build()

from paper_1210_7774_b300 import vbe as V  # noqa: E402
from paper_1210_7774_b300.runner import Executor  # noqa: E402

from emu.emulator import Emulator  # noqa: E402
from parity_cases import _exact_check, oracle_outputs  # noqa: E402
from workloads import blackscholes, gray_scott  # noqa: E402

EMU = Emulator()
FLAGS = V.VBE_FUSE | V.VBE_PACK | V.VBE_RECORD


def context(monkeypatch, env):
    for k, v in env.items():  # read when the context is created, or at planning
        monkeypatch.setenv(k, v)
    return Executor(FLAGS)


def entries(rec):
    return [x.get("entry", "copy") for x in json.loads(rec)["launches"]]


FORMS = {
    # one-dimensional runs staged by bulk copies, 64-element chunks
    "bulk": ({"VBE_STAGING": "64", "VBE_RECORD_BLOCK": "64", "VBE_RECORD_U": "1", "VBE_RECORD_SMS": "2"},
             lambda: blackscholes(3000, "float64")),
    # a tile-fused group in the tensor-copy form (producer warp, two stages)
    "tensor": ({"VBE_RECORD_TILE": "t32x32", "VBE_RECORD_BLOCK": "64", "VBE_RECORD_U": "1", "VBE_RECORD_SMS": "1"},
               lambda: gray_scott(70, 100, 1, "float32")),
}


@pytest.mark.parametrize("how", ["copies_never_land", "zero_polls"])
@pytest.mark.parametrize("form", list(FORMS))
def test_wait_runs_out_and_context_stays_usable(form, how, monkeypatch):
    env, make = FORMS[form]
    p = make()
    with context(monkeypatch, env) as ex:
        L = ex.load(p)
        if how == "zero_polls":
            V.vbe_debug_set_wait_polls(ex.ctx, 0)
        for k in range(len(L.batches)):
            ex.submit(L, k)
            rec = V.vbe_debug_take_launches(ex.ctx)
            names = entries(rec)
            assert any(n.endswith("_tm32x32") if form == "tensor" else n.endswith("_bulk") for n in names), names
            EMU.run(rec, drop_copies=(how == "copies_never_land"))
        with pytest.raises(V.VbeError) as e:
            V.vbe_wait(ex.ctx, 0, 1_000_000_000)
        assert e.value.code == -8  # VBE_ERR_TIMEOUT
        # the error was reported once; the context runs the next batch normally
        V.vbe_debug_set_wait_polls(ex.ctx, -1)
        L2 = ex.load(p)
        for k in range(len(L2.batches)):
            ex.submit(L2, k)
            EMU.run(V.vbe_debug_take_launches(ex.ctx))
        V.vbe_wait(ex.ctx, 0, 1_000_000_000)
        got = {bid: ex.read(L2, bid) for bid in p.outputs}
    want = oracle_outputs(p)
    if form == "tensor":
        _exact_check(p)(got, want)
    else:
        mx = np.maximum(p.bases[1].init, p.bases[2].init)
        for bid in p.outputs:
            assert np.all(np.abs(got[bid] - want[bid]) <= 1e-12 * mx)


def test_wait_limit_is_part_of_the_kernel_source(monkeypatch):
    """The zero-poll setting compiles different kernels (the limit is defined
    ahead of the source, so it is part of the cache key); restoring it
    returns to the normal ones."""
    env, make = FORMS["bulk"]
    p = make()
    with context(monkeypatch, env) as ex:
        L = ex.load(p)
        srcs = []
        for polls in (-1, 0, -1):
            V.vbe_debug_set_wait_polls(ex.ctx, polls)
            ex.submit(L, 0)
            js = json.loads(V.vbe_debug_take_launches(ex.ctx))
            srcs.append([js["sources"][x["key"]] for x in js["launches"] if "key" in x])
        assert any(s.startswith("#define VBE_CWAIT 0u") for s in srcs[1])
        assert not any(s.startswith("#define VBE_CWAIT") for s in srcs[0] + srcs[2])
        with pytest.raises(V.VbeError):
            V.vbe_debug_set_wait_polls(ex.ctx, (1 << 24) + 1)
