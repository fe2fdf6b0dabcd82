"""The host-mirror ownership protocol on the GPU: the seeded scenarios of
the CPU test (host writes with write access, read access, in-batch SYNC and
DISCARD, rejected batches) through the C ABI against the oracle's
ownership model, with repeated batches replayed (graphs) and without, and
one scenario whose batches run on a 2048 x 2048 grid."""
import os

import numpy as np
import pytest

from paper_1210_7774_b300 import build

build.build()

from paper_1210_7774_b300 import vbe as V  # noqa: E402

import ownership_cases as oc  # noqa: E402

pytestmark = pytest.mark.gpu
CACHE = os.environ.get("VBE_CACHE_DIR", "/tmp/vbe_kernel_cache")
FLAGS = {"fused_graphs": V.VBE_FUSE | V.VBE_PACK | V.VBE_GRAPHS, "plain": 0}


@pytest.mark.parametrize("mode", list(FLAGS))
@pytest.mark.parametrize("seed", range(12))
def test_mirror_protocol_matches_model_on_gpu(seed, mode):
    ops = oc.scenario(seed)
    want = oc.run_model(ops)
    got = oc.run_library(ops, FLAGS[mode], cache_dir=CACHE)
    assert oc.same_observations(got, want)


def test_mirror_protocol_large_grid(monkeypatch):
    """The same rules with 2048 x 2048 bases (32 MiB each): copies to and from
    the mirror of that size, a long scenario."""
    monkeypatch.setattr(oc, "SHAPE", (2048, 2048))
    ops = oc.scenario(101, steps=30)
    want = oc.run_model(ops)
    got = oc.run_library(ops, FLAGS["fused_graphs"], cache_dir=CACHE)
    assert oc.same_observations(got, want)
    assert sum(1 for o in want if o[1] == "host") >= 3
