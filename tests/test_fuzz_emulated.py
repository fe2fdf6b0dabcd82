"""Random exact programs (``fuzz_programs``) recorded by the library and run
by the CPU emulation of its kernels, every access bounds-checked, against the
oracle bit for bit, fused and plain. The same programs run on the GPU in
``test_gpu_fuzz.py`` (many more seeds there)."""
import pytest

from paper_1210_7774_b300 import build

build.build()

import os  # noqa: E402

from fuzz_programs import fuzz_cases, nd_cases, reduce_chain_cases, stencil_cases  # noqa: E402
from parity_cases import oracle_outputs  # noqa: E402
from test_emulated_kernels import EMU, MODES, emulate  # noqa: E402

CASES = fuzz_cases(range(4)) + fuzz_cases(range(2), "float32")
REDCHAINS = reduce_chain_cases(range(3))
ND = nd_cases(range(3)) + nd_cases(range(2), "float32")
STENCILS = stencil_cases(range(3))
RED_STENCILS = stencil_cases(range(2), reduce=True)
FORMS = ["8x16", "s32x32", "t32x32", "r32"]


@pytest.fixture(scope="module", autouse=True)
def _prebuild_fuzz_kernels():
    srcs = []
    for case in CASES + REDCHAINS + ND:
        for mode in ("fused", "plain"):
            srcs += emulate(case.program, MODES[mode], (64, 1, 2), run=False)
    EMU.prebuild(srcs)


@pytest.mark.parametrize("mode", ["fused", "plain"])
@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_fuzz_emulated(case, mode):
    case.check(emulate(case.program, MODES[mode], (64, 1, 2)), oracle_outputs(case.program))


@pytest.mark.parametrize("mode", ["fused", "plain"])
@pytest.mark.parametrize("case", REDCHAINS, ids=[c.name for c in REDCHAINS])
def test_fuzz_reduce_chains_emulated(case, mode):
    """Random programs that read reduction results later in the batch."""
    case.check(emulate(case.program, MODES[mode], (64, 1, 2)), oracle_outputs(case.program))


@pytest.mark.parametrize("mode", ["fused", "plain"])
@pytest.mark.parametrize("case", ND, ids=[c.name for c in ND])
def test_fuzz_nd_emulated(case, mode):
    """Random programs over views of rank 1 to 5."""
    case.check(emulate(case.program, MODES[mode], (64, 1, 2)), oracle_outputs(case.program))


@pytest.mark.parametrize("tile", FORMS)
@pytest.mark.parametrize("case", STENCILS + RED_STENCILS, ids=[c.name for c in STENCILS + RED_STENCILS])
def test_fuzz_stencil_emulated(case, tile):
    """Random stencil chains in each group form (VBE_RECORD_TILE), emulated."""
    os.environ["VBE_RECORD_TILE"] = tile
    try:
        got = emulate(case.program, MODES["fused"], (64, 1, 2))
    finally:
        os.environ.pop("VBE_RECORD_TILE")
    case.check(got, oracle_outputs(case.program))
