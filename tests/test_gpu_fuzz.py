"""Random exact programs (``fuzz_programs``) on the GPU against the oracle,
bit for bit, float64 and float32: fused with packing, fused with graph
replay (each program run twice, so the second run replays), staged and
plain. The views alias, overlap in place and partially overlap their own
inputs, so every fusion break, the staging of overlapping operands and the
MIN/ARGMIN pairing are exercised on shapes the hand-written cases do not
have."""
import os

import pytest

from paper_1210_7774_b300 import build

build.build()

from paper_1210_7774_b300 import vbe as V  # noqa: E402
from paper_1210_7774_b300.runner import Executor  # noqa: E402

import oracle  # noqa: E402
from fuzz_programs import fuzz_cases, nd_cases, reduce_chain_cases, stencil_cases  # noqa: E402

pytestmark = pytest.mark.gpu
CACHE = os.environ.get("VBE_CACHE_DIR", "/tmp/vbe_kernel_cache")
FUSED = V.VBE_FUSE | V.VBE_PACK | V.VBE_AUTOTUNE
MODES = {"fused": (FUSED, 1, 0), "fused_graphs": (FUSED | V.VBE_GRAPHS, 2, 0), "fused_staged": (FUSED, 1, 64),
         "plain": (0, 1, 0)}
CASES = fuzz_cases(range(80)) + fuzz_cases(range(40), "float32")
REDCHAINS = reduce_chain_cases(range(40))
ND = nd_cases(range(40))
STENCILS = stencil_cases(range(40)) + stencil_cases(range(12), reduce=True)
# group forms forced by VBE_TILE ("" leaves the choice to the tuner)
FORMS = ["", "32x32", "s32x32", "t32x32", "r24", "r64"]


def _run(program, flags, repeat, staging, tile=""):
    saved = {k: os.environ.pop(k, None) for k in ("VBE_STAGING", "VBE_TILE")}
    if staging:
        os.environ["VBE_STAGING"] = str(staging)  # both read when the context is created
    if tile:
        os.environ["VBE_TILE"] = tile
    try:
        ex = Executor(flags, cache_dir=CACHE)
    finally:
        for k, v in saved.items():
            os.environ.pop(k, None)
            if v is not None:
                os.environ[k] = v
    with ex:
        L = ex.load(program)
        for _ in range(repeat):
            ex.run(L)
        return {bid: ex.read(L, bid) for bid in program.outputs}


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_fuzz_parity(case, mode):
    flags, repeat, staging = MODES[mode]
    # a second run starts from the state the first left: the oracle runs the
    # instructions as many times over the same memory
    mem = oracle.run(case.program, instrs=list(case.program.instrs) * repeat)
    case.check(_run(case.program, flags, repeat, staging), {bid: mem[bid] for bid in case.program.outputs})


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("case", REDCHAINS, ids=[c.name for c in REDCHAINS])
def test_fuzz_reduce_chains(case, mode):
    """Programs whose later instructions read reduction results (int64 sums,
    argmin/argmax indices) through broadcasts: dependencies through
    reductions across fusion breaks, staging and graph replay."""
    flags, repeat, staging = MODES[mode]
    mem = oracle.run(case.program, instrs=list(case.program.instrs) * repeat)
    case.check(_run(case.program, flags, repeat, staging), {bid: mem[bid] for bid in case.program.outputs})


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("case", ND, ids=[c.name for c in ND])
def test_fuzz_nd(case, mode):
    """Programs over views of rank 1 to 5 (axes in any order, reversed,
    strided, broadcast; reductions over every axis)."""
    flags, repeat, staging = MODES[mode]
    mem = oracle.run(case.program, instrs=list(case.program.instrs) * repeat)
    case.check(_run(case.program, flags, repeat, staging), {bid: mem[bid] for bid in case.program.outputs})


@pytest.mark.parametrize("tile", FORMS)
@pytest.mark.parametrize("case", STENCILS, ids=[c.name for c in STENCILS])
def test_fuzz_stencil_groups(case, tile):
    """Random stencil chains (tile-fused into one group, the input renamed
    when updated in place) in every group form, against the oracle bit for
    bit; graph replay, so the second pass of each chain replays."""
    got = _run(case.program, FUSED | V.VBE_GRAPHS, 1, 0, tile)
    mem = oracle.run(case.program)
    case.check(got, {bid: mem[bid] for bid in case.program.outputs})
