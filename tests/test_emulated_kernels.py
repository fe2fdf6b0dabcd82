"""The generated kernels executed on the CPU: a VBE_RECORD context records
every launch the executor makes (the same analysis, code generation,
launch shapes and parameter blocks as on the GPU) and the emulator runs
them with every memory access bounds-checked. Results must match the
oracle under the same rules as the GPU parity tests. This checks the index
arithmetic of every kernel form on the host before it runs on a device."""
import collections
import json
import os
import re

import pytest

from paper_1210_7774_b300 import build

build.build()

from paper_1210_7774_b300 import vbe as V  # noqa: E402
from paper_1210_7774_b300.runner import Executor  # noqa: E402

from emu.emulator import Emulator  # noqa: E402
from parity_cases import (Case, _exact_check, all_small_cases, jacobi_case, oracle_outputs,  # noqa: E402
                          tile_group_cases)
from workloads import gray_scott, shallow_water  # noqa: E402

CASES = all_small_cases()
EMU = Emulator()
# launched tile-fused group kernels by form (the suffix letters of their entry)
GROUP_FORMS = collections.Counter()

MODES = {
    "fused": V.VBE_FUSE | V.VBE_PACK | V.VBE_RECORD,
    "plain": V.VBE_RECORD,
    # fused, with every eligible one-dimensional run staged through shared
    # memory by bulk copies in chunks of 64 elements (several chunks per
    # block, and a tail, at these sizes)
    "staged": V.VBE_FUSE | V.VBE_PACK | V.VBE_RECORD,
}
STAGING = {"staged": 64}
# launch shapes: (block, U, SMs) -- several, so that multi-block and ragged
# tiles are exercised
SHAPES = [(64, 1, 2), (32, 4, 3), (128, 2, 1)]


def emulate(program, flags, shape, run=True, staging=0):
    block, U, sms = shape
    os.environ["VBE_STAGING"] = str(staging)  # read when the context is created
    os.environ["VBE_RECORD_BLOCK"] = str(block)
    os.environ["VBE_RECORD_U"] = str(U)
    os.environ["VBE_RECORD_SMS"] = str(sms)
    sources = []
    ex = Executor(flags)
    os.environ.pop("VBE_STAGING")
    with ex:
        L = ex.load(program)
        for k in range(len(L.batches)):
            ex.submit(L, k)
            rec = V.vbe_debug_take_launches(ex.ctx)
            for launch in json.loads(rec)["launches"]:
                m = re.search(r"_(s[gs]|tm|rs)\d+x\d+$", launch.get("entry", ""))
                if m:
                    GROUP_FORMS[m.group(1)] += 1
            if run:
                EMU.run(rec)
            else:
                sources += list(json.loads(rec)["sources"].values())
        if not run:
            return sources
        return {bid: ex.read(L, bid) for bid in program.outputs}


@pytest.fixture(scope="module", autouse=True)
def _prebuild_kernels():
    """Record every case once (launch records do not depend on data) and
    compile all distinct kernel sources in parallel before the tests run."""
    srcs = []
    for case in CASES:
        for mode, flags in MODES.items():
            srcs += emulate(case.program, flags, SHAPES[hash(case.name) % len(SHAPES)], run=False,
                            staging=STAGING.get(mode, 0))
    EMU.prebuild(srcs)


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_emulated_parity(case, mode):
    want = oracle_outputs(case.program)
    shape = SHAPES[hash(case.name) % len(SHAPES)]
    got = emulate(case.program, MODES[mode], shape, staging=STAGING.get(mode, 0))
    case.check(got, want)


@pytest.mark.parametrize("shape", SHAPES)
def test_emulated_shapes_on_stencil_and_packing(shape):
    for case in CASES:
        if case.name.startswith(("jacobi", "mcpi", "shallow_water24", "chain_full_float32")):
            want = oracle_outputs(case.program)
            got = emulate(case.program, MODES["fused"], shape)
            case.check(got, want)


@pytest.mark.parametrize("tile", ["8x16", "16x32", "32x32", "s32x32", "s16x64", "t32x32", "t16x64", "r32", "r64", "split"])
def test_emulated_tile_groups(tile):
    """Tile-fused groups at several tile shapes (ragged edge tiles, halos
    across tile borders): shallow water (state renamed every step, ghost
    ring copied across) and the synthetic chains, with the inputs read
    through L1, staged through shared memory ("s" shapes) or brought in by
    double-buffered tensor copies ("t" shapes), or swept down the rows by one
    warp per column strip with values in registers ("r": strips of 32 or 64
    rows); and the same groups run as their separate kernels (the choice the
    tuner makes when that is faster)."""
    cases = tile_group_cases()
    if tile.startswith(("t", "r")):  # rows of 16-byte multiples, as tensor copies need
        cases += tile_group_cases(seed=12, N=37, M=52)
    if tile.startswith("t"):
        cases.append(jacobi_case(66, 3))  # stencil, reductions and copy back: a group with a whole-run reduction
    for dt in ("float64", "float32"):
        p = shallow_water(40, 2, dt)
        cases.append(Case(p.name, p, _exact_check(p)))
    if tile.startswith("r"):
        # strips of 32 or 64 rows over 70 rows: full and ragged strips,
        # several warps side by side and a ragged last column strip
        p = shallow_water(72, 2, "float32")
        cases.append(Case(p.name, p, _exact_check(p)))
        p = gray_scott(70, 44, 2, "float64")  # a stacked group with stencil inputs
        cases.append(Case(p.name, p, _exact_check(p)))
        p = shallow_water(35, 2, "float64")  # 33 anchor rows: a last strip of one row
        cases.append(Case(p.name, p, _exact_check(p)))
    before = GROUP_FORMS["rs"]
    var = "VBE_RECORD_SPLIT" if tile == "split" else "VBE_RECORD_TILE"
    os.environ[var] = tile
    # one SM for the tensor-copy form: its two persistent blocks each walk
    # several tiles through both stages
    shape = (64, 1, 1) if tile.startswith("t") else (64, 1, 2)
    try:
        for case in cases:
            got = emulate(case.program, MODES["fused"], shape)
            case.check(got, oracle_outputs(case.program))
    finally:
        os.environ.pop(var)
    if tile.startswith("r"):
        assert GROUP_FORMS["rs"] > before, "no group ran in the row-sweep form"
