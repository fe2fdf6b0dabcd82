"""The host-mirror ownership protocol through the C ABI on the CPU: a
recording context (bases in host memory), with every batch's recorded
launches and host <-> device copies executed by the emulator in order,
against the oracle's ownership model, on seeded scenarios: the ownership
state after every step, the host copy after every read access (bit for bit
wherever the model's value is defined) and the first rejected step."""
import pytest

from paper_1210_7774_b300 import build

build.build()

from paper_1210_7774_b300 import vbe as V  # noqa: E402

from emu.emulator import Emulator  # noqa: E402
from ownership_cases import run_library, run_model, same_observations, scenario  # noqa: E402

EMU = Emulator()


@pytest.mark.parametrize("flags", [V.VBE_FUSE | V.VBE_PACK | V.VBE_RECORD, V.VBE_RECORD], ids=["fused", "plain"])
@pytest.mark.parametrize("seed", range(12))
def test_mirror_protocol_matches_model(seed, flags):
    ops = scenario(seed)
    want = run_model(ops)
    got = run_library(ops, flags, emulator=EMU)
    assert same_observations(got, want)
