"""Random exact programs (``fuzz_programs``) recorded by the library and run
by the CPU emulation of its kernels, every access bounds-checked, against the
oracle bit for bit, fused and plain. The same programs run on the GPU in
``test_gpu_fuzz.py`` (many more seeds there)."""
import pytest

from paper_1210_7774_b300 import build

build.build()

from fuzz_programs import fuzz_cases  # noqa: E402
from parity_cases import oracle_outputs  # noqa: E402
from test_emulated_kernels import EMU, MODES, emulate  # noqa: E402

CASES = fuzz_cases(range(4))


@pytest.fixture(scope="module", autouse=True)
def _prebuild_fuzz_kernels():
    srcs = []
    for case in CASES:
        for mode in ("fused", "plain"):
            srcs += emulate(case.program, MODES[mode], (64, 1, 2), run=False)
    EMU.prebuild(srcs)


@pytest.mark.parametrize("mode", ["fused", "plain"])
@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_fuzz_emulated(case, mode):
    case.check(emulate(case.program, MODES[mode], (64, 1, 2)), oracle_outputs(case.program))
