"""The multi-core blocked CPU interpreter (the paper's mcore engine, a CPU
baseline) against the oracle: the small parity cases under the same checks
as the GPU, with several thread and block counts (one block, fewer blocks
than threads, many ragged blocks), and the kernel formation of the paper's
blockable rule on the Jacobi iteration."""
import numpy as np
import pytest

import mcore
from parity_cases import all_small_cases, jacobi_case, oracle_outputs, workload_cases

mcore.build()

CASES = [c for c in all_small_cases() + workload_cases("medium")
         if not any(i.op.startswith("USER:") for i in c.program.instrs)]


@pytest.mark.parametrize("threads,blocks", [(1, 1), (4, 3), (3, 97)])
@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_mcore_matches_oracle(case, threads, blocks):
    # every kernel on the worker threads, however small
    got = mcore.run(case.program, threads=threads, blocks=blocks, inline_below=0)
    case.check({b: got[b] for b in case.program.outputs}, oracle_outputs(case.program))


def test_mcore_kernels_follow_the_blockable_rule():
    """A Jacobi iteration: the four shifted reads of the grid break no kernel
    (reads never conflict), the stencil sum, scaling and difference block
    together, each reduction is a kernel of its own, and the COPY back into
    the grid (which overlaps the shifted reads without being identical) ends
    up in a kernel of its own."""
    case = jacobi_case(40, 1)
    p = mcore.Prepared(case.program)
    p.run(threads=2, blocks=5, inline_below=0)
    # t=up+down, t+=left, t+=right, t*=.25, d=c-t, d=|d| | r=sum(d,1) | delta=sum(r,0) | center=t
    assert p.kernels == 4
