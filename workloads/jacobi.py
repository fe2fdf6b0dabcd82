"""Jacobi 5-point stencil as bytecodes (section "Numerical Python", the
stencil example, and the Jacobi benchmark of section "Performance Study").

The grid is a ``n x n`` base; ``center/up/down/left/right`` are the shifted
views of the stencil example. One iteration is nine bytecodes:

    t = up + down; t = t + left; t = t + right; t = t * 0.25
    d = center - t; d = |d|; r = ADD_REDUCE(d, axis=1)
    delta[k] = ADD_REDUCE(r, axis=0); center = t

followed by DISCARD of the temporaries ``t, d, r`` so their handles are
reused by the next iteration. The example in the paper (weight 0.2, a
``work`` copy and an un-updated ``delta``) is illustrative; the program here
follows the nine-bytecode form with weight 0.25.
"""
from __future__ import annotations

import numpy as np

from .program import Const, ProgramBuilder

SEED = 1210_7774


def jacobi_inputs(n: int, dtype: str = "float64", seed: int = SEED + 1,
                  init: str = "random", linear=(1, 2, 3)) -> np.ndarray:
    """Initial grid. ``random``: interior uniform[0,1) from ``seed`` and the
    boundary ring fixed at 1.0. ``linear``: every cell ``a + b*i + c*j``
    (small integers, so the stencil arithmetic is exact)."""
    if init == "random":
        rng = np.random.default_rng(seed)
        g = np.ones((n, n), dtype=np.float64)
        g[1:-1, 1:-1] = rng.random((n - 2, n - 2))
    elif init == "linear":
        a, b, c = linear
        i = np.arange(n, dtype=np.float64)[:, None]
        j = np.arange(n, dtype=np.float64)[None, :]
        g = a + b * i + c * j
    else:
        raise ValueError(init)
    return g.astype(np.dtype(dtype))


def jacobi(n: int = 256, iters: int = 10, dtype: str = "float64",
           seed: int = SEED + 1, init: str = "random", linear=(1, 2, 3), history: bool = False,
           one_batch: bool = False):
    """The Jacobi program. Outputs: the grid and ``deltas``: the scalar delta
    of the last iteration (every iteration overwrites it, so all iterations
    are the same batch), or with ``history`` the delta of each iteration.
    ``meta['batches']`` lists one instruction range per iteration, or with
    ``one_batch`` a single range: the whole program is one batch, as the
    paper's Bridge hands over everything recorded up to a flush."""
    b = ProgramBuilder(f"jacobi{n}_{dtype}_{iters}it")
    grid = jacobi_inputs(n, dtype, seed, init, linear)
    full = b.base(dtype, (n, n), grid)
    m = n - 2
    center = b.sub2d(full, 1, n - 1, 1, n - 1)
    up = b.sub2d(full, 0, n - 2, 1, n - 1)
    down = b.sub2d(full, 2, n, 1, n - 1)
    left = b.sub2d(full, 1, n - 1, 0, n - 2)
    right = b.sub2d(full, 1, n - 1, 2, n)
    t = b.base(dtype, (m, m))
    d = b.base(dtype, (m, m))
    r = b.base(dtype, (m,))
    deltas = b.base(dtype, (iters if history else 1,))
    tv, dv, rv = b.whole(t), b.whole(d), b.whole(r)
    batches = []
    for k in range(iters):
        start = len(b.p.instrs)
        b.emit("ADD", tv, up, down)
        b.emit("ADD", tv, tv, left)
        b.emit("ADD", tv, tv, right)
        b.emit("MULTIPLY", tv, tv, Const(0.25))
        b.emit("SUBTRACT", dv, center, tv)
        b.emit("ABSOLUTE", dv, dv)
        b.emit("ADD_REDUCE", rv, dv, axis=1)
        b.emit("ADD_REDUCE", b.view(deltas, k if history else 0, (), ()), rv, axis=0)
        b.emit("COPY", center, tv)
        b.discard(t, d, r)
        batches.append((start, len(b.p.instrs)))
    b.sync(full, deltas)
    p = b.build([full, deltas])
    batches[-1] = (batches[-1][0], len(p.instrs))
    if one_batch:
        batches = [(0, len(p.instrs))]
    p.meta.update(batches=batches, n=n, iters=iters, dtype=dtype, grid=full, deltas=deltas,
                  elements_per_iter=m * m)
    return p
