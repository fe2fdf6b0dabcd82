"""Batched Monte-Carlo estimate of pi: many independent instances of uneven
size, each a short bytecode chain ending in an integer reduction.

Not a workload of the paper; it exercises the paper's rule that
independent instructions may be executed together (section "Vector
Engine": kernels are formed from instructions that share no data) across
many small uneven problems.

Per instance ``i`` with ``n_i`` samples::

    RANDOM x (key = i<<32 | 0, step 2); RANDOM y (key = i<<32 | 1, step 2)
    x = x*x; y = y*y; x = x + y; c = x <= 1.0; ci = CAST(c -> int64)
    count[i] = ADD_REDUCE(ci, axis=0)

RANDOM draws element ``m`` of its output from the counter
``c = key + step*m`` (mod 2^64) with the splitmix64 finaliser applied to
``seed + (c + 1) * 0x9e3779b97f4a7c15`` and the top 53 bits scaled by
2^-53, so instance 0 reproduces a sequential splitmix64 stream with x and
y interleaved.
"""
from __future__ import annotations

import numpy as np

from .program import Const, ProgramBuilder

SEED = 1210_7774


def mc_sizes(n_inst: int = 256, seed: int = SEED + 4, lo: int = 10, hi: int = 24) -> np.ndarray:
    """n_i = floor(2^(lo + (hi - lo) u_i)), u_i ~ U[0,1) from ``seed``."""
    u = np.random.default_rng(seed).random(n_inst)
    return np.floor(np.exp2(lo + (hi - lo) * u)).astype(np.int64)


def montecarlo_pi(n_inst: int = 256, seed: int = SEED + 4, sizes=None, draw_seed: int | None = None,
                  keys=None):
    """The MC-pi program. Output: ``count`` (int64, one per instance).
    ``keys`` gives the instance numbers used in the counters (default
    0..n-1), so that a few instances of a large configuration can be
    rebuilt on their own."""
    sizes = mc_sizes(n_inst, seed) if sizes is None else np.asarray(sizes, dtype=np.int64)
    n_inst = len(sizes)
    keys = list(range(n_inst)) if keys is None else [int(k) for k in keys]
    draw_seed = seed if draw_seed is None else draw_seed
    b = ProgramBuilder(f"mcpi{n_inst}")
    count = b.base("int64", n_inst)
    for i, (n, inst) in enumerate(zip(sizes.tolist(), keys)):
        x = b.base("float64", n)
        y = b.base("float64", n)
        c = b.base("bool", n)
        ci = b.base("int64", n)
        xv, yv, cv, civ = b.whole(x), b.whole(y), b.whole(c), b.whole(ci)
        b.emit("RANDOM", xv, seed=draw_seed, key=(inst << 32) | 0, step=2)
        b.emit("RANDOM", yv, seed=draw_seed, key=(inst << 32) | 1, step=2)
        b.emit("MULTIPLY", xv, xv, xv)
        b.emit("MULTIPLY", yv, yv, yv)
        b.emit("ADD", xv, xv, yv)
        b.emit("LESS_EQUAL", cv, xv, Const(1.0))
        b.emit("CAST", civ, cv)
        b.emit("ADD_REDUCE", b.view(count, i, (), ()), civ, axis=0)
        # the temporaries' values are dead; the handles stay valid so the
        # same batch can be submitted again
        b.discard(x, y, c, ci)
    b.sync(count)
    p = b.build([count])
    p.meta.update(sizes=sizes, count=count, samples=int(sizes.sum()), seed=draw_seed)
    return p
