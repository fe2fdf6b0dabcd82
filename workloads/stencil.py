"""Synthetic stencil: Gray-Scott reaction-diffusion on a 2-D grid, as bytecodes.

The paper's synthetic stencil benchmark (section "Performance Study",
10240 x 1024, ten steps) is not specified beyond its size and its heavy use
of slicing; the program here is a textbook two-field reaction-diffusion
stencil (Pearson, Science 261, 1993) written with shifted views. Fields ``U``
and ``V`` live on ``R x C`` bases whose outer ring stays fixed (Dirichlet).
One explicit Euler step (dt = dx = 1) on the interior, with the five-point
Laplacian ``L(A) = up + down + left + right - 4 A``:

    uvv = U V V
    U' = U + Du L(U) - uvv + F (1 - U)
    V' = V + Dv L(V) + uvv - (F + k) V

Every update is computed from the old fields into temporaries, then copied
into the interiors of ``U`` and ``V`` (so the step reads old values only).
The instruction order inside each line is fixed here and followed by both the
oracle and the executor.
"""
from __future__ import annotations

import numpy as np

from .program import Const, ProgramBuilder

SEED = 1210_7774
DU, DV, F, K = 0.16, 0.08, 0.035, 0.065


def stencil_inputs(R: int, C: int, dtype: str = "float64", seed: int = SEED + 6, patches: int = 12,
                   kind: str = "patches") -> dict:
    """Initial fields. ``patches``: U = 1, V = 0 with ``patches`` seeded
    squares (side R/16 capped at C/4) where U = 0.5, V = 0.25, plus uniform
    noise of amplitude 0.01 on V inside them. ``rest``: U = 1, V = 0."""
    U = np.ones((R, C))
    V = np.zeros((R, C))
    if kind == "patches":
        rng = np.random.default_rng(seed)
        s = max(2, min(R // 16, C // 4))
        for _ in range(patches):
            i = int(rng.integers(1, max(2, R - s - 1)))
            j = int(rng.integers(1, max(2, C - s - 1)))
            U[i:i + s, j:j + s] = 0.5
            V[i:i + s, j:j + s] = 0.25 + 0.01 * rng.random((min(s, R - i), min(s, C - j)))
    elif kind != "rest":
        raise ValueError(kind)
    return {"U": U.astype(dtype), "V": V.astype(dtype)}


def gray_scott(R: int = 10240, C: int = 1024, steps: int = 10, dtype: str = "float64", seed: int = SEED + 6,
               inputs: dict | None = None, Du: float = DU, Dv: float = DV, f: float = F, k: float = K):
    """The synthetic stencil program. Outputs: U, V. ``meta['batches']`` has
    one instruction range per step."""
    b = ProgramBuilder(f"stencil{R}x{C}_{dtype}_{steps}st")
    inp = inputs if inputs is not None else stencil_inputs(R, C, dtype, seed)
    U = b.base(dtype, (R, C), inp["U"])
    V = b.base(dtype, (R, C), inp["V"])
    n, m = R - 2, C - 2
    T = {name: b.base(dtype, (n, m)) for name in ("lu", "lv", "t", "uvv", "nu", "nv")}
    W = {name: b.whole(v) for name, v in T.items()}

    def around(q):
        return (b.sub2d(q, 0, n, 1, m + 1), b.sub2d(q, 2, n + 2, 1, m + 1),
                b.sub2d(q, 1, n + 1, 0, m), b.sub2d(q, 1, n + 1, 2, m + 2))

    cu, cv = b.sub2d(U, 1, n + 1, 1, m + 1), b.sub2d(V, 1, n + 1, 1, m + 1)
    batches = []
    for _ in range(steps):
        start = len(b.p.instrs)
        for lap, q, c in ((W["lu"], U, cu), (W["lv"], V, cv)):
            up, down, left, right = around(q)
            b.emit("ADD", lap, up, down)
            b.emit("ADD", lap, lap, left)
            b.emit("ADD", lap, lap, right)
            b.emit("MULTIPLY", W["t"], c, Const(4.0))
            b.emit("SUBTRACT", lap, lap, W["t"])
        b.emit("MULTIPLY", W["uvv"], cu, cv)
        b.emit("MULTIPLY", W["uvv"], W["uvv"], cv)
        # U' = U + Du L(U) - uvv + F (1 - U)
        b.emit("MULTIPLY", W["nu"], W["lu"], Const(Du))
        b.emit("SUBTRACT", W["nu"], W["nu"], W["uvv"])
        b.emit("SUBTRACT", W["t"], Const(1.0), cu)
        b.emit("MULTIPLY", W["t"], W["t"], Const(f))
        b.emit("ADD", W["nu"], W["nu"], W["t"])
        b.emit("ADD", W["nu"], W["nu"], cu)
        # V' = V + Dv L(V) + uvv - (F + k) V
        b.emit("MULTIPLY", W["nv"], W["lv"], Const(Dv))
        b.emit("ADD", W["nv"], W["nv"], W["uvv"])
        b.emit("MULTIPLY", W["t"], cv, Const(f + k))
        b.emit("SUBTRACT", W["nv"], W["nv"], W["t"])
        b.emit("ADD", W["nv"], W["nv"], cv)
        b.emit("COPY", cu, W["nu"])
        b.emit("COPY", cv, W["nv"])
        b.discard(*T.values())
        batches.append((start, len(b.p.instrs)))
    b.sync(U, V)
    p = b.build([U, V])
    batches[-1] = (batches[-1][0], len(p.instrs))
    p.meta.update(batches=batches, R=R, C=C, steps=steps, dtype=dtype, U=U, V=V, cells=R * C,
                  Du=Du, Dv=Dv, F=f, k=k)
    return p
