"""Shallow-water equations, two-step (Richtmyer) Lax-Wendroff, as bytecodes.

The paper's shallow-water benchmark (section "Performance Study") is a
translation of Burkardt's MATLAB program, which is not reproduced here; the
scheme is restated from the textbook. State: height ``H`` and momenta
``U = h u`` (along axis 0, "x") and ``V = h v`` (along axis 1, "y") on
``N x N`` bases that include a one-cell ghost ring (interior ``n = N-2``).
Gravity ``g``, spacings ``dx = dy = 1`` and time step ``dt``.

One step:

1. reflective ghost ring: copy ``H`` and the tangential momentum from the
   first interior row/column, negate the normal momentum (columns first,
   then rows);
2. cell fluxes on the whole grid: ``FxU = U^2/H + g/2 H^2``,
   ``FxV = U V / H`` (also the y-flux of ``U``), ``FyV = V^2/H + g/2 H^2``;
3. x half step on the ``(n+1) x n`` faces between rows ``f`` and ``f+1``:
   ``Q_x = (Q_hi + Q_lo)/2 - dt/(2dx) (F_hi - F_lo)`` for ``Q = H, U, V``
   with fluxes ``U, FxU, FxV``; then face fluxes ``Ux``,
   ``GxU = Ux^2/Hx + g/2 Hx^2``, ``GxV = Ux Vx / Hx``;
4. y half step on the ``n x (n+1)`` faces, fluxes ``V, FxV, FyV``; face
   fluxes ``Vy``, ``GyU = Vy Uy / Hy``, ``GyV = Vy^2/Hy + g/2 Hy^2``;
5. full step on the interior:
   ``Q -= dt/dx (Gx_hi - Gx_lo) + dt/dy (Gy_hi - Gy_lo)``
   (the two differences are subtracted one after the other).
"""
from __future__ import annotations

import numpy as np

from .program import Const, ProgramBuilder

SEED = 1210_7774
G = 9.8
DT = 0.1
DX = 1.0


def sw_inputs(N: int, dtype: str = "float64", seed: int = SEED + 3, centred: bool = False,
              kind: str = "droplet") -> dict:
    """Initial state. ``droplet``: ``H = 1 + 0.5 exp(-r^2 / (2 w^2))`` with
    ``w = N/16`` around a centre drawn uniformly in ``[0.4N, 0.6N]^2``
    (exactly the grid centre when ``centred``), ``U = V = 0``.
    ``rest``: ``H = 1``, ``U = V = 0``."""
    dt = np.dtype(dtype)
    if kind == "rest":
        H = np.ones((N, N))
    else:
        if centred:
            x0 = y0 = (N - 1) / 2.0
        else:
            x0, y0 = np.random.default_rng(seed).uniform(0.4 * N, 0.6 * N, 2)
        w = N / 16.0
        i = np.arange(N, dtype=np.float64)[:, None]
        j = np.arange(N, dtype=np.float64)[None, :]
        H = 1.0 + 0.5 * np.exp(-((i - x0) ** 2 + (j - y0) ** 2) / (2.0 * w * w))
    U = np.zeros((N, N))
    V = np.zeros((N, N))
    return {"H": H.astype(dt), "U": U.astype(dt), "V": V.astype(dt)}


def shallow_water(N: int = 4096, steps: int = 50, dtype: str = "float64", seed: int = SEED + 3,
                  inputs: dict | None = None, g: float = G, dt: float = DT, dx: float = DX):
    """The shallow-water program. Outputs: H, U, V. ``meta['batches']`` has
    one instruction range per time step."""
    b = ProgramBuilder(f"shallow_water{N}_{dtype}_{steps}st")
    inp = inputs if inputs is not None else sw_inputs(N, dtype, seed)
    n = N - 2
    H = b.base(dtype, (N, N), inp["H"])
    U = b.base(dtype, (N, N), inp["U"])
    V = b.base(dtype, (N, N), inp["V"])
    cx = dt / (2.0 * dx)
    kx = dt / dx

    def col(bid, j):
        return b.view(bid, j, (N,), (N,))

    def row(bid, i):
        return b.view(bid, i * N, (N,), (1,))

    # temporaries: cell fluxes (N x N), x faces ((n+1) x n), y faces (n x (n+1))
    cell = {k: b.base(dtype, (N, N)) for k in ("uh", "vh", "a", "hh", "b2", "FxU", "FxV", "FyV")}
    xf = {k: b.base(dtype, (n + 1, n)) for k in ("s", "df", "Hx", "Ux", "Vx", "uxh", "a", "hh",
                                                  "GxU", "GxV")}
    yf = {k: b.base(dtype, (n, n + 1)) for k in ("s", "df", "Hy", "Uy", "Vy", "vyh", "a", "hh",
                                                  "GyU", "GyV")}
    it = {k: b.base(dtype, (n, n)) for k in ("a", "b")}
    W = {k: b.whole(v) for k, v in cell.items()}
    X = {k: b.whole(v) for k, v in xf.items()}
    Y = {k: b.whole(v) for k, v in yf.items()}
    I = {k: b.whole(v) for k, v in it.items()}

    def xlo(bid):  # rows 0..n, cols 1..n of an N x N base
        return b.sub2d(bid, 0, n + 1, 1, n + 1)

    def xhi(bid):
        return b.sub2d(bid, 1, n + 2, 1, n + 1)

    def ylo(bid):  # rows 1..n, cols 0..n
        return b.sub2d(bid, 1, n + 1, 0, n + 1)

    def yhi(bid):
        return b.sub2d(bid, 1, n + 1, 1, n + 2)

    def half(T, out, qlo, qhi, flo, fhi, c):
        b.emit("ADD", T["s"], qhi, qlo)
        b.emit("MULTIPLY", T["s"], T["s"], Const(0.5))
        b.emit("SUBTRACT", T["df"], fhi, flo)
        b.emit("MULTIPLY", T["df"], T["df"], Const(c))
        b.emit("SUBTRACT", out, T["s"], T["df"])

    center = {q: b.sub2d(q, 1, n + 1, 1, n + 1) for q in (H, U, V)}
    batches = []
    for _ in range(steps):
        start = len(b.p.instrs)
        # 1. reflective ghost ring: columns, then rows
        for (dst, src) in ((0, 1), (N - 1, N - 2)):
            b.emit("COPY", col(H, dst), col(H, src))
            b.emit("COPY", col(U, dst), col(U, src))
            b.emit("NEGATIVE", col(V, dst), col(V, src))
        for (dst, src) in ((0, 1), (N - 1, N - 2)):
            b.emit("COPY", row(H, dst), row(H, src))
            b.emit("NEGATIVE", row(U, dst), row(U, src))
            b.emit("COPY", row(V, dst), row(V, src))
        # 2. cell fluxes on the whole grid
        Hw, Uw, Vw = b.whole(H), b.whole(U), b.whole(V)
        b.emit("DIVIDE", W["uh"], Uw, Hw)
        b.emit("DIVIDE", W["vh"], Vw, Hw)
        b.emit("MULTIPLY", W["a"], Uw, W["uh"])
        b.emit("MULTIPLY", W["hh"], Hw, Hw)
        b.emit("MULTIPLY", W["hh"], W["hh"], Const(g / 2.0))
        b.emit("ADD", W["FxU"], W["a"], W["hh"])
        b.emit("MULTIPLY", W["FxV"], Uw, W["vh"])
        b.emit("MULTIPLY", W["b2"], Vw, W["vh"])
        b.emit("ADD", W["FyV"], W["b2"], W["hh"])
        # 3. x half step and x-face fluxes
        half(X, X["Hx"], xlo(H), xhi(H), xlo(U), xhi(U), cx)
        half(X, X["Ux"], xlo(U), xhi(U), xlo(cell["FxU"]), xhi(cell["FxU"]), cx)
        half(X, X["Vx"], xlo(V), xhi(V), xlo(cell["FxV"]), xhi(cell["FxV"]), cx)
        b.emit("DIVIDE", X["uxh"], X["Ux"], X["Hx"])
        b.emit("MULTIPLY", X["a"], X["Ux"], X["uxh"])
        b.emit("MULTIPLY", X["hh"], X["Hx"], X["Hx"])
        b.emit("MULTIPLY", X["hh"], X["hh"], Const(g / 2.0))
        b.emit("ADD", X["GxU"], X["a"], X["hh"])
        b.emit("MULTIPLY", X["GxV"], X["Vx"], X["uxh"])
        # 4. y half step and y-face fluxes
        half(Y, Y["Hy"], ylo(H), yhi(H), ylo(V), yhi(V), cx)
        half(Y, Y["Uy"], ylo(U), yhi(U), ylo(cell["FxV"]), yhi(cell["FxV"]), cx)
        half(Y, Y["Vy"], ylo(V), yhi(V), ylo(cell["FyV"]), yhi(cell["FyV"]), cx)
        b.emit("DIVIDE", Y["vyh"], Y["Vy"], Y["Hy"])
        b.emit("MULTIPLY", Y["GyU"], Y["Uy"], Y["vyh"])
        b.emit("MULTIPLY", Y["a"], Y["Vy"], Y["vyh"])
        b.emit("MULTIPLY", Y["hh"], Y["Hy"], Y["Hy"])
        b.emit("MULTIPLY", Y["hh"], Y["hh"], Const(g / 2.0))
        b.emit("ADD", Y["GyV"], Y["a"], Y["hh"])
        # 5. full step on the interior
        for q, gx, gy in ((H, xf["Ux"], yf["Vy"]), (U, xf["GxU"], yf["GyU"]),
                          (V, xf["GxV"], yf["GyV"])):
            b.emit("SUBTRACT", I["a"], b.sub2d(gx, 1, n + 1, 0, n), b.sub2d(gx, 0, n, 0, n))
            b.emit("MULTIPLY", I["a"], I["a"], Const(kx))
            b.emit("SUBTRACT", I["b"], b.sub2d(gy, 0, n, 1, n + 1), b.sub2d(gy, 0, n, 0, n))
            b.emit("MULTIPLY", I["b"], I["b"], Const(kx))
            b.emit("SUBTRACT", center[q], center[q], I["a"])
            b.emit("SUBTRACT", center[q], center[q], I["b"])
        b.discard(*cell.values(), *xf.values(), *yf.values(), *it.values())
        batches.append((start, len(b.p.instrs)))
    b.sync(H, U, V)
    p = b.build([H, U, V])
    batches[-1] = (batches[-1][0], len(p.instrs))
    p.meta.update(batches=batches, N=N, steps=steps, dtype=dtype, H=H, U=U, V=V,
                  cells=N * N, g=g, dt=dt, dx=dx)
    return p
