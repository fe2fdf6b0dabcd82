"""Request mix for the serving loop: self-contained bytecode programs whose
inputs are generated on the device by RANDOM bytecodes, so requests carry
no host data in and only their results out.

Mix (seeded): half Jacobi solves on a grid of side log-uniform in
[128, 2048] (rounded to a multiple of 32), float32 or float64, 1..20
iterations; half Black-Scholes pricings of log-uniform 1K..4M options,
float32 or float64. Arrival times are a Poisson process.
"""
from __future__ import annotations

import numpy as np

from .blackscholes import _cnd
from .program import Const, ProgramBuilder

SEED = 1210_7774


def request_mix(n_req: int, seed: int = SEED + 5):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_req):
        dtype = "float32" if rng.random() < 0.5 else "float64"
        if rng.random() < 0.5:
            side = int(np.exp(rng.uniform(np.log(128), np.log(2048))))
            side = max(128, min(2048, (side // 32) * 32))
            out.append(("jacobi", dict(n=side, iters=int(rng.integers(1, 21)), dtype=dtype, seed=seed * 7 + i)))
        else:
            nopt = int(np.exp(rng.uniform(np.log(1024), np.log(4 << 20))))
            out.append(("blackscholes", dict(n=nopt, dtype=dtype, seed=seed * 11 + i)))
    return out


def poisson_arrivals(n_req: int, rate: float, seed: int = SEED + 6) -> np.ndarray:
    gaps = np.random.default_rng(seed).exponential(1.0 / rate, n_req)
    return np.cumsum(gaps)


def _uniform(b: ProgramBuilder, out_view, dtype, lo, hi, seed, key, tmp):
    """out = lo + (hi - lo) * U[0,1), drawn by RANDOM (float64) then cast."""
    b.emit("RANDOM", tmp, seed=seed, key=key, step=1)
    b.emit("MULTIPLY", tmp, tmp, Const(hi - lo))
    b.emit("ADD", tmp, tmp, Const(lo))
    if dtype == "float64":
        b.emit("COPY", out_view, tmp)
    else:
        b.emit("CAST", out_view, tmp)


def jacobi_request(n: int, iters: int, dtype: str, seed: int):
    """Grid with boundary 1.0 and a RANDOM interior, then ``iters`` Jacobi
    iterations; results: the grid and the last delta."""
    b = ProgramBuilder(f"req_jacobi{n}")
    m = n - 2
    full = b.base(dtype, (n, n))
    rnd = b.base("float64", (m, m))
    t = b.base(dtype, (m, m))
    d = b.base(dtype, (m, m))
    r = b.base(dtype, (m,))
    delta = b.base(dtype, (1,))
    b.emit("COPY", b.whole(full), Const(1.0))
    center = b.sub2d(full, 1, n - 1, 1, n - 1)
    b.emit("RANDOM", b.whole(rnd), seed=seed, key=0, step=1)
    b.emit("CAST" if dtype == "float32" else "COPY", center, b.whole(rnd))
    b.free(rnd)
    up = b.sub2d(full, 0, n - 2, 1, n - 1)
    down = b.sub2d(full, 2, n, 1, n - 1)
    left = b.sub2d(full, 1, n - 1, 0, n - 2)
    right = b.sub2d(full, 1, n - 1, 2, n)
    tv, dv, rv = b.whole(t), b.whole(d), b.whole(r)
    for _ in range(iters):
        b.emit("ADD", tv, up, down)
        b.emit("ADD", tv, tv, left)
        b.emit("ADD", tv, tv, right)
        b.emit("MULTIPLY", tv, tv, Const(0.25))
        b.emit("SUBTRACT", dv, center, tv)
        b.emit("ABSOLUTE", dv, dv)
        b.emit("ADD_REDUCE", rv, dv, axis=1)
        b.emit("ADD_REDUCE", b.view(delta, 0, (), ()), rv, axis=0)
        b.emit("COPY", center, tv)
        b.discard(t, d, r)
    b.sync(full, delta)
    p = b.build([full, delta])
    p.meta.update(kind="jacobi", cells=n * n, iters=iters, grid=full, delta=delta)
    return p


def blackscholes_request(n: int, dtype: str, seed: int):
    """RANDOM option parameters (same ranges as the Black-Scholes workload),
    then the pricing; results: call and put."""
    b = ProgramBuilder(f"req_bs{n}")
    tmp = b.whole(b.base("float64", n))
    ins = {}
    for k, (lo, hi) in zip("SKTV", ((10.0, 100.0), (10.0, 100.0), (0.1, 2.0), (0.1, 0.5))):
        ins[k] = b.whole(b.base(dtype, n))
        _uniform(b, ins[k], dtype, lo, hi, seed, "SKTV".index(k) << 32, tmp)
    ins["R"] = b.whole(b.base(dtype, n))
    b.emit("COPY", ins["R"], Const(0.05))
    b.free(tmp.base)
    call = b.base(dtype, n)
    put = b.base(dtype, n)
    names = ["a", "sT", "vsT", "q2", "d1", "d2", "n1", "n2", "x", "k", "p", "e", "w", "om", "disc", "Kd",
             "c1", "c2", "m1", "m2", "p1", "p2"]
    tv = {nm: b.whole(b.base(dtype, n)) for nm in names}
    c = b.whole(b.base("bool", n))
    S, K, T, R, V = (ins[k] for k in "SKTRV")
    b.emit("DIVIDE", tv["a"], S, K)
    b.emit("LOG", tv["a"], tv["a"])
    b.emit("SQRT", tv["sT"], T)
    b.emit("MULTIPLY", tv["vsT"], V, tv["sT"])
    b.emit("MULTIPLY", tv["q2"], V, V)
    b.emit("MULTIPLY", tv["q2"], tv["q2"], Const(0.5))
    b.emit("ADD", tv["q2"], R, tv["q2"])
    b.emit("MULTIPLY", tv["q2"], tv["q2"], T)
    b.emit("ADD", tv["d1"], tv["a"], tv["q2"])
    b.emit("DIVIDE", tv["d1"], tv["d1"], tv["vsT"])
    b.emit("SUBTRACT", tv["d2"], tv["d1"], tv["vsT"])
    tmp7 = (tv["x"], tv["k"], tv["p"], tv["e"], tv["w"], tv["om"], c)
    _cnd(b, dtype, n, tv["d1"], tv["n1"], tmp7)
    _cnd(b, dtype, n, tv["d2"], tv["n2"], tmp7)
    b.emit("MULTIPLY", tv["disc"], R, T)
    b.emit("NEGATIVE", tv["disc"], tv["disc"])
    b.emit("EXP", tv["disc"], tv["disc"])
    b.emit("MULTIPLY", tv["Kd"], K, tv["disc"])
    b.emit("MULTIPLY", tv["c1"], S, tv["n1"])
    b.emit("MULTIPLY", tv["c2"], tv["Kd"], tv["n2"])
    b.emit("SUBTRACT", b.whole(call), tv["c1"], tv["c2"])
    b.emit("SUBTRACT", tv["m2"], Const(1.0), tv["n2"])
    b.emit("MULTIPLY", tv["p1"], tv["Kd"], tv["m2"])
    b.emit("SUBTRACT", tv["m1"], Const(1.0), tv["n1"])
    b.emit("MULTIPLY", tv["p2"], S, tv["m1"])
    b.emit("SUBTRACT", b.whole(put), tv["p1"], tv["p2"])
    b.discard(*(v.base for v in tv.values()), c.base, *(v.base for v in ins.values()))
    b.sync(call, put)
    p = b.build([call, put])
    p.meta.update(kind="blackscholes", options=n, S=S.base, K=K.base)
    return p


def request_program(kind: str, params: dict):
    if kind == "jacobi":
        return jacobi_request(**params)
    return blackscholes_request(**params)
