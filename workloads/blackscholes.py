"""Black-Scholes call and put pricing as elementwise bytecodes.

Not a workload of the paper: it stands for the long elementwise chains a
vectorised NumPy program sends through the Bridge (section "Bridge":
instructions are recorded into a batch until a flush). Inputs per option:
spot ``S``, strike ``K``, expiry ``T``, rate ``R`` (an array filled with
0.05) and volatility ``V``. The normal CDF is the Abramowitz & Stegun
26.2.17 polynomial with a SELECT on the sign of its argument:

    k = 1 / (1 + 0.2316419 |d|)
    w = phi(d) * k * (a1 + k (a2 + k (a3 + k (a4 + k a5))))
    N(d) = 1 - w if d > 0 else w

    d1 = (log(S/K) + (R + V^2/2) T) / (V sqrt(T)),  d2 = d1 - V sqrt(T)
    call = S N(d1) - K e^{-RT} N(d2)
    put  = K e^{-RT} (1 - N(d2)) - S (1 - N(d1))
"""
from __future__ import annotations

import numpy as np

from .program import Const, ProgramBuilder

SEED = 1210_7774

# Abramowitz & Stegun, Handbook of Mathematical Functions, formula 26.2.17
# (|error| < 7.5e-8): p and the five coefficients b1..b5.
AS_P = 0.2316419
AS_B = (0.319381530, -0.356563782, 1.781477937, -1.821255978, 1.330274429)
INV_SQRT_2PI = 0.3989422804014327  # 1/sqrt(2*pi), rounded to double


def bs_inputs(n: int, dtype: str = "float64", seed: int = SEED + 2) -> dict:
    """S, K ~ U[10,100], T ~ U[0.1,2], V ~ U[0.1,0.5], R = 0.05; drawn in
    float64 and then cast, so the float32 run prices the same options."""
    rng = np.random.default_rng(seed)
    S = rng.uniform(10.0, 100.0, n)
    K = rng.uniform(10.0, 100.0, n)
    T = rng.uniform(0.1, 2.0, n)
    V = rng.uniform(0.1, 0.5, n)
    R = np.full(n, 0.05)
    dt = np.dtype(dtype)
    return {k: v.astype(dt) for k, v in dict(S=S, K=K, T=T, R=R, V=V).items()}


def _cnd(b: ProgramBuilder, dtype: str, n: int, d, out, tmp):
    """Emit the A&S normal CDF of view ``d`` into view ``out``."""
    x, k, p, e, w, om, c = tmp
    b.emit("ABSOLUTE", x, d)
    b.emit("MULTIPLY", k, x, Const(AS_P))
    b.emit("ADD", k, k, Const(1.0))
    b.emit("DIVIDE", k, Const(1.0), k)
    b.emit("MULTIPLY", p, k, Const(AS_B[4]))
    for coef in (AS_B[3], AS_B[2], AS_B[1]):
        b.emit("ADD", p, p, Const(coef))
        b.emit("MULTIPLY", p, p, k)
    b.emit("ADD", p, p, Const(AS_B[0]))
    b.emit("MULTIPLY", p, p, k)
    b.emit("MULTIPLY", e, d, d)
    b.emit("MULTIPLY", e, e, Const(-0.5))
    b.emit("EXP", e, e)
    b.emit("MULTIPLY", e, e, Const(INV_SQRT_2PI))
    b.emit("MULTIPLY", w, e, p)
    b.emit("GREATER", c, d, Const(0.0))
    b.emit("SUBTRACT", om, Const(1.0), w)
    b.emit("SELECT", out, c, om, w)


def blackscholes(n: int = 1 << 24, dtype: str = "float64", seed: int = SEED + 2,
                 inputs: dict | None = None):
    """The Black-Scholes program over ``n`` options. Outputs: call, put."""
    b = ProgramBuilder(f"blackscholes{n}_{dtype}")
    inp = inputs if inputs is not None else bs_inputs(n, dtype, seed)
    S, K, T, R, V = (b.whole(b.base(dtype, n, inp[k])) for k in "SKTRV")
    call = b.base(dtype, n)
    put = b.base(dtype, n)
    names = ["a", "sT", "vsT", "q2", "d1", "d2", "n1", "n2", "x", "k", "p", "e", "w", "om",
             "disc", "Kd", "c1", "c2", "m1", "m2", "p1", "p2"]
    tb = {nm: b.base(dtype, n) for nm in names}
    cb = b.base("bool", n)
    tv = {nm: b.whole(i) for nm, i in tb.items()}
    c = b.whole(cb)
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
    tmp = (tv["x"], tv["k"], tv["p"], tv["e"], tv["w"], tv["om"], c)
    _cnd(b, dtype, n, tv["d1"], tv["n1"], tmp)
    _cnd(b, dtype, n, tv["d2"], tv["n2"], tmp)
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
    b.discard(*tb.values(), cb)
    b.sync(call, put)
    p = b.build([call, put])
    p.meta.update(n=n, dtype=dtype, call=call, put=put, inputs=inp,
                  input_ids={k: v.base for k, v in zip("SKTRV", (S, K, T, R, V))})
    return p
