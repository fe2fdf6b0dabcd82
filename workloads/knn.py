"""Naive k-nearest-neighbour search as bytecodes (the kNN benchmark of the
paper's section "Performance Study": 10,000 elements and a query set of 1K,
O(n^2) work; the dimension and k are not given there, see the design notes).

Points ``X`` (N x D) and queries ``Q`` (M x D). Squared distances by
broadcast views over an (M, N, D) iteration space,

    diff = Q[:, None, :] - X[None, :, :];  diff = diff * diff
    d = ADD_REDUCE(diff, axis=2)                                  (M x N)

then k rounds, each taking the nearest remaining point of every query and
masking it out through an index comparison with ``iota`` (0..N-1):

    dist[:, r] = MIN_REDUCE(d, axis=1);  idx[:, r] = ARGMIN_REDUCE(d, axis=1)
    mask = EQUAL(iota[None, :], idx[:, r][:, None]);  d = SELECT(mask, +inf, d)

Ties go to the lower point index (first occurrence).
"""
from __future__ import annotations

import numpy as np

from .program import Const, ProgramBuilder, View

SEED = 1210_7774


def knn_inputs(n_points: int, n_queries: int, dim: int, dtype: str = "float64", seed: int = SEED + 7) -> dict:
    """Points and queries uniform in the unit cube, drawn in float64 and cast."""
    rng = np.random.default_rng(seed)
    X = rng.random((n_points, dim))
    Q = rng.random((n_queries, dim))
    return {"X": X.astype(dtype), "Q": Q.astype(dtype)}


def knn(n_points: int = 10_000, n_queries: int = 1_000, dim: int = 16, k: int = 4, dtype: str = "float64",
        seed: int = SEED + 7, inputs: dict | None = None):
    """The kNN program. Outputs: ``dist`` (M x k squared distances, ascending)
    and ``idx`` (M x k point indices)."""
    N, M, D = n_points, n_queries, dim
    b = ProgramBuilder(f"knn{N}x{M}x{D}k{k}_{dtype}")
    inp = inputs if inputs is not None else knn_inputs(N, M, D, dtype, seed)
    X = b.base(dtype, (N, D), inp["X"])
    Q = b.base(dtype, (M, D), inp["Q"])
    iota = b.base("int64", (N,), np.arange(N, dtype=np.int64))
    dist = b.base(dtype, (M, k), np.zeros(M * k, dtype))
    idx = b.base("int64", (M, k), np.zeros(M * k, np.int64))
    diff = b.base(dtype, (M, N, D))
    d = b.base(dtype, (M, N))
    mask = b.base("bool", (M, N))
    b.emit("SUBTRACT", b.whole(diff), View(Q, 0, (M, N, D), (D, 0, 1)), View(X, 0, (M, N, D), (0, D, 1)))
    b.emit("MULTIPLY", b.whole(diff), b.whole(diff), b.whole(diff))
    b.emit("ADD_REDUCE", b.whole(d), b.whole(diff), axis=2)
    b.discard(diff)
    for r in range(k):
        b.emit("MIN_REDUCE", View(dist, r, (M,), (k,)), b.whole(d), axis=1)
        b.emit("ARGMIN_REDUCE", View(idx, r, (M,), (k,)), b.whole(d), axis=1)
        if r + 1 < k:
            b.emit("EQUAL", b.whole(mask), View(iota, 0, (M, N), (0, 1)), View(idx, r, (M, N), (k, 0)))
            b.emit("SELECT", b.whole(d), b.whole(mask), Const(float("inf")), b.whole(d))
    b.discard(d, mask)
    b.sync(dist, idx)
    p = b.build([dist, idx])
    p.meta.update(N=N, M=M, D=D, k=k, dtype=dtype, X=X, Q=Q, dist=dist, idx=idx)
    return p
