"""Scenarios of the data-ownership scheme run two ways: by the oracle's
model (``oracle.OwnershipModel``) and through the library's C ABI
(vbe_mirror_* and vbe_submit), on a recording context whose launches the
emulator executes on the CPU, or on a GPU. Each returns the same list of
observations: after every step the ownership state of each mirrored base,
after every read access the host copy's contents, and the first error.

The program: mirrored float64 bases x and y (37 x 53), a base z without a
host copy, and batches built from the fragments below. Values are small
integers and every operation is + - * by small integers or a copy, so all
results are exact and the observations must match bit for bit."""
from __future__ import annotations

import numpy as np

import oracle
from workloads import Const, ProgramBuilder
from workloads.program import Instr

SHAPE = (37, 53)


def program():
    b = ProgramBuilder("ownership")
    x = b.base("float64", SHAPE)
    y = b.base("float64", SHAPE)
    z = b.base("float64", SHAPE, np.arange(SHAPE[0] * SHAPE[1]) % 11 - 5.0)
    X, Y, Z = b.whole(x), b.whole(y), b.whole(z)
    rows = b.view(x, 0, (5, SHAPE[1]), (SHAPE[1], 1))
    frag = {
        "y=3x+1": [("MULTIPLY", Y, X, Const(3.0)), ("ADD", Y, Y, Const(1.0))],
        "x=x+y": [("ADD", X, X, Y)],
        "x=x-2": [("SUBTRACT", X, X, Const(2.0))],
        "z=x-y": [("SUBTRACT", Z, X, Y)],
        "y=z*2": [("MULTIPLY", Y, Z, Const(2.0))],
        "x=7": [("COPY", X, Const(7.0))],
        "x[:5]=9": [("COPY", rows, Const(9.0))],
        "SYNC x": [("SYNC", X)], "SYNC y": [("SYNC", Y)],
        "DISCARD x": [("DISCARD", X)], "DISCARD y": [("DISCARD", Y)],
    }
    p = b.build([x, y, z])
    return p, x, y, z, frag


def fragments_to_instrs(frag, names):
    return [Instr(op, o, tuple(ins)) for nm in names for op, o, *ins in frag[nm]]


def small_ints(rng):
    return rng.integers(-20, 21, SHAPE).astype(np.float64)


def scenario(seed, steps=24):
    """A seeded sequence of steps that follows the rules: the host writes
    only with write access (after release) or right before a discard. A
    candidate step that the model rejects (a read of a base whose value no
    copy holds, or of a base discarded earlier in the same batch) is
    dropped, except that with probability 1/8 it ends the scenario, so the
    error paths are covered too."""
    import copy
    rng = np.random.default_rng(seed)
    p, x, y, z, frag = program()
    bases = {"x": x, "y": y}
    ops = [("attach", x, small_ints(rng)), ("attach", y, small_ints(rng))]
    names = [k for k in frag]
    model = oracle.OwnershipModel(p)
    for op in ops:
        _apply(model, frag, op)
    while len(ops) < steps + 2:
        r = rng.random()
        bid = bases["x" if rng.random() < 0.6 else "y"]
        if r < 0.45:
            k = int(rng.integers(1, 4))
            cand = [("submit", [names[i] for i in rng.choice(len(names), k)])]
        elif r < 0.65:
            cand = [("sync", bid)]
        elif r < 0.82:
            cand = [("release", bid), ("store", bid, small_ints(rng))]
        else:
            cand = [("sync", bid), ("store_then_discard", bid, small_ints(rng))]
        trial = copy.deepcopy(model)
        try:
            for op in cand:
                _apply(trial, frag, op)
        except oracle.OracleError:
            if rng.random() < 0.125:
                return ops + cand
            continue
        model = trial
        ops += cand
    return ops


def _apply(m, frag, op):
    kind = op[0]
    if kind == "attach":
        m.attach(op[1], op[2])
    elif kind == "submit":
        m.submit(fragments_to_instrs(frag, op[1]))
    elif kind == "sync":
        return m.sync(op[1])
    elif kind == "release":
        m.release(op[1])
    elif kind == "store":
        m.store(op[1], op[2])
    elif kind == "store_then_discard":
        m.store(op[1], op[2], declared_by_discard=True)
        m.discard(op[1])
    return None


def run_model(ops):
    p, x, y, z, frag = program()
    m = oracle.OwnershipModel(p)
    obs = []
    for step, op in enumerate(ops):
        try:
            got = _apply(m, frag, op)
            if op[0] == "sync":
                obs.append((step, "host", op[1], got.copy()))
        except oracle.OracleError:
            obs.append((step, "error"))
            return obs
        obs.append((step, "state", {b: m.state(b) for b in (x, y) if b in m.host}))
    return obs


def run_library(ops, flags, emulator=None, device=0, cache_dir=None):
    """The same steps through the C ABI; ``emulator`` executes each batch's
    recorded launches (and copies) on a recording context."""
    from paper_1210_7774_b300 import vbe as V
    from paper_1210_7774_b300.runner import Executor
    p, x, y, z, frag = program()
    obs = []
    host = {}
    with Executor(flags, device=device, cache_dir=cache_dir) as ex:
        L = ex.load(p)  # uploads z, the base without a host copy
        h = L.base
        batches = {}

        def flush():
            if emulator is not None:
                emulator.run(V.vbe_debug_take_launches(ex.ctx))

        for step, op in enumerate(ops):
            try:
                kind = op[0]
                if kind == "attach":
                    host[op[1]] = np.array(op[2], dtype=np.float64).reshape(-1).copy()
                    V.vbe_mirror_attach(ex.ctx, h[op[1]], host[op[1]].ctypes.data, host[op[1]].nbytes)
                elif kind == "submit":
                    key = tuple(op[1])
                    if key not in batches:
                        batches[key] = ex.encode(L, fragments_to_instrs(frag, op[1]))
                    arr, n = batches[key]
                    V.vbe_submit(ex.ctx, arr, n)
                    flush()
                elif kind == "sync":
                    V.vbe_mirror_sync(ex.ctx, h[op[1]])
                    obs.append((step, "host", op[1], host[op[1]].copy()))
                elif kind == "release":
                    V.vbe_mirror_release(ex.ctx, h[op[1]])
                elif kind == "store":
                    host[op[1]][...] = np.asarray(op[2]).reshape(-1)
                elif kind == "store_then_discard":
                    host[op[1]][...] = np.asarray(op[2]).reshape(-1)
                    V.vbe_mirror_discard(ex.ctx, h[op[1]])
            except V.VbeError:
                flush()
                obs.append((step, "error"))
                return obs
            obs.append((step, "state", {b: V.vbe_mirror_state(ex.ctx, h[b]) for b in (x, y) if b in host}))
    return obs


def same_observations(got, want):
    """The library's observations equal the model's; in a host copy, an
    element the model holds as NaN (a discarded value: every defined value
    here is a small integer) may hold anything."""
    if len(got) != len(want):
        return False
    for g, w in zip(got, want):
        if g[:2] != w[:2]:
            return False
        if w[1] == "host":
            gv, wv = g[3], w[3]
            if g[2] != w[2] or not np.array_equal(gv[~np.isnan(wv)], wv[~np.isnan(wv)]):
                return False
        elif g != w:
            return False
    return True
