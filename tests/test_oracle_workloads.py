"""Pins for the oracle on whole workloads: closed forms, invariants and
pure-Python loops on tiny inputs, each written from the mathematics of the
workload rather than from the oracle's code."""
import math

import numpy as np
import pytest

import oracle
from workloads import (Const, ProgramBuilder, blackscholes, bs_inputs, gray_scott, jacobi, jacobi_inputs,
                       montecarlo_pi, shallow_water, stencil_inputs, sw_inputs)
from workloads.blackscholes import AS_B, AS_P, _cnd

# ---------------------------------------------------------------- Jacobi


def _jacobi_brute(g, iters):
    g = [list(r) for r in g]
    n = len(g)
    deltas = []
    for _ in range(iters):
        new = [list(r) for r in g]
        total = []
        for i in range(1, n - 1):
            for j in range(1, n - 1):
                t = ((g[i - 1][j] + g[i + 1][j]) + g[i][j - 1]) + g[i][j + 1]
                t = t * 0.25
                new[i][j] = t
                total.append(abs(g[i][j] - t))
        deltas.append(math.fsum(total))
        g = new
    return np.array(g), deltas


def test_jacobi_matches_loops_bitwise():
    n, iters = 8, 4
    p = jacobi(n, iters, seed=11, history=True)
    mem = oracle.run(p)
    grid0 = jacobi_inputs(n, seed=11)
    want, deltas = _jacobi_brute(grid0.tolist(), iters)
    assert np.array_equal(mem[p.meta["grid"]].reshape(n, n), want)
    got_d = mem[p.meta["deltas"]]
    for a, b in zip(got_d.tolist(), deltas):
        assert abs(a - b) <= 1e-14 * max(1.0, abs(b))


def test_jacobi_linear_data_is_a_fixed_point():
    # a + b i + c j is discrete-harmonic; small integers keep it exact
    n = 12
    p = jacobi(n, 3, init="linear", linear=(5, 3, 7), history=True)
    mem = oracle.run(p)
    assert np.array_equal(mem[p.meta["grid"]], jacobi_inputs(n, init="linear", linear=(5, 3, 7)).ravel())
    assert mem[p.meta["deltas"]].tolist() == [0.0, 0.0, 0.0]


def test_jacobi_converges_to_boundary_and_keeps_maximum_principle():
    n = 10
    p = jacobi(n, 400, seed=3, history=True)
    mem = oracle.run(p)
    g = mem[p.meta["grid"]]
    g0 = jacobi_inputs(n, seed=3)
    assert g.min() >= g0.min() and g.max() <= 1.0
    assert np.max(np.abs(g - 1.0)) < 1e-6
    d = mem[p.meta["deltas"]]
    assert np.all(np.diff(d[5:]) <= 1e-15)  # contraction: deltas shrink


# ---------------------------------------------------------------- Black-Scholes


def _phi(x):
    return 0.5 * math.erfc(-x / math.sqrt(2.0))


def test_as_coefficients_match_golden():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "abramowitz_stegun_26_2_17.txt")
    vals = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    assert vals["p"] == AS_P
    assert tuple(vals[f"b{i}"] for i in range(1, 6)) == AS_B


def test_cnd_within_abramowitz_stegun_bound():
    d = np.linspace(-7.0, 7.0, 2001)
    d = np.concatenate([d, [0.0, -0.0, 1e-300, -1e-300]])
    b = ProgramBuilder("cnd")
    dv = b.whole(b.base("float64", d.size, d))
    out = b.base("float64", d.size)
    tmp = [b.whole(b.base("float64", d.size)) for _ in range(6)] + [b.whole(b.base("bool", d.size))]
    _cnd(b, "float64", d.size, dv, b.whole(out), tmp)
    got = oracle.run(b.build([out]))[out]
    for x, y in zip(d.tolist(), got.tolist()):
        assert abs(y - _phi(x)) < 7.5e-8
    # symmetry N(d) + N(-d) = 1 up to a few roundings, away from d = 0 (where
    # the polynomial's own error makes N(0) + N(0) = 1 + O(1e-9))
    half = got[:2001]
    sym = np.abs(half + half[::-1] - 1.0)
    sym[1000] = 0.0
    assert d[1000] == 0.0 and np.max(sym) <= 1e-15


@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_blackscholes_against_closed_form(dtype):
    n = 2000
    p = blackscholes(n, dtype, seed=5)
    mem = oracle.run(p)
    call, put = mem[p.meta["call"]].astype(np.float64), mem[p.meta["put"]].astype(np.float64)
    inp = bs_inputs(n, "float64", seed=5)
    bound_rel = 7.5e-8 if dtype == "float64" else 2e-5
    for i in range(n):
        S, K, T, r, v = (float(inp[k][i]) for k in "SKTRV")
        if dtype == "float32":
            S, K, T, r, v = (float(np.float32(x)) for x in (S, K, T, r, v))
        d1 = (math.log(S / K) + (r + v * v / 2) * T) / (v * math.sqrt(T))
        d2 = d1 - v * math.sqrt(T)
        kd = K * math.exp(-r * T)
        c = S * _phi(d1) - kd * _phi(d2)
        pu = kd * _phi(-d2) - S * _phi(-d1)
        tol = bound_rel * (S + kd) + 1e-12 * max(S, K)
        assert abs(call[i] - c) <= tol and abs(put[i] - pu) <= tol, i
        # put-call parity holds by construction up to a few roundings
        assert abs((call[i] - put[i]) - (S - kd)) <= (1e-12 if dtype == "float64" else 3e-5) * max(S, K)


# ---------------------------------------------------------------- shallow water


def _sw_brute(H, U, V, steps, g=9.8, dt=0.1, dx=1.0):
    """Two-step Lax-Wendroff written per cell from the conservation law
    q_t + F(q)_x + G(q)_y = 0, q = (h, hu, hv)."""
    N = len(H)
    n = N - 2
    H = [list(r) for r in H]
    U = [list(r) for r in U]
    V = [list(r) for r in V]

    def F(h, u, v):  # flux along axis 0
        return (u, u * u / h + 0.5 * g * h * h, u * v / h)

    def Gf(h, u, v):  # flux along axis 1
        return (v, u * v / h, v * v / h + 0.5 * g * h * h)

    for _ in range(steps):
        for i in range(N):
            H[i][0], U[i][0], V[i][0] = H[i][1], U[i][1], -V[i][1]
            H[i][N - 1], U[i][N - 1], V[i][N - 1] = H[i][N - 2], U[i][N - 2], -V[i][N - 2]
        for j in range(N):
            H[0][j], U[0][j], V[0][j] = H[1][j], -U[1][j], V[1][j]
            H[N - 1][j], U[N - 1][j], V[N - 1][j] = H[N - 2][j], -U[N - 2][j], V[N - 2][j]
        # half step values on faces (i+1/2, j) and (i, j+1/2)
        fx = {}
        for i in range(0, n + 1):
            for j in range(1, n + 1):
                qa = (H[i][j], U[i][j], V[i][j])
                qb = (H[i + 1][j], U[i + 1][j], V[i + 1][j])
                Fa, Fb = F(*qa), F(*qb)
                qh = [(qa[k] + qb[k]) / 2 - dt / (2 * dx) * (Fb[k] - Fa[k]) for k in range(3)]
                fx[i, j] = F(*qh)
        fy = {}
        for i in range(1, n + 1):
            for j in range(0, n + 1):
                qa = (H[i][j], U[i][j], V[i][j])
                qb = (H[i][j + 1], U[i][j + 1], V[i][j + 1])
                Ga, Gb = Gf(*qa), Gf(*qb)
                qh = [(qa[k] + qb[k]) / 2 - dt / (2 * dx) * (Gb[k] - Ga[k]) for k in range(3)]
                fy[i, j] = Gf(*qh)
        for i in range(1, n + 1):
            for j in range(1, n + 1):
                for k, Q in enumerate((H, U, V)):
                    Q[i][j] = (Q[i][j] - dt / dx * (fx[i, j][k] - fx[i - 1, j][k])
                               - dt / dx * (fy[i, j][k] - fy[i, j - 1][k]))
    return np.array(H), np.array(U), np.array(V)


def test_shallow_water_matches_cell_loops():
    N, steps = 14, 4
    inp = sw_inputs(N, seed=9)
    inp["U"] = np.random.default_rng(1).uniform(-0.05, 0.05, (N, N))
    inp["V"] = np.random.default_rng(2).uniform(-0.05, 0.05, (N, N))
    p = shallow_water(N, steps, inputs=inp)
    mem = oracle.run(p)
    bh, bu, bv = _sw_brute(inp["H"], inp["U"], inp["V"], steps)
    sl = (slice(1, N - 1), slice(1, N - 1))
    for got, want in ((mem[p.meta["H"]], bh), (mem[p.meta["U"]], bu), (mem[p.meta["V"]], bv)):
        got = got.reshape(N, N)
        assert np.max(np.abs(got[sl] - want[sl])) <= 1e-12


def test_shallow_water_lake_at_rest_is_bitwise_steady():
    N = 16
    inp = sw_inputs(N, kind="rest")
    inp["H"] = inp["H"] * 1.25
    p = shallow_water(N, 5, inputs=inp)
    mem = oracle.run(p)
    sl = (slice(1, N - 1), slice(1, N - 1))
    assert np.all(mem[p.meta["H"]].reshape(N, N)[sl] == 1.25)
    assert np.all(mem[p.meta["U"]].reshape(N, N)[sl] == 0.0)
    assert np.all(mem[p.meta["V"]].reshape(N, N)[sl] == 0.0)


def test_shallow_water_conserves_mass_and_mirror_symmetry():
    N = 24
    inp = sw_inputs(N, centred=True)
    p = shallow_water(N, 30, inputs=inp)
    mem = oracle.run(p)
    sl = (slice(1, N - 1), slice(1, N - 1))
    H = mem[p.meta["H"]].reshape(N, N)
    U = mem[p.meta["U"]].reshape(N, N)
    V = mem[p.meta["V"]].reshape(N, N)
    m0 = math.fsum(inp["H"][sl].ravel().tolist())
    m1 = math.fsum(H[sl].ravel().tolist())
    assert abs(m1 - m0) <= 1e-12 * m0
    assert np.max(np.abs(H[sl] - H[sl][::-1, :])) <= 1e-13
    assert np.max(np.abs(U[sl] + U[sl][::-1, :])) <= 1e-13
    assert np.max(np.abs(H[sl] - H[sl][:, ::-1])) <= 1e-13
    assert np.max(np.abs(V[sl] + V[sl][:, ::-1])) <= 1e-13
    assert np.max(np.abs(U)) > 1e-3  # the droplet has moved


def _sw_1d(h, m, steps, g=9.8, dt=0.1, dx=1.0):
    """Two-step Lax-Wendroff for the 1-D shallow-water equations
    h_t + (hu)_x = 0, (hu)_t + (hu^2/h + g h^2 / 2)_x = 0, state (h, m = hu),
    reflective ends (h copied, m negated in the ghost cells)."""
    h, m = list(h), list(m)
    N = len(h)

    def flux(hh, mm):
        return (mm, mm * mm / hh + 0.5 * g * hh * hh)

    for _ in range(steps):
        h[0], m[0] = h[1], -m[1]
        h[N - 1], m[N - 1] = h[N - 2], -m[N - 2]
        half = []
        for i in range(N - 1):
            fa, fb = flux(h[i], m[i]), flux(h[i + 1], m[i + 1])
            hh = (h[i] + h[i + 1]) / 2 - dt / (2 * dx) * (fb[0] - fa[0])
            mm = (m[i] + m[i + 1]) / 2 - dt / (2 * dx) * (fb[1] - fa[1])
            half.append(flux(hh, mm))
        for i in range(1, N - 1):
            h[i] -= dt / dx * (half[i][0] - half[i - 1][0])
            m[i] -= dt / dx * (half[i][1] - half[i - 1][1])
    return np.array(h), np.array(m)


def test_shallow_water_y_uniform_state_follows_the_1d_scheme():
    """A state uniform along axis 1 with V = 0 stays uniform along axis 1
    with V = 0 (its y fluxes cancel exactly), and its interior follows the
    1-D scheme along axis 0."""
    N, steps = 20, 12
    x = np.arange(N, dtype=np.float64)
    h1 = 1.0 + 0.4 * np.exp(-((x - 8.3) ** 2) / 8.0)
    m1 = 0.05 * np.sin(x / 3.0)
    inp = {"H": np.repeat(h1[:, None], N, axis=1), "U": np.repeat(m1[:, None], N, axis=1), "V": np.zeros((N, N))}
    p = shallow_water(N, steps, inputs=inp)
    mem = oracle.run(p)
    H = mem[p.meta["H"]].reshape(N, N)[:, 1:N - 1]
    U = mem[p.meta["U"]].reshape(N, N)[:, 1:N - 1]
    V = mem[p.meta["V"]].reshape(N, N)[1:N - 1, 1:N - 1]
    assert np.all(V == 0.0)
    assert np.all(H[1:N - 1] == H[1:N - 1, :1]) and np.all(U[1:N - 1] == U[1:N - 1, :1])
    bh, bm = _sw_1d(h1, m1, steps)
    assert np.max(np.abs(H[1:N - 1, 0] - bh[1:N - 1])) <= 1e-13
    assert np.max(np.abs(U[1:N - 1, 0] - bm[1:N - 1])) <= 1e-13
    assert np.max(np.abs(U[1:N - 1, 0] - m1[1:N - 1])) > 1e-3  # the state has evolved


# ---------------------------------------------------------------- Monte-Carlo pi


def _mc_brute(seed, sizes):
    M = (1 << 64) - 1
    counts = []
    for i, n in enumerate(sizes):
        hits = 0
        for m in range(n):
            u = []
            for j in (0, 1):
                c = ((i << 32) | j) + 2 * m
                z = (seed + (c + 1) * 0x9E3779B97F4A7C15) & M
                z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
                z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
                z ^= z >> 31
                u.append((z >> 11) * 2.0**-53)
            x, y = u
            if x * x + y * y <= 1.0:
                hits += 1
        counts.append(hits)
    return counts


def test_montecarlo_counts_exact():
    sizes = [1, 1000, 4096, 37]
    p = montecarlo_pi(seed=77, sizes=sizes)
    mem = oracle.run(p)
    assert mem[p.meta["count"]].tolist() == _mc_brute(77, sizes)


def test_montecarlo_estimate_is_statistically_sound():
    n = 1 << 20
    p = montecarlo_pi(seed=5, sizes=[n, n])
    mem = oracle.run(p)
    q = math.pi / 4
    sigma = math.sqrt(q * (1 - q) / n)
    for c in mem[p.meta["count"]].tolist():
        assert abs(c / n - q) < 5 * sigma


# ------------------------------------------------------ synthetic stencil

def _gray_scott_loops(U, V, steps, Du, Dv, f, k):
    """Explicit Euler steps of the Gray-Scott equations, one cell at a time
    in plain Python floats (the ring stays fixed), with the five-point
    Laplacian summed up, down, left, right, then minus 4 times the centre."""
    U = [list(map(float, r)) for r in U]
    V = [list(map(float, r)) for r in V]
    R, C = len(U), len(U[0])
    for _ in range(steps):
        nU = [r[:] for r in U]
        nV = [r[:] for r in V]
        for i in range(1, R - 1):
            for j in range(1, C - 1):
                u, v = U[i][j], V[i][j]
                lu = U[i - 1][j] + U[i + 1][j] + U[i][j - 1] + U[i][j + 1] - u * 4.0
                lv = V[i - 1][j] + V[i + 1][j] + V[i][j - 1] + V[i][j + 1] - v * 4.0
                uvv = u * v * v
                nU[i][j] = lu * Du - uvv + (1.0 - u) * f + u
                nV[i][j] = lv * Dv + uvv - v * (f + k) + v
        U, V = nU, nV
    return np.array(U), np.array(V)


def test_stencil_matches_cell_loops_bitwise():
    inp = stencil_inputs(11, 13, patches=3, seed=4)
    p = gray_scott(11, 13, 3, inputs=inp)
    mem = oracle.run(p)
    U, V = _gray_scott_loops(inp["U"], inp["V"], 3, p.meta["Du"], p.meta["Dv"], p.meta["F"], p.meta["k"])
    assert np.array_equal(mem[p.meta["U"]].reshape(11, 13), U)
    assert np.array_equal(mem[p.meta["V"]].reshape(11, 13), V)


@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_stencil_rest_state_is_bitwise_steady(dtype):
    """U = 1, V = 0 is a fixed point: every Laplacian is exactly 0 and the
    reaction terms vanish."""
    inp = stencil_inputs(12, 14, dtype, kind="rest")
    p = gray_scott(12, 14, 4, dtype, inputs=inp)
    mem = oracle.run(p)
    assert np.array_equal(mem[p.meta["U"]], inp["U"].ravel())
    assert np.array_equal(mem[p.meta["V"]], inp["V"].ravel())


def test_stencil_keeps_row_mirror_symmetry_bitwise():
    """A state symmetric under i -> R-1-i stays so bitwise (up and down
    enter the Laplacian through one commutative addition)."""
    R, C = 14, 10
    rng = np.random.default_rng(3)
    half = rng.random((R // 2, C))
    V = np.concatenate([half, half[::-1]]) * 0.25
    U = 1.0 - V
    p = gray_scott(R, C, 5, inputs={"U": U, "V": V})
    mem = oracle.run(p)
    for q in ("U", "V"):
        a = mem[p.meta[q]].reshape(R, C)
        assert np.array_equal(a, a[::-1])


# ------------------------------------------------------------------- kNN

@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_knn_matches_sorted_brute_force(dtype):
    """The k nearest points of every query equal the first k entries of a
    stable sort of all squared distances, computed here per pair in plain
    float64 (for these draws no two candidates are close enough for float32
    rounding to swap them); an exact duplicate point checks the lower-index
    tie rule."""
    from workloads import knn, knn_inputs
    inp = knn_inputs(200, 30, 4, dtype, seed=8)
    inp["X"][150] = inp["X"][20]          # an exact duplicate: ties go to index 20
    inp["Q"][3] = inp["X"][20]
    p = knn(200, 30, 4, 5, dtype, inputs=inp)
    mem = oracle.run(p)
    X, Q = inp["X"].astype(np.float64), inp["Q"].astype(np.float64)
    d2 = [[sum((Q[m, j] - X[n, j]) ** 2 for j in range(4)) for n in range(200)] for m in range(30)]
    want = [sorted(range(200), key=lambda n: (d2[m][n], n))[:5] for m in range(30)]
    got = mem[p.meta["idx"]].reshape(30, 5).tolist()
    assert got == want
    assert got[3][:2] == [20, 150]
    dist = mem[p.meta["dist"]].reshape(30, 5)
    assert np.all(np.diff(dist, axis=1) >= 0)
