"""Pins of the oracle's lower-dimensional fracture continuum (Section 2,
Eqs. mm-md / mm-tc; Section 3.1, Eqs. app-md / app-tc): mesh geometry and
junction transmissibilities by hand, the fracture's cosine modes, sigma = 0
decoupling, mass identities, constant states, and the coupled matrix built
equation by equation."""

import numpy as np
import pytest

import mc_inputs as mi
from oracle import metrics
from oracle.fv import FVSystem
from oracle.schemes import Oracle
from oracle.fracture1d import FractureMesh, MixedOracle, MixedSystem, from_workload


def test_horizontal_segment_pieces():
    """A segment across the square at mid-height of row 2 of a 5 x 5 grid: five
    pieces of length h, hosted by the cells of row 2, consecutive pieces
    joined with T = k_f / h (two-point value, d = h/2 + h/2)."""
    n, kf = 5, 3.0
    y = 2.5 / n
    m = FractureMesh([[-0.1, y, 1.2, y]], n, n)
    assert m.P == n
    np.testing.assert_allclose(m.length, 1.0 / n, rtol=1e-13)
    np.testing.assert_array_equal(m.host, 2 * n + np.arange(n))
    T = m.transmissibility(kf).toarray()
    want = np.zeros((n, n))
    for l in range(n - 1):
        want[l, l + 1] = want[l + 1, l] = kf * n
    np.testing.assert_allclose(T, want, rtol=1e-13)


def test_cross_junction_star_delta():
    """Two segments crossing at the centre of a cell: four half-pieces of
    length l meet at one point; each has t = k_f / (l/2), and each of the six
    pairs gets T = t t / (4 t) = k_f / (2 l)."""
    n, kf = 4, 2.0
    c = 1.5 / n   # centre of cell (1, 1)
    hw = 0.25 / n
    m = FractureMesh([[c - hw, c, c + hw, c], [c, c - hw, c, c + hw]], n, n)
    assert m.P == 4
    np.testing.assert_allclose(m.length, hw, rtol=1e-12)
    assert len(m.junctions) == 1 and len(m.junctions[0]) == 4
    T = m.transmissibility(kf).toarray()
    off = T[~np.eye(4, dtype=bool)]
    np.testing.assert_allclose(off, kf / (2 * hw), rtol=1e-12)
    np.testing.assert_array_equal(m.host, np.full(4, 1 * n + 1))


def test_total_length_and_hosts_of_random_network():
    w = mi.fracture1d(1, n=40)
    m = FractureMesh(w.frac.segments, 40, 40)
    total = 0.0
    from oracle.fracture1d import clip_segment
    for s in w.frac.segments:
        c = clip_segment(*s)
        if c is not None:
            total += (c[1] - c[0]) * np.hypot(s[2] - s[0], s[3] - s[1])
    np.testing.assert_allclose(m.length.sum(), total, rtol=1e-12)
    # every piece lies in its host cell (midpoint inside, length <= diagonal)
    h = 1.0 / 40
    i, j = m.host % 40, m.host // 40
    assert np.all((m.mid[:, 0] >= i * h - 1e-12) & (m.mid[:, 0] <= (i + 1) * h + 1e-12))
    assert np.all((m.mid[:, 1] >= j * h - 1e-12) & (m.mid[:, 1] <= (j + 1) * h + 1e-12))
    assert np.all(m.length <= np.sqrt(2) * h + 1e-12)
    # crossings exist in this network: some junction joins more than two pieces
    assert max(len(g) for g in m.junctions) >= 3


def _straight_fracture_system(n, kf, cf, sigma, k_m=1.0):
    y = 2.5 / n
    fv = FVSystem(n, n, 1, [np.full((n, n), k_m)], [0.5])
    mesh = FractureMesh([[0.0, y, 1.0, y]], n, n)
    return MixedSystem(fv, mesh, kf, cf, [sigma])


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_fracture_cosine_mode_decay(mode):
    """sigma_f = 0, a straight fracture of n pieces of length h: the fracture
    block is the 1-D two-point Laplacian with zero-flux ends, so
    cos(pi m (l + 1/2) / n) is an eigenvector with lambda = 2 (k_f/h)
    (1 - cos(pi m / n)), and one backward-Euler step multiplies it by
    1 / (1 + tau lambda / (c_f h))."""
    n, kf, cf, tau = 8, 0.7, 2.0, 0.01
    ms = _straight_fracture_system(n, kf, cf, 0.0)
    o = MixedOracle(ms, tau)
    h = 1.0 / n
    v = np.cos(np.pi * mode * (np.arange(n) + 0.5) / n)
    lam = 2 * (kf / h) * (1 - np.cos(np.pi * mode / n))
    g = 1.0 / (1.0 + tau * lam / (cf * h))
    for scheme in ("coupled", "D", "L", "U"):
        p1 = o.step([np.zeros(n * n), v], [np.zeros(n * n)], scheme)
        np.testing.assert_allclose(p1[1], g * v, rtol=1e-12, atol=1e-14)
        assert np.abs(p1[0]).max() == 0.0


@pytest.mark.parametrize("scheme", ["coupled", "D", "L", "U"])
def test_sigma_zero_decouples(scheme):
    """sigma_f = 0: the matrix continua follow the plain finite-volume scheme
    of the co-located model (independent oracle), the fracture its own 1-D
    evolution."""
    w = mi.fracture1d(2, n=16, wells=False, p0=0.0)
    w.F[1][3, 4] = 1.0
    w.F[0][12, 10] = -0.5
    w.frac.sigma_f = np.zeros(2)
    o, p0 = from_workload(w)
    o.ms.Ff[:] = 0.0
    o.ms.Ff[3] = 2.0
    p0[2] = np.linspace(0.0, 1.0, o.ms.P)
    pm = o.run(p0, w.F, 3, scheme)
    fv = FVSystem(w.nx, w.ny, w.L, w.k, w.c, w.sigma)
    ref = Oracle(fv, w.tau).run(p0[:2], w.F, 3, scheme)
    for a in range(2):
        np.testing.assert_allclose(pm[a], ref[a], rtol=1e-12, atol=1e-14)
    # the fracture alone: (M/tau + D_f) p^n = M/tau p^{n-1} + F_f
    # (dense solve with two refinement sweeps whose residual is formed in
    # extended precision: the fracture block is stiff, kappa ~ 1e5)
    ms = o.ms
    Af = (np.diag(ms.mf / w.tau) + ms.block(2, 2).toarray())
    Ae = np.diag((ms.mf / w.tau).astype(np.longdouble)) + ms.block(2, 2, np.longdouble).toarray()
    pf = p0[2].copy()
    for _ in range(3):
        b = ms.mf / w.tau * pf + ms.Ff
        x = np.linalg.solve(Af, b)
        for _ in range(2):
            r = b.astype(np.longdouble) - Ae @ x.astype(np.longdouble)
            x = x + np.linalg.solve(Af, np.asarray(r, dtype=np.float64))
        pf = x
    np.testing.assert_allclose(pm[2], pf, rtol=1e-12, atol=1e-14)


def test_constant_state_is_steady():
    """No sources, no wells, p = 1 in every continuum and piece: every
    scheme keeps it (A 1 = 0: every flux and exchange term is a difference)."""
    w = mi.fracture1d(2, n=20, wells=False, p0=1.0)
    o, p0 = from_workload(w)
    for scheme in ("coupled", "D", "L", "U"):
        p = o.run(p0, w.F, 2, scheme)
        for x in p:
            np.testing.assert_allclose(x, 1.0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("scheme", ["coupled", "D"])
def test_mass_identity(scheme):
    """Coupled: sum M dp = tau sum (F + W (p_w - p^n)) (1^T A = 0).
    D-scheme (Section 3.3, the exchange lagged): the same plus
    tau sum over pairs of the exchange q (dp_a + dp_b); for the
    fracture-matrix pair the sum runs over pieces with the host cell's
    matrix value."""
    w = mi.fracture1d(2, n=24)
    o, p0 = from_workload(w)
    ms = o.ms
    p1 = o.step(p0, w.F, scheme)
    dp = [x - y for x, y in zip(p1, p0)]
    lhs = sum(float(np.dot(ms.mass(a), dp[a])) for a in range(3))
    rhs = 0.0
    for a in range(3):
        W, wp = ms.well(a)
        rhs += float(np.sum(ms.source(a, w.F) + wp - W * p1[a]))
    rhs *= w.tau
    if scheme == "D":
        ex = float(np.dot(ms.fv.q[(0, 1)], dp[0] + dp[1]))
        for a in range(2):
            ex += float(np.dot(ms.q[a], dp[a][ms.mesh.host] + dp[2]))
        lhs += w.tau * ex
    scale = sum(float(np.dot(ms.mass(a), np.abs(p1[a]))) for a in range(3))
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs)


def test_coupled_matrix_equation_by_equation():
    """Eq. app-tc written out cell by cell and piece by piece into a dense
    matrix on a 6 x 6 grid with three segments must equal the oracle's
    assembled coupled step matrix."""
    n = 6
    rng = np.random.default_rng(11)
    segs = np.array([[0.05, 0.1, 0.9, 0.8], [0.1, 0.85, 0.95, 0.2], [0.5, 0.02, 0.52, 0.97]])
    k = [np.exp(rng.standard_normal((n, n))), 3.0 * np.exp(rng.standard_normal((n, n)))]
    c = [0.3, 0.7]
    s12 = 2.0
    kf, cf, sf = 50.0, 0.4, [1.5, 0.5]
    tau = 0.05
    fv = FVSystem(n, n, 2, k, c, np.array([[0, s12], [s12, 0]]))
    mesh = FractureMesh(segs, n, n)
    ms = MixedSystem(fv, mesh, kf, cf, sf)
    o = MixedOracle(ms, tau)
    A = o._matrix("coupled", np.float64).toarray()
    h = 1.0 / n
    N, P = n * n, mesh.P
    B = np.zeros((2 * N + P, 2 * N + P))

    def harm(a, b):
        return 2 * a * b / (a + b)

    for a in range(2):
        for j in range(n):
            for i in range(n):
                r = a * N + j * n + i
                B[r, r] += c[a] * h * h / tau
                for (ii, jj) in ((i + 1, j), (i - 1, j), (i, j + 1), (i, j - 1)):
                    if 0 <= ii < n and 0 <= jj < n:
                        T = harm(k[a][j, i], k[a][jj, ii])
                        B[r, r] += T
                        B[r, a * N + jj * n + ii] -= T
                q12 = s12 * h * h
                B[r, r] += q12
                B[r, (1 - a) * N + j * n + i] -= q12
    T = mesh.transmissibility(kf).toarray()
    for l in range(P):
        r = 2 * N + l
        B[r, r] += cf * mesh.length[l] / tau
        for m_ in range(P):
            if m_ != l and T[l, m_] != 0.0:
                B[r, r] += T[l, m_]
                B[r, 2 * N + m_] -= T[l, m_]
        for a in range(2):
            q = sf[a] * mesh.length[l] / (h / 4)
            ci = a * N + mesh.host[l]
            B[r, r] += q
            B[r, ci] -= q
            B[ci, ci] += q
            B[ci, r] -= q
    np.testing.assert_allclose(A, B, rtol=1e-13, atol=1e-12 * np.abs(B).max())


def test_splitting_error_first_order_in_tau():
    """D-scheme minus coupled at a fixed final time shrinks about 2x per
    halving of tau (splitting error O(tau), Section 3.3)."""
    w = mi.fracture1d(1, n=12, wells=True)
    errs = []
    for m in (32, 64, 128):
        w.tau = 0.002 / m
        o, p0 = from_workload(w)
        pc = o.run(p0, w.F, m, "coupled")
        pd = o.run(p0, w.F, m, "D")
        errs.append(metrics.rel_l2([x - 1.0 for x in pc], [x - 1.0 for x in pd]))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.6 < r1 < 2.6 and 1.6 < r2 < 2.6, errs
