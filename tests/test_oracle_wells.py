"""Pins of the oracle's implicit well term (Section 5's source
f = q_w (p_w - p) in the well cells, taken implicitly in p).

Each check is fixed by something other than the oracle's own formula: the
one-cell relaxation closed form, a 2 x 2 recurrence for uniform fields
written out by hand, the steady state of a zero-flux problem with a well, the
mass identities with the well flux, and a dense operator built equation by
equation on tiny grids.
"""

import numpy as np
import pytest

from oracle import metrics
from oracle.fv import FVSystem
from oracle.schemes import Oracle


def _k(rng, nx, ny, L):
    return [np.exp(1.2 * rng.standard_normal((ny, nx))) * 10.0 ** a for a in range(L)]


@pytest.mark.parametrize("scheme", ["coupled", "D", "L", "U"])
def test_uniform_well_relaxation_closed_form(scheme):
    """One continuum, heterogeneous k, a well of index q_w in every cell:
    a uniform state stays uniform (D 1 = 0) and p^n - p_w = g^n (p^0 - p_w)
    with g = (c/tau) / (c/tau + q_w) (per unit area)."""
    rng = np.random.default_rng(5)
    nx, ny, c, tau, qw, pw = 6, 5, 0.3, 0.01, 40.0, 1.2
    fv0 = FVSystem(nx, ny, 1, _k(rng, nx, ny, 1), [c])
    h2 = fv0.h ** 2
    fv = FVSystem(nx, ny, 1, fv0.k, [c], wells={0: (np.full(nx * ny, qw * h2), pw)})
    o = Oracle(fv, tau)
    p = [np.ones(nx * ny)]
    F = [np.zeros(nx * ny)]
    g = (c / tau) / (c / tau + qw)
    for n in range(1, 6):
        p = o.step(p, F, "coupled" if scheme == "coupled" else scheme)
        np.testing.assert_allclose(p[0], pw + g ** n * (1.0 - pw), rtol=0, atol=1e-13)


@pytest.mark.parametrize("scheme", ["coupled", "D"])
def test_two_continuum_uniform_recurrence_with_well(scheme):
    """Uniform fields, L = 2, exchange sigma, a well only in continuum 2.
    Per unit area the uniform state obeys
      coupled: [c1/t + s, -s; -s, c2/t + s + w] p^n = [c1/t p1; c2/t p2 + w pw]
      D:       [c1/t + s, 0; 0, c2/t + s + w] p^n = [c1/t p1 + s p2; c2/t p2 + s p1 + w pw]
    (right-hand sides at layer n-1), solved here by Cramer's rule."""
    rng = np.random.default_rng(8)
    nx, ny = 5, 4
    c1, c2, s, w, pw, t = 1.0, 0.1, 10.0, 300.0, 1.2, 0.02
    fv0 = FVSystem(nx, ny, 2, _k(rng, nx, ny, 2), [c1, c2])
    h2 = fv0.h ** 2
    fv = FVSystem(nx, ny, 2, fv0.k, [c1, c2], np.array([[0, s], [s, 0]]),
                  wells={1: (np.full(nx * ny, w * h2), np.full((ny, nx), pw))})
    o = Oracle(fv, t)
    p1, p2 = 1.0, 0.5
    p = [np.full(nx * ny, p1), np.full(nx * ny, p2)]
    F = [np.zeros(nx * ny)] * 2
    for _ in range(4):
        if scheme == "coupled":
            a11, a12, a21, a22 = c1 / t + s, -s, -s, c2 / t + s + w
            b1, b2 = c1 / t * p1, c2 / t * p2 + w * pw
        else:
            a11, a12, a21, a22 = c1 / t + s, 0.0, 0.0, c2 / t + s + w
            b1, b2 = c1 / t * p1 + s * p2, c2 / t * p2 + s * p1 + w * pw
        det = a11 * a22 - a12 * a21
        p1, p2 = (b1 * a22 - a12 * b2) / det, (a11 * b2 - b1 * a21) / det
        p = o.step(p, F, scheme)
        np.testing.assert_allclose(p[0], p1, rtol=1e-13)
        np.testing.assert_allclose(p[1], p2, rtol=1e-13)


def test_steady_state_is_the_well_pressure():
    """Zero-flux walls, no other source, a well in a small box: the only
    steady state is p = p_w in every cell of every connected continuum."""
    rng = np.random.default_rng(9)
    nx = ny = 12
    W = np.zeros((ny, nx))
    W[2:4, 2:4] = 1e3 / nx ** 2
    fv = FVSystem(nx, ny, 2, _k(rng, nx, ny, 2), [0.1, 1.0], np.array([[0, 5.0], [5.0, 0]]),
                  wells={1: (W, 1.2)})
    o = Oracle(fv, 1e4)
    p = [np.ones(nx * ny), np.ones(nx * ny)]
    F = [np.zeros(nx * ny)] * 2
    for scheme in ("coupled", "D"):
        q = p
        for _ in range(40):
            q = o.step(q, F, scheme)
        for a in range(2):
            np.testing.assert_allclose(q[a], 1.2, rtol=0, atol=1e-9)


def test_mass_identities_with_well_flux():
    """Summing each scheme's equations over all cells (1^T D = 0):
    coupled: sum m dp = tau (sum F + sum W (p_w - p^n));
    D:       sum m dp + tau sum_{a<b} q (dp_a + dp_b) = tau (sum F + sum W (p_w - p^n))."""
    rng = np.random.default_rng(12)
    nx, ny, L, tau = 9, 7, 3, 0.03
    sig = np.array([[0, 2.0, 1.0], [2.0, 0, 4.0], [1.0, 4.0, 0]])
    W = [np.zeros(nx * ny), np.where(rng.random(nx * ny) < 0.2, 5.0, 0.0), np.zeros(nx * ny)]
    W[2][[3, 40]] = 7.0
    pw = [np.zeros(nx * ny), np.full(nx * ny, 1.5), np.full(nx * ny, -0.5)]
    fv = FVSystem(nx, ny, L, _k(rng, nx, ny, L), [1.0, 0.2, 0.05], sig,
                  wells={a: (W[a], pw[a]) for a in range(L)})
    o = Oracle(fv, tau)
    p0 = [rng.standard_normal(nx * ny) for _ in range(L)]
    F = [rng.standard_normal(nx * ny) * 0.1 for _ in range(L)]
    for scheme in ("coupled", "D"):
        p1 = o.step(p0, F, scheme)
        well = sum(float(np.dot(W[a], pw[a] - p1[a])) for a in range(L))
        lhs = metrics.mass_change(fv, p1, p0)
        if scheme == "D":
            lhs += tau * metrics.exchange_change(fv, p1, p0)
        rhs = tau * (metrics.total_source(F) + well)
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs) + 1.0)


def _dense_step_matrix(fv, tau, W, scheme):
    """M/tau + A (+ W) written equation by equation (coupled), or the block
    diagonal of it for the decoupled D-scheme, on a tiny grid."""
    nx, ny, L = fv.nx, fv.ny, fv.L
    N = nx * ny
    h = fv.h
    K = np.zeros((L * N, L * N))
    for a in range(L):
        for j in range(ny):
            for i in range(nx):
                row = a * N + j * nx + i
                K[row, row] += fv.c[a] * h * h / tau + W[a][j * nx + i]
                for (di, dj) in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                    ii, jj = i + di, j + dj
                    if 0 <= ii < nx and 0 <= jj < ny:
                        k1, k2 = fv.k[a][j, i], fv.k[a][jj, ii]
                        T = 2 * k1 * k2 / (k1 + k2)
                        K[row, row] += T
                        K[row, a * N + jj * nx + ii] -= T
                for b in range(L):
                    if b != a:
                        q = fv.q[(a, b)][j * nx + i]
                        K[row, row] += q
                        if scheme == "coupled":
                            K[row, b * N + j * nx + i] -= q
    return K


@pytest.mark.parametrize("nx,ny,L", [(4, 4, 2), (3, 5, 3)])
def test_dense_brute_force_step_matrices_with_wells(nx, ny, L):
    rng = np.random.default_rng(nx + 10 * ny + 100 * L)
    sig = rng.uniform(0.5, 5.0, (L, L))
    sig = sig + sig.T
    np.fill_diagonal(sig, 0)
    W = [rng.uniform(0, 3.0, nx * ny) * (rng.random(nx * ny) < 0.5) for _ in range(L)]
    fv = FVSystem(nx, ny, L, _k(rng, nx, ny, L), rng.uniform(0.1, 1.0, L), sig,
                  wells={a: (W[a], 1.0 + a) for a in range(L)})
    tau = 0.05
    o = Oracle(fv, tau)
    K = _dense_step_matrix(fv, tau, W, "coupled")
    np.testing.assert_allclose(o.coupled_matrix().toarray(), K, rtol=1e-14,
                               atol=1e-14 * np.abs(K).max())
    Kd = _dense_step_matrix(fv, tau, W, "D")
    N = nx * ny
    for a in range(L):
        np.testing.assert_allclose(o.split_matrix(a).toarray(), Kd[a * N:(a + 1) * N, a * N:(a + 1) * N],
                                   rtol=1e-14, atol=1e-14 * np.abs(Kd).max())


@pytest.mark.parametrize("L", [2, 3])
@pytest.mark.parametrize("scheme", ["coupled", "D", "U"])
def test_paper_workload_maximum_principle_and_mass(L, scheme):
    """The paper-shaped workload (p^0 = 1, wells at p_w = 1.2, no other
    source) at a small size: every scheme's step matrix is an M-matrix whose
    right-hand side weights p^{n-1} and p_w non-negatively, so 1 <= p <= 1.2
    in every cell; pressure rises at the wells; mass balances the well flux."""
    import mc_inputs as mi
    from oracle.schemes import from_workload
    w = mi.paper_wells(L, n=40)
    o = from_workload(w)
    p = [np.ravel(x).copy() for x in w.p0]
    F = [np.ravel(x) for x in w.F]
    Wf, pw = (np.ravel(x) for x in w.wells[L - 1])
    for _ in range(5):
        q = o.step(p, F, scheme)
        for a in range(L):
            assert q[a].min() >= 1.0 - 1e-12 and q[a].max() <= 1.2 + 1e-12
        well = float(np.dot(Wf, pw - q[L - 1]))
        lhs = metrics.mass_change(o.fv, q, p)
        if scheme != "coupled":
            # U-scheme: only the continuum solved second uses the new layer
            wts = {"D": (1.0, 1.0), "U": (1.0, 0.0)}[scheme]
            for a in range(L):
                for b in range(a + 1, L):
                    da, db = q[a] - p[a], q[b] - p[b]
                    lhs += w.tau * float(np.dot(o.fv.q[(a, b)], wts[0] * da + wts[1] * db))
        assert abs(lhs - w.tau * well) <= 1e-12 * (abs(lhs) + 1e-30) + 1e-16
        p = q
    assert q[L - 1][Wf > 0].min() > 1.0
