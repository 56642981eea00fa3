"""Pins of the oracle's time schemes (Sections 3.2 and 3.3)."""

import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

import mc_inputs as mi
from oracle import metrics
from oracle.fv import FVSystem
from oracle.schemes import Oracle, from_workload

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden_uniform():
    out = {}
    with open(os.path.join(GOLD, "uniform_two_continuum.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            s, a, b, c, d = line.split()
            out[s] = (float(Fraction(int(a), int(b))), float(Fraction(int(c), int(d))))
    return out


def _random_k(rng, nx, ny, L):
    return [np.exp(1.5 * rng.standard_normal((ny, nx))) * 10.0 ** (2 * a) for a in range(L)]


@pytest.mark.parametrize("scheme", ["coupled", "D", "L", "U"])
def test_uniform_state_golden(scheme):
    """Heterogeneous k, uniform state: every cell follows the hand-derived
    2 x 2 recurrence of the golden file."""
    g = _golden_uniform()[scheme]
    rng = np.random.default_rng(11)
    nx, ny = 5, 4
    fv = FVSystem(nx, ny, 2, _random_k(rng, nx, ny, 2), [1.0, 0.1],
                  np.array([[0, 10.0], [10.0, 0]]))
    o = Oracle(fv, 1.0 / 50)
    p = o.step([np.ones(nx * ny), np.zeros(nx * ny)], [np.zeros(nx * ny)] * 2, scheme)
    np.testing.assert_allclose(p[0], g[0], rtol=1e-13)
    np.testing.assert_allclose(p[1], g[1], rtol=1e-13)


def test_uniform_difference_decay_factors():
    """d = p1 - p2 decays by g_C = 1/(1 + tau sigma (1/c1 + 1/c2)) per coupled
    step and by g_D = 1 - sigma/(c1/tau + sigma) - sigma/(c2/tau + sigma) per
    D-scheme step (closed forms of the uniform recurrence)."""
    rng = np.random.default_rng(3)
    nx = ny = 6
    c1, c2, s, tau = 0.7, 0.2, 3.0, 0.05
    fv = FVSystem(nx, ny, 2, _random_k(rng, nx, ny, 2), [c1, c2],
                  np.array([[0, s], [s, 0]]))
    o = Oracle(fv, tau)
    p0 = [np.full(nx * ny, 2.0), np.full(nx * ny, -1.0)]
    F = [np.zeros(nx * ny)] * 2
    gC = 1 / (1 + tau * s * (1 / c1 + 1 / c2))
    gD = 1 - s / (c1 / tau + s) - s / (c2 / tau + s)
    for scheme, gfac in (("coupled", gC), ("D", gD)):
        hist = o.run(p0, F, 4, scheme, keep=True)
        for n in range(1, 5):
            d = hist[n][0] - hist[n][1]
            np.testing.assert_allclose(d, 3.0 * gfac ** n, rtol=1e-12)


def test_uniform_three_continuum_recurrence():
    """L = 3, uniform state and uniform sources f |cell|: p^n = G p^{n-1} + g
    with G = (C/tau + S0)^{-1}(C/tau - S1), S the sigma-Laplacian over the
    continua, S0 its part kept implicit by each scheme."""
    rng = np.random.default_rng(5)
    nx, ny = 4, 3
    c = np.array([1.0, 0.2, 0.05])
    sig = np.array([[0, 5.0, 1.0], [5.0, 0, 20.0], [1.0, 20.0, 0]])
    f = np.array([0.3, -0.1, 0.25])
    tau = 1.0 / 200
    fv = FVSystem(nx, ny, 3, _random_k(rng, nx, ny, 3), c, sig)
    o = Oracle(fv, tau)
    S = np.diag(sig.sum(axis=1)) - sig
    C = np.diag(c / tau)
    parts = {
        "coupled": (S, np.zeros((3, 3))),
        "D": (np.diag(np.diag(S)), S - np.diag(np.diag(S))),
        "L": (np.tril(S), np.triu(S, 1)),
        "U": (np.triu(S), np.tril(S, -1)),
    }
    p0 = np.array([1.0, -2.0, 0.5])
    for scheme, (S0, S1) in parts.items():
        x = p0.copy()
        hist = o.run([np.full(nx * ny, v) for v in p0],
                     [np.full(nx * ny, fa * fv.area) for fa in f], 5, scheme, keep=True)
        for n in range(1, 6):
            x = np.linalg.solve(C + S0, (C - S1) @ x + f)
            for a in range(3):
                np.testing.assert_allclose(hist[n][a], x[a], rtol=1e-12, atol=1e-14)


def test_sigma_zero_decouples_exactly():
    rng = np.random.default_rng(9)
    nx, ny, L = 9, 7, 3
    k = _random_k(rng, nx, ny, L)
    c = [1.0, 0.3, 0.05]
    fv = FVSystem(nx, ny, L, k, c, np.zeros((L, L)))
    o = Oracle(fv, 0.01)
    p0 = [rng.standard_normal(nx * ny) for _ in range(L)]
    F = [rng.standard_normal(nx * ny) * fv.area for _ in range(L)]
    single = []
    for a in range(L):
        oa = Oracle(FVSystem(nx, ny, 1, [k[a]], [c[a]]), 0.01)
        single.append(oa.run([p0[a]], [F[a]], 3)[0])
    for scheme in ("coupled", "D", "L", "U"):
        p = o.run(p0, F, 3, scheme)
        for a in range(L):
            np.testing.assert_allclose(p[a], single[a], rtol=1e-13, atol=1e-14)


def test_mass_balance_identities():
    """Coupled: sum m dp = tau sum F. D-scheme: sum m dp + tau sum_pairs
    q (dp_a + dp_b) = tau sum F (the lagged exchange, Eq. si-mc)."""
    w = mi.dual_64(n=16)
    o = from_workload(w)
    fv = o.fv
    F = [np.ravel(x) for x in w.F]
    F[0] = F[0] + 0.01
    p = [np.ravel(x) for x in w.p0]
    for scheme in ("coupled", "D"):
        q = o.step(p, F, scheme)
        lhs = metrics.mass_change(fv, q, p)
        if scheme == "D":
            lhs += o.tau * metrics.exchange_change(fv, q, p)
        rhs = o.tau * metrics.total_source(F)
        assert abs(lhs - rhs) < 1e-13 * max(abs(rhs), 1e-3)


@pytest.mark.parametrize("scheme", ["coupled", "D", "L", "U"])
def test_energy_non_increasing_without_sources(scheme):
    """Theorems 2 and 3 with F = 0: ||p^n||_A <= ||p^{n-1}||_A."""
    w = mi.triple_1024(n=16)
    o = from_workload(w)
    rng = np.random.default_rng(1)
    p = [rng.standard_normal(o.fv.N) for _ in range(3)]
    F = [np.zeros(o.fv.N)] * 3
    e = metrics.energy(o.fv, p)
    for _ in range(6):
        p = o.step(p, F, scheme)
        e2 = metrics.energy(o.fv, p)
        assert e2 <= e * (1 + 1e-12)
        e = e2


def test_theorem2_bound_with_sources():
    """||p^n||_A^2 <= ||p^{n-1}||_A^2 + tau/2 ||F||^2_{(M + tau/2 A)^{-1}}."""
    w = mi.dual_64(n=12)
    o = from_workload(w)
    fv = o.fv
    A = fv.A()
    B = (fv.M() + 0.5 * o.tau * A).toarray()
    rng = np.random.default_rng(2)
    F = [rng.standard_normal(fv.N) * fv.area for _ in range(2)]
    Fv = np.concatenate(F)
    bound = 0.5 * o.tau * Fv @ np.linalg.solve(B, Fv)
    p = [rng.standard_normal(fv.N) for _ in range(2)]
    for _ in range(3):
        q = o.step(p, F, "coupled")
        assert metrics.energy(fv, q) <= metrics.energy(fv, p) + bound * (1 + 1e-10)
        p = q


@pytest.mark.parametrize("L", [2, 3])
def test_split_condition_A0_minus_A1(L):
    """A0 - A1 >= 0 (Eq. dc-op) for the D-, L- and U-splittings: the
    symmetric part of A0 - A1 has no negative eigenvalue."""
    rng = np.random.default_rng(L)
    nx, ny = 4, 4
    sig = rng.uniform(1, 10, (L, L))
    sig = sig + sig.T
    np.fill_diagonal(sig, 0)
    fv = FVSystem(nx, ny, L, _random_k(rng, nx, ny, L), np.ones(L), sig)
    A = fv.A().toarray()
    N = fv.N
    blk = lambda X, a, b: X[a * N:(a + 1) * N, b * N:(b + 1) * N]
    for scheme in ("D", "L", "U"):
        A0 = np.zeros_like(A)
        for a in range(L):
            for b in range(L):
                keep = (a == b) or (scheme == "L" and b < a) or (scheme == "U" and b > a)
                if keep:
                    blk(A0, a, b)[:] = blk(A, a, b)
        A1 = A - A0
        S = A0 - A1
        assert np.linalg.eigvalsh(0.5 * (S + S.T)).min() > -1e-10 * np.abs(A).max()


def test_splitting_error_first_order_in_tau():
    """The decoupled solution approaches the coupled one as O(tau) at a fixed
    final time (Section 3.3: only the exchange is lagged by one layer)."""
    w = mi.dual_64(n=16)
    fv = FVSystem(w.nx, w.ny, w.L, w.k, w.c, w.sigma)
    T = 0.2
    rng = np.random.default_rng(4)
    p0 = [rng.standard_normal(fv.N), rng.standard_normal(fv.N)]
    F = [np.ravel(x) for x in w.F]
    errs = []
    for nsteps in (10, 20, 40, 80):
        o = Oracle(fv, T / nsteps)
        pc = o.run(p0, F, nsteps, "coupled")
        pd = o.run(p0, F, nsteps, "D")
        errs.append(metrics.rel_l2(pc, pd))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(1.7 < r < 2.3 for r in ratios), ratios


def test_oracle_forward_error_two_orderings():
    """Self-accuracy: two fill-reducing orderings agree far below the 1e-10
    parity bar. With an FP64 refinement residual they differed by 2e-11 for
    the coupled three-continuum system at 64 x 64 (constant mode held only by
    the small mass term); the extended-precision residual closes the gap."""
    w = mi.triple_1024(n=64)
    oa = from_workload(w)
    ob = from_workload(w)
    ob.permc_spec = "MMD_AT_PLUS_A"
    F = [np.ravel(x) for x in w.F]
    for scheme in ("coupled", "D"):
        pa = oa.run(w.p0, F, 3, scheme)
        pb = ob.run(w.p0, F, 3, scheme)
        assert metrics.rel_l2(pa, pb) < 1e-13
