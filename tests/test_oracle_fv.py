"""Pins of the oracle's finite-volume assembly (Section 3.1)."""

import os

import numpy as np
import pytest

from oracle.fv import FVSystem, harmonic_face
from oracle.schemes import Oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            out[parts[0]] = [float(x) for x in parts[1:]]
    return out


def test_two_cell_hand_example():
    g = _read_golden("two_cell_hand.txt")
    fv = FVSystem(2, 1, 1, [np.array([[1.0, 3.0]])], [2.0])
    assert fv.TE[0].shape == (1, 1) and fv.TN[0].shape == (0, 2)
    assert fv.TE[0][0, 0] == pytest.approx(g["T12"][0], rel=1e-15)
    o = Oracle(fv, 0.25)
    p = o.run([np.zeros(2)], [np.array([1.0, 0.0])], 1, "coupled")
    assert p[0][0] == pytest.approx(g["p1"][0], rel=1e-14)
    assert p[0][1] == pytest.approx(g["p2"][0], rel=1e-14)


def test_harmonic_mean_special_cases():
    assert harmonic_face(2.0, 2.0) == 2.0
    assert harmonic_face(0.0, 5.0) == 0.0
    assert harmonic_face(0.0, 0.0) == 0.0
    # harmonic mean lies between min and 2*min
    a, b = 1e-2, 1e4
    v = harmonic_face(a, b)
    assert a < v < 2 * a


@pytest.mark.parametrize("nx,ny", [(8, 8), (6, 10)])
@pytest.mark.parametrize("m,l", [(1, 0), (0, 1), (2, 3), (5, 1)])
def test_cosine_modes_are_eigenvectors(nx, ny, m, l):
    """For uniform k, cos(pi m (i+1/2)/nx) cos(pi l (j+1/2)/ny) is an
    eigenvector of the zero-flux TPFA matrix with eigenvalue
    2k (2 - cos(pi m/nx) - cos(pi l/ny)); one backward-Euler step scales it
    by 1/(1 + tau lambda / (c h^2))."""
    k0, c, tau = 3.7, 0.6, 0.01
    fv = FVSystem(nx, ny, 1, [np.full((ny, nx), k0)], [c])
    i = np.arange(nx) + 0.5
    j = np.arange(ny) + 0.5
    v = np.outer(np.cos(np.pi * l * j / ny), np.cos(np.pi * m * i / nx)).ravel()
    lam = 2 * k0 * (2 - np.cos(np.pi * m / nx) - np.cos(np.pi * l / ny))
    np.testing.assert_allclose(fv.D[0] @ v, lam * v, atol=1e-12 * max(lam, 1))
    o = Oracle(fv, tau)
    p = o.run([v], [np.zeros(nx * ny)], 1, "coupled")[0]
    np.testing.assert_allclose(p, v / (1 + tau * lam / (c * fv.h ** 2)), atol=1e-13)


def _brute_dense(nx, ny, k, c, sigma, h):
    """The coupled operator written equation by equation from Eq. app:
    for each continuum a and cell i, the flux T (p_a,i - p_a,j) to every
    neighbour j plus sigma |cell| (p_a,i - p_b,i) to every other continuum."""
    L = len(k)
    N = nx * ny
    A = np.zeros((L * N, L * N))
    M = np.zeros(L * N)
    for a in range(L):
        for j in range(ny):
            for i in range(nx):
                row = a * N + j * nx + i
                M[row] = c[a] * h * h
                for (di, dj) in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                    ii, jj = i + di, j + dj
                    if 0 <= ii < nx and 0 <= jj < ny:
                        k1, k2 = k[a][j, i], k[a][jj, ii]
                        T = 2 * k1 * k2 / (k1 + k2) * h / h
                        A[row, row] += T
                        A[row, a * N + jj * nx + ii] -= T
                for b in range(L):
                    if b != a:
                        s = sigma[a][b] * h * h
                        A[row, row] += s
                        A[row, b * N + j * nx + i] -= s
    return A, M


@pytest.mark.parametrize("nx,ny,L", [(4, 4, 2), (3, 5, 2), (4, 4, 3), (3, 5, 3)])
def test_dense_brute_force_operator(nx, ny, L):
    rng = np.random.default_rng(nx * 100 + ny * 10 + L)
    k = [np.exp(2 * rng.standard_normal((ny, nx))) * 10 ** a for a in range(L)]
    c = rng.uniform(0.1, 1.0, L)
    sig = rng.uniform(0.5, 5.0, (L, L))
    sig = sig + sig.T
    np.fill_diagonal(sig, 0)
    fv = FVSystem(nx, ny, L, k, c, sig)
    A, M = _brute_dense(nx, ny, k, c, sig, 1.0 / nx)
    np.testing.assert_allclose(fv.A().toarray(), A, rtol=1e-14, atol=1e-14 * np.abs(A).max())
    np.testing.assert_allclose(fv.M().diagonal(), M, rtol=1e-15)


def test_operator_symmetric_and_conservative():
    rng = np.random.default_rng(7)
    nx, ny, L = 7, 5, 3
    k = [np.exp(rng.standard_normal((ny, nx))) for _ in range(L)]
    sc = {(0, 2): rng.uniform(0, 3, (ny, nx))}
    sig = np.array([[0, 1.0, 2.0], [1.0, 0, 4.0], [2.0, 4.0, 0]])
    fv = FVSystem(nx, ny, L, k, np.ones(L), sig, sc)
    A = fv.A().toarray()
    np.testing.assert_allclose(A, A.T, atol=1e-14)
    # 1^T (D + Q) = 0: every flux leaves one cell and enters another.
    np.testing.assert_allclose(A.sum(axis=0), 0, atol=1e-13)
    assert np.linalg.eigvalsh(A).min() > -1e-12
    # per-cell sigma overrides the constant for that pair only
    assert np.allclose(fv.q[(0, 2)], sc[(0, 2)].ravel() * fv.area)
    assert np.allclose(fv.q[(1, 2)], 4.0 * fv.area)
