"""Pins of the oracle's NLMC coarse model (Section 4)."""

import numpy as np
import pytest

import mc_inputs as mi
from oracle import metrics
from oracle.fv import FVSystem
from oracle.nlmc import NLMC
from oracle.schemes import Oracle, from_workload


@pytest.mark.parametrize("scheme", ["coupled", "D", "L", "U"])
def test_one_cell_blocks_reproduce_fine_scheme(scheme):
    """Coarse block = one fine cell: the constraints fix psi completely,
    R = I, A_bar = A, M_bar = M, F_bar = F, and every coarse scheme is the
    fine scheme."""
    w = mi.triple_1024(n=8)
    o = from_workload(w)
    nl = NLMC(o.fv, w.tau, 8, 8, 1)
    np.testing.assert_allclose(nl.R.toarray(), np.eye(3 * 64), atol=1e-13)
    np.testing.assert_allclose(nl.Abar, o.fv.A().toarray(), atol=1e-10)
    pf = o.run(w.p0, w.F, 4, scheme)
    pb = nl.run(w.p0, w.F, 4, scheme)
    np.testing.assert_allclose(pb, np.concatenate(pf), rtol=1e-11, atol=1e-14)


def test_constraints_and_coarse_operator_properties():
    w = mi.nlmc_1024(n=32, ncoarse=4, layers=1)
    o = from_workload(w)
    nl = NLMC(o.fv, w.tau, 4, 4, 1)
    assert nl.constraint_residual < 1e-12
    # block means of every basis function, recomputed from R: delta_ij delta_ab
    # on the blocks of its region (and zero elsewhere is not required).
    Rd = nl.R.toarray()
    N = o.fv.N
    for row in range(Rd.shape[0]):
        beta, i = divmod(row, nl.Nc)
        I, J = i % 4, i // 4
        I0, I1, J0, J1 = nl.region(I, J)
        for a in range(2):
            means = metrics.block_mean(Rd[row, a * N:(a + 1) * N], 32, 32, 8, 8).reshape(4, 4)
            for JJ in range(J0, J1):
                for II in range(I0, I1):
                    want = 1.0 if (a == beta and II == I and JJ == J) else 0.0
                    assert abs(means[JJ, II] - want) < 1e-12
    A = nl.Abar
    assert np.abs(A - A.T).max() < 1e-10 * np.abs(A).max()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > -1e-9 * np.abs(A).max()


def test_global_oversampling_partition_of_unity():
    """With a region covering the whole domain the constant function is the
    energy minimiser for unit means, so sum of all basis functions = 1 and
    A_bar annihilates the constant coarse vector."""
    w = mi.triple_1024(n=16)
    o = from_workload(w)
    nl = NLMC(o.fv, w.tau, 4, 4, 4)
    s = np.asarray(nl.R.sum(axis=0)).ravel()
    np.testing.assert_allclose(s, 1.0, atol=1e-9)
    np.testing.assert_allclose(nl.Abar @ np.ones(nl.Abar.shape[0]), 0.0,
                               atol=1e-9 * np.abs(nl.Abar).max())


def test_global_oversampling_steady_exactness():
    """Sources constant on each coarse block and a region covering the whole
    domain: the fine steady solution lies in the multiscale space, so with a
    vanishing mass term the coarse solution equals the fine block means. The
    global constant (the null mode of D + Q, fixed only by the vanishing mass
    term) is removed from both sides before comparing."""
    w = mi.triple_1024(n=32)
    fv = FVSystem(w.nx, w.ny, w.L, w.k, w.c, w.sigma)
    tau = 1e9
    o = Oracle(fv, tau)
    F = [np.zeros((32, 32)) for _ in range(3)]
    F[2][4:8, 4:8] = 1 / 16
    F[2][24:28, 24:28] = -1 / 16
    F[0][0:4, 8:12] = 0.3 / 16
    F[0][8:12, 0:4] = -0.3 / 16
    nl = NLMC(fv, tau, 8, 8, 8)
    pf = o.run(w.p0, F, 2, "coupled")
    pb = nl.run(w.p0, F, 2, "coupled")
    ref = nl.coarse_mean(pf)
    cw = np.repeat(w.c, nl.Nc)
    pb = pb - np.dot(cw, pb) / cw.sum()
    ref = ref - np.dot(cw, ref) / cw.sum()
    assert np.linalg.norm(pb - ref) / np.linalg.norm(ref) < 1e-7


def test_oversampling_error_decays_with_layers():
    w = mi.triple_1024(n=32)
    fv = FVSystem(w.nx, w.ny, w.L, w.k, w.c, w.sigma)
    tau = 1e6
    o = Oracle(fv, tau)
    F = [np.zeros((32, 32)) for _ in range(3)]
    F[2][4:8, 4:8] = 1 / 16
    F[2][24:28, 24:28] = -1 / 16
    pf = o.run(w.p0, F, 2, "coupled")
    errs = []
    for lay in (1, 2, 3):
        nl = NLMC(fv, tau, 8, 8, lay)
        cw = np.repeat(w.c, nl.Nc)
        ref = nl.coarse_mean(pf)
        ref = ref - np.dot(cw, ref) / cw.sum()
        pb = nl.run(w.p0, F, 2, "coupled")
        pb = pb - np.dot(cw, pb) / cw.sum()
        errs.append(np.linalg.norm(pb - ref) / np.linalg.norm(ref))
    assert errs[0] > 3 * errs[1] > 9 * errs[2], errs
