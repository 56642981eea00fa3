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


# -- the Dirichlet ghost of the local problems ----------------------------------

def _strip_psi(m, k, two_sided):
    """Hand-solved basis function of one block of m cells on a strip, layers = 0,
    uniform k, one continuum. The constraint makes A psi constant on the block,
    so psi is proportional to u = A^-1 1: a discrete parabola, u_i =
    C - (i - s)^2 / (2k). Two-sided (both ends inside the domain, ghost
    T = 2k at h/2): vertex s = (m-1)/2 and the end equation
    2k u_0 + k (u_0 - u_1) = 1 gives u_0 = m/(4k). One-sided (the left end on
    the zero-flux wall): s = -1/2 and the right end gives u_{m-1} = m/(2k).
    psi = u / mean(u)."""
    i = np.arange(m, dtype=np.float64)
    if two_sided:
        C = m / (4 * k) + (m - 1) ** 2 / (8 * k)
        u = C - (i - (m - 1) / 2) ** 2 / (2 * k)
    else:
        C = m / (2 * k) + (m - 0.5) ** 2 / (2 * k)
        u = C - (i + 0.5) ** 2 / (2 * k)
    return u / u.mean()


@pytest.mark.parametrize("axis", ["x", "y"])
def test_dirichlet_ghost_closed_form(axis):
    """Basis functions of a strip of blocks against the hand-solved parabola:
    pins the interior-boundary ghost T = 2k (with T = k the end value would
    be m/(2k) for the two-sided block and the shape would differ)."""
    m, across, nblk, k = 7, 3, 4, 2.5
    if axis == "x":
        nx, ny, ncx, ncy = m * nblk, across, nblk, 1
    else:
        nx, ny, ncx, ncy = across, m * nblk, 1, nblk
    fv = FVSystem(nx, ny, 1, [np.full((ny, nx), k)], [1.0])
    nl = NLMC(fv, 0.01, ncx, ncy, 0)
    R = nl.R.toarray()
    for blk, two_sided in ((0, False), (1, True), (2, True)):
        psi = R[blk].reshape(ny, nx)
        if axis == "x":
            part = psi[:, blk * m:(blk + 1) * m]
        else:
            part = psi[blk * m:(blk + 1) * m, :].T
        want = _strip_psi(m, k, two_sided)
        np.testing.assert_allclose(part, np.broadcast_to(want, part.shape), rtol=1e-12, atol=1e-13)
        outside = np.delete(psi, np.s_[blk * m:(blk + 1) * m], axis=1 if axis == "x" else 0)
        assert np.abs(outside).max() == 0.0
    # the last block mirrors the first
    last = R[nblk - 1].reshape(ny, nx)
    part = last[:, -m:] if axis == "x" else last[-m:, :].T
    np.testing.assert_allclose(part, np.broadcast_to(_strip_psi(m, k, False)[::-1], part.shape),
                               rtol=1e-12, atol=1e-13)


# -- continua that live on part of the domain (K_j^alpha = Omega_alpha ∩ K_j) ---

def _fracture_case(n=32, nc=4):
    # seed 4045: 15 of the 16 blocks hold fracture cells at 32^2
    w = mi.fracture_instance(4045, n=n, L=2)
    return w, from_workload(w), [None, w.support[1]], nc


def test_support_constraints_and_active_unknowns():
    w, o, sup, nc = _fracture_case()
    nl = NLMC(o.fv, w.tau, nc, nc, 1, support=sup)
    bs = w.nx // nc
    frac_blocks = sup[1].reshape(nc, bs, nc, bs).any(axis=(1, 3)).ravel()
    np.testing.assert_array_equal(nl.active, np.concatenate([np.ones(nc * nc, bool), frac_blocks]))
    assert not frac_blocks.all()   # the case has blocks without fracture cells
    assert nl.constraint_residual < 1e-12
    Rd = nl.R.toarray()
    N = o.fv.N
    for row in range(Rd.shape[0]):
        beta, i = divmod(row, nl.Nc)
        if not nl.active[row]:
            assert np.abs(Rd[row]).max() == 0.0
            continue
        I, J = i % nc, i // nc
        I0, I1, J0, J1 = nl.region(I, J)
        for a in range(2):
            f = Rd[row, a * N:(a + 1) * N].reshape(w.ny, w.nx)
            for JJ in range(J0, J1):
                for II in range(I0, I1):
                    if not nl.active[a * nl.Nc + JJ * nc + II]:
                        continue
                    cells = sup[1] if a == 1 else np.ones_like(sup[1])
                    blk = np.zeros_like(cells)
                    blk[JJ * bs:(JJ + 1) * bs, II * bs:(II + 1) * bs] = True
                    mean = f[cells & blk].mean()
                    want = 1.0 if (a == beta and II == I and JJ == J) else 0.0
                    assert abs(mean - want) < 1e-12
    assert np.abs(nl.mbar[~nl.active]).max() == 0.0
    np.testing.assert_allclose(nl.mbar[nl.Nc:][frac_blocks],
                               0.1 * o.fv.area * sup[1].reshape(nc, bs, nc, bs).sum(axis=(1, 3)).ravel()[frac_blocks])


def test_support_global_oversampling_partition_of_unity():
    """Global oversampling: the constant vector satisfies every constraint
    (mean 1 over every K_j^alpha) with zero energy, so the basis functions of
    the unknowns that exist sum to 1 on every cell, the fracture continuum's
    cells outside Omega_f included, and A_bar annihilates the constant."""
    w, o, sup, nc = _fracture_case()
    nl = NLMC(o.fv, w.tau, nc, nc, nc, support=sup)
    s = np.asarray(nl.R.sum(axis=0)).ravel()
    np.testing.assert_allclose(s, 1.0, atol=1e-9)
    ix = np.flatnonzero(nl.active)
    A = nl.Abar[np.ix_(ix, ix)]
    np.testing.assert_allclose(A @ np.ones(ix.size), 0.0, atol=1e-9 * np.abs(A).max())
    # the conservative option changes nothing where A_bar 1 = 0 already
    nc2 = NLMC(o.fv, w.tau, nc, nc, nc, support=sup, conservative=True)
    np.testing.assert_allclose(nc2.Abar, nl.Abar, rtol=0, atol=1e-9 * np.abs(A).max())


def test_support_global_oversampling_steady_exactness():
    """Sources constant on the cells of each K_j^alpha (zero elsewhere) and
    global oversampling: A p = F lies in the range of C^T, so the fine steady
    solution is in the multiscale space and the coarse coupled solution with
    a vanishing mass term equals the fine means over K_j^alpha (the null
    constant removed from both)."""
    w, o0, sup, nc = _fracture_case()
    fv = FVSystem(w.nx, w.ny, w.L, w.k, w.c, w.sigma, w.sigma_cell)
    tau = 1e9
    o = Oracle(fv, tau)
    bs = w.nx // nc
    F = [np.zeros((w.ny, w.nx)) for _ in range(2)]
    F[0][0:bs, 0:bs] = 0.5 / bs ** 2
    F[0][3 * bs:4 * bs, 2 * bs:3 * bs] = -0.5 / bs ** 2
    nl = NLMC(fv, tau, nc, nc, nc, support=sup)
    act_f = np.flatnonzero(nl.active[nl.Nc:])
    j1, j2 = act_f[0], act_f[-1]
    for j, v in ((j1, 1.0), (j2, -1.0)):
        blk = np.zeros((w.ny, w.nx), bool)
        blk[(j // nc) * bs:(j // nc + 1) * bs, (j % nc) * bs:(j % nc + 1) * bs] = True
        cells = blk & sup[1]
        F[1][cells] = v / cells.sum()
    pf = o.run(w.p0, F, 2, "coupled")
    pb = nl.run(w.p0, F, 2, "coupled")
    ref = nl.coarse_mean(pf)
    cw = np.where(nl.active, nl.mbar, 0.0)
    pb = np.where(nl.active, pb - np.dot(cw, pb) / cw.sum(), 0.0)
    ref = np.where(nl.active, ref - np.dot(cw, ref) / cw.sum(), 0.0)
    assert np.linalg.norm(pb - ref) / np.linalg.norm(ref) < 1e-7


@pytest.mark.parametrize("scheme", ["coupled", "D"])
def test_conservative_coarse_mass_identity(scheme):
    """With local oversampling the conservative coarse operator has
    1^T A_bar = 0, so the coarse coupled step keeps the mass identity
    sum M_bar dp_bar = tau sum (F_bar + W_bar p_w - W_bar p_bar^n) to
    roundoff, and a constant state without sources stays constant; the
    plain Galerkin operator does neither. D-scheme: the lagged exchange adds
    tau sum over pairs of (A_bar_ab block) terms; the identity checked is the
    coupled one for the coupled scheme and constant preservation for both."""
    w = mi.paper_wells(2, n=40)
    o = from_workload(w)
    sup = [None, w.support[1]]
    for cons in (True, False):
        nl = NLMC(o.fv, w.tau, 4, 4, 1, support=sup, conservative=cons)
        ix = np.flatnonzero(nl.active)
        one = np.where(nl.active, 1.0, 0.0)
        # constant state, no sources or wells: unchanged
        save = nl.wbar.copy(), nl.wpbar.copy()
        nl.wbar[:] = 0.0
        nl.wpbar[:] = 0.0
        nl._fact = {}
        p1 = nl.step(one, np.zeros_like(one), scheme)
        dev = np.abs(p1[ix] - 1.0).max()
        if cons:
            assert dev < 1e-9, dev
        else:
            assert dev > 1e-3, dev
        nl.wbar[:], nl.wpbar[:] = save
        nl._fact = {}
        if scheme == "coupled" and cons:
            p0 = nl.coarse_mean(w.p0)
            Fb = nl.coarse_source(w.F)
            p1 = nl.step(p0, Fb, scheme)
            lhs = np.dot(nl.mbar, p1 - p0)
            rhs = w.tau * np.sum(Fb + nl.wpbar - nl.wbar * p1)
            scale = np.dot(nl.mbar, np.abs(p1)) + w.tau * np.sum(np.abs(nl.wpbar) + nl.wbar * np.abs(p1))
            assert abs(lhs - rhs) < 1e-12 * scale


@pytest.mark.parametrize("scheme", ["coupled", "D", "U"])
def test_one_cell_blocks_reproduce_fine_scheme_with_wells(scheme):
    """Coarse blocks of one cell with wells: R = I, the coarse well sums are
    the fine well terms, and the coarse schemes are the fine ones."""
    w = mi.paper_wells(2, n=10)
    o = from_workload(w)
    nl = NLMC(o.fv, w.tau, 10, 10, 1)
    np.testing.assert_allclose(nl.R.toarray(), np.eye(200), atol=1e-13)
    pf = o.run(w.p0, w.F, 3, scheme)
    pb = nl.run(w.p0, w.F, 3, scheme)
    np.testing.assert_allclose(pb, np.concatenate(pf), rtol=1e-11, atol=1e-14)
