"""GPU parity of the NLMC coarse model (Section 4) against the oracle.

Basis functions, A_bar = R A R^T, M_bar, F_bar and the coarse coupled / D /
L / U runs are compared with the oracle's direct KKT solves. The basis PCG
stops at a 1e-12 reduction of its preconditioned residual; the tolerances
below follow from that (measured values are well inside them).
"""

import numpy as np
import pytest

import mc_inputs as mi
from oracle.nlmc import NLMC as ONLMC
from oracle.schemes import from_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    import paper_2209_01158_gb300 as m
    m._lib()
    return m


def _pair(mc, w, ncx, layers, support=False, conservative=False):
    ctx = mc.Context.from_workload(w)
    sup = [w.support.get(a) for a in range(w.L)] if support else None
    nl = mc.NLMC(ctx, ncx, ncx, layers, support=sup, conservative=conservative)
    o = from_workload(w)
    onl = ONLMC(o.fv, w.tau, ncx, ncx, layers, support=sup, conservative=conservative)
    return ctx, nl, o, onl


def _compare(mc, w, ncx, layers, support, conservative, nsteps=10, schemes=("coupled", "D", "L", "U"),
             basis_blocks=None):
    ctx, nl, o, onl = _pair(mc, w, ncx, layers, support, conservative)
    Nc = ncx * ncx
    np.testing.assert_array_equal(nl.active(), onl.active)
    R = onl.R.toarray() if basis_blocks is None else None
    worst = 0.0
    blocks = range(Nc) if basis_blocks is None else basis_blocks
    for i in blocks:
        for beta in range(w.L):
            ref = R[beta * Nc + i] if R is not None else onl.R.getrow(beta * Nc + i).toarray().ravel()
            got = nl.basis(i, beta)
            if not onl.active[beta * Nc + i]:
                assert np.abs(got).max() == 0.0 and np.abs(ref).max() == 0.0
                continue
            worst = max(worst, np.linalg.norm(got - ref) / np.linalg.norm(ref))
    # With a support mask the fracture continuum's cells outside Omega_f
    # (k = 1e-2, no exchange) are unconstrained: the local problems are about
    # 1e6 times stiffer than with whole-block constraints, and the same
    # 1e-12 basis tolerance leaves basis errors of a few 1e-9 (measured
    # 1.1e-9 .. 5.5e-9); A_bar and the coarse runs keep their bars.
    assert worst < (1e-8 if support else 1e-9), worst
    A, m, f = nl.operator()
    np.testing.assert_allclose(A, onl.Abar, rtol=0, atol=1e-9 * np.abs(onl.Abar).max())
    np.testing.assert_allclose(m, onl.mbar, rtol=1e-14)
    np.testing.assert_allclose(f, onl.coarse_source(w.F), rtol=0, atol=1e-14)
    np.testing.assert_allclose(nl.get_state(), onl.coarse_mean(w.p0), rtol=1e-14, atol=1e-15)
    for scheme in schemes:
        nl.set_state(onl.coarse_mean(w.p0))
        nl.step(scheme, nsteps)
        got = nl.get_state()
        ref = onl.run(w.p0, w.F, nsteps, scheme)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < 1e-8, (scheme, err)
        assert np.abs(got[~onl.active]).max(initial=0.0) == 0.0
    nl.close()
    ctx.close()


CASES = [
    ("triple_32_c4_l1", lambda: mi.triple_1024(n=32), 4, 1),
    ("triple_40_c5_l2", lambda: mi.triple_1024(n=40), 5, 2),
    ("fracture_64_c8_l2", lambda: mi.fracture_instance(4005, n=64, L=2), 8, 2),
    ("fracture_48_c6_l1_L3", lambda: mi.fracture_instance(4006, n=48, L=3), 6, 1),
]


@pytest.mark.parametrize("name,make,ncx,layers", CASES)
def test_basis_operator_and_runs(mc, name, make, ncx, layers):
    w = make()
    ctx, nl, o, onl = _pair(mc, w, ncx, layers)
    Nc = ncx * ncx
    R = onl.R.toarray()
    worst = 0.0
    for i in range(Nc):
        for beta in range(w.L):
            ref = R[beta * Nc + i]
            got = nl.basis(i, beta)
            worst = max(worst, np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert worst < 1e-9, worst
    A, m, f = nl.operator()
    np.testing.assert_allclose(A, onl.Abar, rtol=0, atol=1e-9 * np.abs(onl.Abar).max())
    np.testing.assert_allclose(m, onl.mbar, rtol=1e-14)
    np.testing.assert_allclose(f, onl.coarse_source(w.F), rtol=0, atol=1e-14)
    np.testing.assert_allclose(nl.get_state(), onl.coarse_mean(w.p0), atol=1e-15)
    for scheme in ("coupled", "D", "L", "U"):
        nl.set_state(onl.coarse_mean(w.p0))
        nl.step(scheme, 10)
        got = nl.get_state()
        ref = onl.run(w.p0, w.F, 10, scheme)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < 1e-8, (scheme, err)
    nl.close()
    ctx.close()


def test_one_cell_blocks_reproduce_fine_gpu_scheme(mc):
    """Coarse block = one fine cell: NLMC on the GPU must follow the fine
    oracle exactly (R = I)."""
    w = mi.triple_1024(n=12)
    ctx = mc.Context.from_workload(w)
    nl = mc.NLMC(ctx, 12, 12, 1)
    o = from_workload(w)
    for scheme in ("coupled", "D", "U"):
        nl.set_state(np.concatenate([np.ravel(x) for x in w.p0]))
        nl.step(scheme, 5)
        ref = np.concatenate(o.run(w.p0, w.F, 5, scheme))
        got = nl.get_state()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-9
    nl.close()
    ctx.close()


SUPPORT_CASES = [
    # seed 4045: fracture cells in 15 of 16 blocks at 32^2, 56 of 64 at 64^2
    ("fracture_64_c8_l2_support", lambda: mi.fracture_instance(4045, n=64, L=2), 8, 2, True, False),
    ("fracture_64_c8_l2_support_cons", lambda: mi.fracture_instance(4045, n=64, L=2), 8, 2, True, True),
    ("fracture_48_c6_l1_L3_cons", lambda: mi.fracture_instance(4006, n=48, L=3), 6, 1, False, True),
    ("fracture_48_c6_l1_L3_support", lambda: mi.fracture_instance(4011, n=48, L=3), 6, 1, True, True),
]


@pytest.mark.parametrize("name,make,ncx,layers,support,cons", SUPPORT_CASES)
def test_support_and_conservative(mc, name, make, ncx, layers, support, cons):
    """K_j^alpha = Omega_alpha ∩ K_j (fracture cells only) and the
    conservative coarse operator, against the oracle."""
    _compare(mc, make(), ncx, layers, support, cons)


def test_coarse_wells(mc):
    """Paper-shaped 2C problem (p0 = 1, wells) on a coarse grid: the coarse
    well sums and the implicit coarse well term of every scheme."""
    _compare(mc, mi.paper_wells(2, n=40), 4, 1, True, True)


def test_config5_block_geometry(mc):
    """The kernel shape of the 1024^2 coarse workload: 32 x 32-cell coarse
    blocks, 2 oversampling layers (regions of up to 160 x 160 cells x 2
    continua, 1024-thread CTAs looping over 51,200 unknowns), on a 256^2 crop
    of the same recipe (8 x 8 blocks), fracture support and conservative
    operator. Basis functions checked on a sample of blocks (corner, edge,
    interior), A_bar, M_bar, F_bar and 10 coarse steps of every scheme."""
    w = mi.nlmc_1024(n=256, ncoarse=8, layers=2)
    _compare(mc, w, 8, 2, True, True, basis_blocks=[0, 3, 27, 36, 63])
