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


def _pair(mc, w, ncx, layers):
    ctx = mc.Context.from_workload(w)
    nl = mc.NLMC(ctx, ncx, ncx, layers)
    o = from_workload(w)
    onl = ONLMC(o.fv, w.tau, ncx, ncx, layers)
    return ctx, nl, o, onl


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
