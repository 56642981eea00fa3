"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerance: relative L2 over all continuum cells <= 1e-10 for the FP64 path
(the PCG stops at ||r|| <= 1e-12 ||b||; the oracle's own forward error is
below 1e-13). Coefficients and single operator applications are compared
element by element to a few ulps.
"""

import numpy as np
import pytest

import mc_inputs as mi
from oracle import metrics
from oracle.fv import FVSystem
from oracle.schemes import Oracle, from_workload

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


@pytest.fixture(scope="module")
def mc():
    import paper_2209_01158_gb300 as m
    m._lib()
    return m


def gpu_run(mc, w, scheme, nsteps, **opt):
    o = mc.mc_default_opts()
    for k, v in opt.items():
        setattr(o, k, v)
    ctx = mc.Context.from_workload(w, opts=o)
    st = ctx.step(scheme, nsteps)
    p = ctx.get_state()
    ctx.close()
    return p, st


def oracle_run(w, scheme, nsteps):
    return from_workload(w).run(w.p0, w.F, nsteps, scheme)


def test_coefficients_match(mc):
    for w in (mi.dual_64(), mi.fracture_instance(4001, n=40, L=3)):
        ctx = mc.Context.from_workload(w)
        fv = FVSystem(w.nx, w.ny, w.L, w.k, w.c, w.sigma, w.sigma_cell)
        o = Oracle(fv, w.tau)
        for a in range(w.L):
            TE, TN, dg = ctx.coefficients(a)
            TE = TE.reshape(w.ny, w.nx)
            TN = TN.reshape(w.ny, w.nx)
            np.testing.assert_allclose(TE[:, :-1], fv.TE[a], rtol=1e-15, atol=0)
            assert np.all(TE[:, -1] == 0)
            np.testing.assert_allclose(TN[:-1, :], fv.TN[a], rtol=1e-15, atol=0)
            assert np.all(TN[-1, :] == 0)
            np.testing.assert_allclose(dg, o.split_matrix(a).diagonal(), rtol=1e-14)
        ctx.close()


@pytest.mark.parametrize("scheme", ["D", "coupled"])
def test_operator_and_rhs_match(mc, scheme):
    w = mi.fracture_instance(4002, n=37, L=3)
    ctx = mc.Context.from_workload(w)
    o = from_workload(w)
    rng = np.random.default_rng(0)
    x = [rng.standard_normal(w.nx * w.ny) for _ in range(w.L)]
    y = ctx.apply(scheme, x)
    if scheme == "coupled":
        ref = o.coupled_matrix() @ np.concatenate(x)
        ref = [ref[a * o.fv.N:(a + 1) * o.fv.N] for a in range(w.L)]
    else:
        ref = [o.split_matrix(a) @ x[a] for a in range(w.L)]
    for a in range(w.L):
        np.testing.assert_allclose(y[a], ref[a], rtol=0, atol=1e-13 * np.abs(ref[a]).max())
    ctx.set_state(x)
    b = ctx.rhs_decoupled()
    F = [np.ravel(f) for f in w.F]
    for a in range(w.L):
        rb = o.rhs_split(a, x, [None] * w.L, F)
        np.testing.assert_allclose(b[a], rb, rtol=0, atol=1e-14 * np.abs(rb).max())
    ctx.close()


@pytest.mark.parametrize("scheme", ["D", "L", "U", "coupled"])
def test_dual_64_full_run(mc, scheme):
    """The dual-continuum 64 x 64 workload, all 50 steps."""
    w = mi.dual_64()
    p, st = gpu_run(mc, w, scheme, w.nsteps)
    ref = oracle_run(w, scheme, w.nsteps)
    err = metrics.rel_l2(ref, p)
    assert st["steps_done"] == w.nsteps
    assert err <= FP64_TOL, err
    assert st["mass_defect"] < 1e-9


@pytest.mark.parametrize("scheme", ["D", "L", "U", "coupled"])
def test_three_continuum_ragged(mc, scheme):
    """100 x 100 is not a multiple of the 64 x 8 stencil tile in either
    direction: several tiles plus a ragged tail."""
    w = mi.triple_1024(n=100)
    p, st = gpu_run(mc, w, scheme, 8)
    ref = oracle_run(w, scheme, 8)
    assert metrics.rel_l2(ref, p) <= FP64_TOL


@pytest.mark.parametrize("scheme", ["D", "coupled"])
def test_fracture_instance_per_cell_exchange(mc, scheme):
    w = mi.fracture_instance(4003, n=72, L=3)
    p, st = gpu_run(mc, w, scheme, 6)
    ref = oracle_run(w, scheme, 6)
    assert metrics.rel_l2(ref, p) <= FP64_TOL


@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 9), (13, 1), (65, 3)])
def test_degenerate_grids(mc, nx, ny):
    rng = np.random.default_rng(nx * 31 + ny)
    L = 2
    k = [np.exp(rng.standard_normal((ny, nx))), 100 * np.exp(rng.standard_normal((ny, nx)))]
    sig = np.array([[0, 3.0], [3.0, 0]])
    w = mi.Workload("deg", nx, ny, L, k, np.array([1.0, 0.1]), sig, 0.02, 5,
                    [rng.standard_normal((ny, nx)) * 1e-3 for _ in range(L)],
                    [rng.standard_normal((ny, nx)) for _ in range(L)])
    for scheme in ("D", "U", "coupled"):
        p, st = gpu_run(mc, w, scheme, 5)
        ref = oracle_run(w, scheme, 5)
        assert metrics.rel_l2(ref, p) <= FP64_TOL


def test_single_continuum_and_no_exchange(mc):
    w = mi.triple_1024(n=48)
    w.sigma = np.zeros((3, 3))
    pd, _ = gpu_run(mc, w, "D", 4)
    pc, _ = gpu_run(mc, w, "coupled", 4)
    ref = oracle_run(w, "coupled", 4)
    assert metrics.rel_l2(ref, pd) <= FP64_TOL
    assert metrics.rel_l2(ref, pc) <= FP64_TOL
    w1 = mi.Workload("one", 48, 48, 1, [w.k[2]], np.array([0.05]), np.zeros((1, 1)), w.tau, 4,
                     [w.F[2]], [w.p0[2]])
    p1, _ = gpu_run(mc, w1, "D", 4)
    assert metrics.rel_l2(oracle_run(w1, "D", 4), p1) <= FP64_TOL


def test_zero_state_zero_source_and_zero_steps(mc):
    w = mi.dual_64(n=16)
    w.F = [np.zeros((16, 16))] * 2
    p, st = gpu_run(mc, w, "D", 3)
    assert all(np.all(x == 0) for x in p)
    assert st["iters"][:2] == [0, 0]
    w2 = mi.dual_64(n=16)
    p2, st2 = gpu_run(mc, w2, "D", 0)
    assert st2["steps_done"] == 0 and all(np.all(x == 0) for x in p2)


def test_noconv_rolls_back_to_last_completed_step(mc):
    import paper_2209_01158_gb300 as m
    w = mi.dual_64(n=32)
    o = mc.mc_default_opts()
    ctx = mc.Context.from_workload(w, opts=o)
    ctx.step("D", 2)
    good = [x.copy() for x in ctx.get_state()]
    o.max_iter = 2
    ctx.set_opts(o)
    st = ctx.step("D", 3, check=False)
    assert st["return"] == m.N.MC_E_NOCONV and st["steps_done"] == 0
    after = ctx.get_state()
    for a in range(2):
        np.testing.assert_array_equal(after[a], good[a])
    ctx.close()


def test_barrier_timeout_is_reported_and_context_survives(mc):
    """A one-poll spin limit makes the first grid barrier give up: the run
    returns MC_E_TIMEOUT, the state is rolled back, and the same context then
    steps normally."""
    import paper_2209_01158_gb300 as m
    w = mi.dual_64(n=64)
    o = mc.mc_default_opts()
    o.spin_limit = 1
    ctx = mc.Context.from_workload(w, opts=o)
    st = ctx.step("D", 2, check=False)
    assert st["return"] == m.N.MC_E_TIMEOUT
    assert all(np.all(x == 0) for x in ctx.get_state())
    ctx.set_opts(mc.mc_default_opts())
    ctx.step("D", 2)
    ref = oracle_run(w, "D", 2)
    assert metrics.rel_l2(ref, ctx.get_state()) <= FP64_TOL
    ctx.close()


def test_invalid_arguments_rejected(mc):
    import paper_2209_01158_gb300 as m
    w = mi.dual_64(n=8)
    bad = [np.ravel(w.k[0]).copy(), np.ravel(w.k[1]).copy()]
    bad[0][3] = np.nan
    with pytest.raises(m.MCError) as e:
        m.Context(8, 8, bad, w.c, w.sigma, None, w.tau)
    assert e.value.status == m.N.MC_E_ARG
    with pytest.raises(m.MCError):
        m.Context(8, 8, [np.ravel(x) for x in w.k], w.c, w.sigma, None, -1.0)
    asym = np.array([[0, 1.0], [2.0, 0]])
    with pytest.raises(m.MCError):
        m.Context(8, 8, [np.ravel(x) for x in w.k], w.c, asym, None, w.tau)
    ctx = m.Context.from_workload(w)
    with pytest.raises(m.MCError):
        ctx.step_decoupled(7, 1)
    ctx.close()


def test_deterministic_and_restartable(mc):
    """Same inputs give bit-identical states; 3 + 2 steps through a host
    checkpoint equal 5 uninterrupted steps bit for bit."""
    w = mi.triple_1024(n=80)
    a, _ = gpu_run(mc, w, "D", 5)
    b, _ = gpu_run(mc, w, "D", 5)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    ctx = mc.Context.from_workload(w)
    ctx.step("D", 3)
    ck = [x.copy() for x in ctx.get_state()]
    ctx.close()
    ctx2 = mc.Context.from_workload(w)
    ctx2.set_state(ck)
    ctx2.step("D", 2)
    c = ctx2.get_state()
    ctx2.close()
    for x, y in zip(a, c):
        np.testing.assert_array_equal(x, y)
