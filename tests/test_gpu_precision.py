"""GPU parity of the precision form: FP32 inner PCG (transmissibilities in
FP32 or BF16) inside FP64 iterative refinement, decoupled schemes.

Bar: relative L2 <= 1e-8 against the FP64 oracle (the mixed-precision
target), with the outer FP64 residual driven to rtol = 1e-10.
"""

import numpy as np
import pytest

import mc_inputs as mi
from oracle import metrics
from oracle.schemes import from_workload

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-8


@pytest.fixture(scope="module")
def mc():
    import paper_2209_01158_gb300 as m
    m._lib()
    return m


def run(mc, w, scheme, nsteps, precision, rtol=1e-10, inner_form=0):
    o = mc.mc_default_opts()
    o.precision = precision
    o.rtol = rtol
    o.inner_form = inner_form
    ctx = mc.Context.from_workload(w, opts=o)
    st = ctx.step(scheme, nsteps)
    p = ctx.get_state()
    ctx.close()
    return p, st


# inner_form 0: single-reduction (Chronopoulos-Gear) inner PCG, the default;
# 1: the two-reduction textbook recurrences
@pytest.mark.parametrize("inner_form", [0, 1])
@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("scheme", ["D", "L", "U"])
def test_three_continuum_ragged(mc, precision, scheme, inner_form):
    w = mi.triple_1024(n=100)
    p, st = run(mc, w, scheme, 6, precision, inner_form=inner_form)
    ref = from_workload(w).run(w.p0, w.F, 6, scheme)
    assert metrics.rel_l2(ref, p) <= MIXED_TOL
    assert st["ir_sweeps"] > 0


@pytest.mark.parametrize("inner_form", [0, 1])
@pytest.mark.parametrize("precision", [1, 2])
def test_dual_64_full_run(mc, precision, inner_form):
    w = mi.dual_64()
    p, st = run(mc, w, "D", w.nsteps, precision, inner_form=inner_form)
    ref = from_workload(w).run(w.p0, w.F, w.nsteps, "D")
    assert metrics.rel_l2(ref, p) <= MIXED_TOL


@pytest.mark.parametrize("inner_form", [0, 1])
def test_fracture_instance_per_cell_exchange(mc, inner_form):
    w = mi.fracture_instance(4007, n=72, L=3)
    p, st = run(mc, w, "D", 5, 2, inner_form=inner_form)
    ref = from_workload(w).run(w.p0, w.F, 5, "D")
    assert metrics.rel_l2(ref, p) <= MIXED_TOL


def test_inner_form_out_of_range_rejected(mc):
    w = mi.dual_64(n=16)
    o = mc.mc_default_opts()
    o.precision = 1
    o.inner_form = 2
    with pytest.raises(Exception):
        mc.Context.from_workload(w, opts=o)


def test_coupled_scheme_rejects_precision_form(mc):
    w = mi.dual_64(n=16)
    o = mc.mc_default_opts()
    o.precision = 1
    ctx = mc.Context.from_workload(w, opts=o)
    st = ctx.step("coupled", 1, check=False)
    assert st["return"] == mc.N.MC_E_ARG
    ctx.close()


@pytest.mark.parametrize("precision", [1, 2])
def test_precision_recipe_1024_against_oracle(mc, precision):
    """The 4096^2 precision workload's recipe (k2 contrast 1e5) at 1024^2,
    two steps, against the oracle's direct solves."""
    w = mi.precision_4096(n=1024)
    p, st = run(mc, w, "D", 2, precision)
    ref = from_workload(w).run(w.p0, w.F, 2, "D")
    assert metrics.rel_l2(ref, p) <= MIXED_TOL, st


def test_precision_4096_against_fp64_path(mc):
    """At 4096^2 the sparse direct oracle does not fit (32-bit indices); the
    mixed path is compared with the GPU FP64 path, itself checked against the
    oracle at up to 1024^2 (one step, FP64 at rtol 1e-12)."""
    w = mi.precision_4096(n=4096)
    p_mixed, _ = run(mc, w, "D", 1, 1)
    p_fp64, _ = run(mc, w, "D", 1, 0, rtol=1e-12)
    assert metrics.rel_l2(p_fp64, p_mixed) <= MIXED_TOL
