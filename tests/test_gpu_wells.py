"""GPU parity of the implicit well term (Section 5's well source, taken
implicitly: W added to the continuum's own diagonal, W p_w to its right-hand
side) on the paper-shaped workloads (p^0 = 1, wells at p_w = 1.2 in the
fracture continuum, tau = 4e-5), against the FP64 oracle.

Bars as elsewhere: rel-L2 <= 1e-10 for the FP64 path at rtol 1e-12, <= 1e-8
for the precision forms. Grid sizes are not multiples of the 64 x 16 tile.
"""

import numpy as np
import pytest

import mc_inputs as mi
from oracle import metrics
from oracle.schemes import from_workload

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-8


@pytest.fixture(scope="module")
def mc():
    import paper_2209_01158_gb300 as m
    m._lib()
    return m


def opts(mc, precision=0, rtol=1e-12):
    o = mc.mc_default_opts()
    o.precision = precision
    o.rtol = rtol
    return o


@pytest.mark.parametrize("L,n", [(2, 72), (3, 50)])
@pytest.mark.parametrize("scheme", ["coupled", "D", "L", "U"])
def test_fp64_schemes_with_wells(mc, L, n, scheme):
    w = mi.paper_wells(L, n=n)
    ctx = mc.Context.from_workload(w, opts=opts(mc))
    st = ctx.step(scheme, 8)
    p = ctx.get_state()
    ctx.close()
    ref = from_workload(w).run(w.p0, w.F, 8, scheme)
    assert metrics.rel_l2(ref, p) <= FP64_TOL, st
    assert st["mass_defect"] < 1e-9, st
    assert min(x.min() for x in p) >= 1.0 - 1e-9 and max(x.max() for x in p) <= 1.2 + 1e-9


@pytest.mark.parametrize("precision", [1, 2])
def test_precision_form_with_wells(mc, precision):
    w = mi.paper_wells(3, n=66)
    ctx = mc.Context.from_workload(w, opts=opts(mc, precision, rtol=1e-12))
    ctx.step("D", 6)
    p = ctx.get_state()
    ctx.close()
    ref = from_workload(w).run(w.p0, w.F, 6, "D")
    assert metrics.rel_l2(ref, p) <= MIXED_TOL


def test_batch_with_wells(mc):
    ws = [mi.paper_wells(2, n=48), mi.paper_wells(3, n=40), mi.fracture_instance(4101, n=40, L=2)]
    o = opts(mc, 1)
    ctxs = [mc.Context.from_workload(w, opts=o) for w in ws]
    b = mc.Batch(ctxs, o)
    b.step("D", 4)
    for w, c in zip(ws, ctxs):
        ref = from_workload(w).run(w.p0, w.F, 4, "D")
        assert metrics.rel_l2(ref, c.get_state()) <= MIXED_TOL, w.name
    b.close()
    for c in ctxs:
        c.close()


def test_remove_wells_and_change_precision(mc):
    """Wells removed through W = NULL: the run matches the oracle without
    wells; wells set again between FP32 steps are seen by the FP32 copies."""
    w = mi.paper_wells(2, n=40)
    wells = w.wells
    ctx = mc.Context.from_workload(w, opts=opts(mc))
    ctx.set_well(1, None, None)
    ctx.step("D", 3)
    w.wells = {}
    ref = from_workload(w).run(w.p0, w.F, 3, "D")
    assert metrics.rel_l2(ref, ctx.get_state()) <= FP64_TOL
    ctx.set_opts(opts(mc, 1))
    ctx.step("D", 1)  # FP32 copies made without wells
    W, pw = wells[1]
    ctx.set_well(1, W, pw)
    ctx.set_state(w.p0)
    ctx.step("D", 3)
    w.wells = wells
    ref = from_workload(w).run(w.p0, w.F, 3, "D")
    assert metrics.rel_l2(ref, ctx.get_state()) <= MIXED_TOL
    ctx.close()


def test_well_arguments(mc):
    w = mi.paper_wells(2, n=32)
    ctx = mc.Context.from_workload(w)
    W, pw = w.wells[1]
    bad = np.array(W, copy=True)
    bad[3, 3] = -1.0
    with pytest.raises(mc.MCError):
        ctx.set_well(1, bad, pw)
    with pytest.raises(mc.MCError):
        ctx.set_well(2, W, pw)
    ctx.close()


def test_well_toggle_reuses_buffers(mc):
    """Removing and re-adding a well reuses the context's well buffers, and
    the re-enabled well acts as before."""
    w = mi.paper_wells(2, n=32)
    ctx = mc.Context.from_workload(w)
    W, pw = w.wells[1]
    b0 = ctx.device_bytes()
    for _ in range(3):
        ctx.set_well(1, None, None)
        ctx.set_well(1, W, pw)
    assert ctx.device_bytes() == b0
    ctx.step("D", 3)
    ref = from_workload(w).run(w.p0, w.F, 3, "D")
    assert metrics.rel_l2(ref, ctx.get_state()) <= 1e-10
    ctx.close()
