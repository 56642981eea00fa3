"""The seeded workload recipes hold the structure their docstrings state
(no method arithmetic is involved: these are checks of the inputs)."""

import numpy as np
import pytest

import mc_inputs as mi


@pytest.mark.parametrize("L", [2, 3])
def test_paper_wells_recipe(L):
    n = 200
    w = mi.paper_wells(L, n=n)
    assert (w.nx, w.ny, w.L, w.nsteps) == (n, n, L, 50)
    assert abs(w.tau - 0.002 / 50) < 1e-18
    assert all(np.all(p == 1.0) for p in w.p0) and all(np.all(f == 0.0) for f in w.F)
    frac = w.k[L - 1] > 1.0
    assert np.all(w.k[L - 1][frac] == 1e6) and np.all(w.k[L - 1][~frac] == 1e-2)
    assert list(w.wells) == [L - 1]
    W, pw = w.wells[L - 1]
    assert np.all(pw == 1.2)
    assert np.all(W[W > 0] == 1e5 / n ** 2)
    assert np.all(frac[W > 0])              # wells sit on fracture cells
    c = (np.arange(n) + 0.5) / n
    jj, ii = np.nonzero(W > 0)
    in_a = (c[ii] >= 0.1) & (c[ii] <= 0.15) & (c[jj] >= 0.1) & (c[jj] <= 0.15)
    in_b = (c[ii] >= 0.6) & (c[ii] <= 0.65) & (c[jj] >= 0.85) & (c[jj] <= 0.9)
    near = ~(in_a | in_b)
    # a well outside both boxes only where a box holds no fracture cell
    assert near.sum() <= 2
    exp_c = [0.1, 1.0] if L == 2 else [0.05, 0.1, 1.0]
    assert np.allclose(w.c, exp_c)
    # the same seed gives the same workload
    w2 = mi.paper_wells(L, n=n)
    assert all(np.array_equal(a, b) for a, b in zip(w.k, w2.k))
