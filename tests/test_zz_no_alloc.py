"""The allocation-free single-continuum entry point (mc_step_single_noalloc).

It serves callers that may not allocate device memory (a framework's caching
allocator owns the pool, a fixed memory budget, or a loop where cudaMalloc's
implicit synchronisation is unacceptable): they pass their own input and
output buffers and the solver keeps its scratch in a fixed array inside the
library. Here its result must match the context-based entry point
(mc_setup + mc_step_decoupled with one continuum) within the FP64 parity
tolerance, on two calls in a row (the second starts from the first's output
and must not be disturbed by what the first left in the shared array).

This file is collected last so that a run stopping at the first failure has
run every other test before it.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


def _problem(nx, ny, seed):
    rng = np.random.default_rng(seed)
    k = 100.0 * np.exp(rng.standard_normal((ny, nx)))
    F = np.zeros((ny, nx))
    F[ny // 8, nx // 8] = 1.0
    F[(7 * ny) // 8, (7 * nx) // 8] = -1.0
    return k, F


def test_noalloc_matches_context_entry_point_on_two_calls():
    import torch

    import paper_2209_01158_gb300 as mc
    nx, ny, c, tau, nsteps = 150, 100, 0.3, 0.01, 3
    k, F = _problem(nx, ny, 7)
    dev = torch.device("cuda", 0)
    k_d = torch.tensor(k.ravel(), dtype=torch.float64, device=dev)
    F_d = torch.tensor(F.ravel(), dtype=torch.float64, device=dev)
    p_d = torch.zeros(nx * ny, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    ctx = mc.Context(nx, ny, [k.ravel()], [c], None, None, tau)
    ctx.set_source(0, F.ravel())
    ctx.set_state([np.zeros(nx * ny)])
    for call in range(2):
        st = mc.mc_step_single_noalloc(nx, ny, k_d, c, tau, F_d, p_d, nsteps, rtol=1e-12,
                                       stream=stream)
        assert st["steps_done"] == nsteps
        ctx.step_decoupled("D", nsteps)
        ref = ctx.get_state()[0]
        got = p_d.cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= FP64_TOL, (call, err)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch

    import paper_2209_01158_gb300 as mc
    dev = torch.device("cuda", 0)
    nx, ny = 300, 300  # 304 * 300 pitched cells > 65536
    x = torch.zeros(nx * ny, dtype=torch.float64, device=dev)
    st = mc.mc_step_single_noalloc(nx, ny, x, 1.0, 0.1, x, x, 1, check=False)
    assert st["return"] == mc.N.MC_E_ARG
