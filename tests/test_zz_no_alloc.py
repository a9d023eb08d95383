"""The allocation-free wave step (molt_wave_step_noalloc), for callers that
cannot call cudaMalloc, against the context-based molt_step on the same
inputs, on two calls in a row (the shared static scratch is reused).  This
file is collected last so that a run stopping at its first failure has run
every other test first."""
import numpy as np
import pytest

from paper_2007_03041_gb300 import molt as M
from paper_2007_03041_gb300 import workloads
from tests.gpu_util import need_gpu, rel_l2, to_dev, TOL_F32

pytestmark = pytest.mark.gpu


def _desc(n):
    h = 1.0 / (n - 1)
    return M.make_desc((n, n, n), bc=[M.BC_DIRICHLET] * 3, P=2, quad_points=6, beta=0.8, pde=M.PDE_WAVE, c=1.0,
                       dt=2 * h, prec=M.PREC_F32_F64UPDATE)


def test_noalloc_wave_step_matches_molt_step_twice():
    import torch
    need_gpu()
    n = 48
    d = _desc(n)
    u0 = to_dev(workloads.wave_bumps(n), torch.float64)
    # existing entry point: two steps from rest
    ctx = M.molt_create(d)
    try:
        u = u0.clone()
        up = torch.zeros_like(u)
        t = M.molt_step(ctx, u, up, nsteps=1, t=[0.0])
        ref1 = u.clone()
        M.molt_step(ctx, u, up, nsteps=1, t=t)
        ref2 = u.clone()
    finally:
        M.molt_destroy(ctx)
    # allocation-free entry point, two calls in a row
    out1 = torch.empty_like(u0)
    M.molt_wave_step_noalloc(d, u0, None, out1, from_rest=1)
    out2 = torch.empty_like(u0)
    M.molt_wave_step_noalloc(d, out1, u0, out2, from_rest=0)
    torch.cuda.synchronize()
    assert rel_l2(out1.cpu().numpy(), ref1.cpu().numpy()) < TOL_F32
    assert rel_l2(out2.cpu().numpy(), ref2.cpu().numpy()) < TOL_F32


def test_noalloc_rejects_grids_beyond_the_scratch():
    import torch
    need_gpu()
    d = _desc(128)          # 2,097,152 points > 1,048,576
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MoltError) as ei:
        M.molt_wave_step_noalloc(d, x, x, x, from_rest=0)
    assert ei.value.status == M.MOLT_EINVAL
