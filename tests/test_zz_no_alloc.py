"""The allocation-free wave step, molt_wave_step_noalloc.

Callers that cannot call cudaMalloc (a fixed device-memory budget, a
framework allocator that owns the device's memory, latency-critical code)
advance a wave problem with it; its scratch is a static device array of the
library that every call shares.  Each case runs two calls in a row (start
from rest, then a leapfrog step written over u^{n-1}, the usual rotation) and
checks both results against the FP64 oracle and against molt_step on the
same inputs, in 1-D, 2-D and 3-D, on periodic and Dirichlet axes.  A NaN in
u must come back as MOLT_ENONFINITE, and the scratch limit and the aliasing
rule are enforced.  This file is collected last so that a run stopping at
its first failure has run every other test first."""
import numpy as np
import pytest

from oracle import schemes
from paper_2007_03041_gb300 import molt as M
from paper_2007_03041_gb300 import workloads
from tests.gpu_util import need_gpu, to_dev, assert_parity, TOL_F32, MAX_F32

pytestmark = pytest.mark.gpu

BC = {M.BC_PERIODIC: "periodic", M.BC_DIRICHLET: "dirichlet"}


def _problem(ndim, bc, n):
    """Descriptor and initial state: [0,1]^ndim, n points per axis, P = 2,
    6-point rule, dt = 2h (x first in the descriptor, C order in the array)."""
    h = 1.0 / (n if bc == M.BC_PERIODIC else n - 1)
    d = M.make_desc((n,) * ndim, bc=[bc] * ndim, P=2, quad_points=6, beta=0.8, pde=M.PDE_WAVE, c=1.0, dt=2 * h,
                    prec=M.PREC_F32_F64UPDATE)
    g = np.random.default_rng(11 + ndim)
    if ndim == 3:
        u0 = workloads.wave_bumps(n)
    else:
        x = np.arange(n) * h
        u0 = np.sin(2 * np.pi * x)
        if ndim == 2:
            u0 = np.add.outer(np.cos(2 * np.pi * x), u0)
        u0 = u0 + 0.05 * g.standard_normal(u0.shape)
    if bc == M.BC_DIRICHLET:
        for ax in range(ndim):
            idx = [slice(None)] * ndim
            idx[ax] = 0
            u0[tuple(idx)] = 0.0
            idx[ax] = n - 1
            u0[tuple(idx)] = 0.0
    return d, h, np.ascontiguousarray(u0)


@pytest.mark.parametrize("ndim,n", [(1, 300), (2, 70), (3, 40)])
@pytest.mark.parametrize("bc", [M.BC_PERIODIC, M.BC_DIRICHLET])
def test_noalloc_two_calls_match_oracle_and_molt_step(ndim, n, bc):
    import torch
    need_gpu()
    d, h, u0 = _problem(ndim, bc, n)
    dt = 2 * h
    # oracle: the Taylor start, then one leapfrog step
    bcs = [BC[bc]] * ndim
    w1 = schemes.wave_step(u0, None, [h] * ndim, dt, 1.0, 0.8, bcs, 6, 2, from_rest=True)
    w2 = schemes.wave_step(w1, u0, [h] * ndim, dt, 1.0, 0.8, bcs, 6, 2)
    # existing entry point: two steps from rest
    ctx = M.molt_create(d)
    try:
        u = to_dev(u0, torch.float64)
        up = torch.zeros_like(u)
        t = M.molt_step(ctx, u, up, nsteps=1, t=[0.0])
        ref1 = u.cpu().numpy()
        M.molt_step(ctx, u, up, nsteps=1, t=t)
        ref2 = u.cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    # allocation-free entry point, two calls in a row; the second writes
    # u^{n+1} over u^{n-1}
    a = to_dev(u0, torch.float64)
    b = torch.empty_like(a)
    M.molt_wave_step_noalloc(d, a, None, b, from_rest=1)
    torch.cuda.synchronize()
    got1 = b.cpu().numpy()
    M.molt_wave_step_noalloc(d, b, a, a, from_rest=0)
    torch.cuda.synchronize()
    got2 = a.cpu().numpy()
    for got, want, ref, what in ((got1, w1, ref1, "first call"), (got2, w2, ref2, "second call")):
        for ax in range(ndim):
            assert_parity(got, want, TOL_F32, MAX_F32, line_axis=ax, what="%s vs oracle" % what)
        assert_parity(got, ref, TOL_F32, MAX_F32, what="%s vs molt_step" % what)


def test_noalloc_reports_non_finite_values():
    import torch
    need_gpu()
    d, h, u0 = _problem(2, M.BC_PERIODIC, 64)
    u0[10, 20] = np.nan
    a = to_dev(u0, torch.float64)
    b = torch.empty_like(a)
    with pytest.raises(M.MoltError) as ei:
        M.molt_wave_step_noalloc(d, a, None, b, from_rest=1)
    assert ei.value.status == M.MOLT_ENONFINITE
    # the next call starts from a cleared status word
    d, h, u0 = _problem(2, M.BC_PERIODIC, 64)
    a = to_dev(u0, torch.float64)
    M.molt_wave_step_noalloc(d, a, None, b, from_rest=1)
    torch.cuda.synchronize()
    assert np.isfinite(b.cpu().numpy()).all()


def test_noalloc_rejects_grids_beyond_the_scratch_and_u_next_aliasing_u():
    import torch
    need_gpu()
    d = _problem(3, M.BC_DIRICHLET, 128)[0]          # 2,097,152 points > 1,048,576
    x, y, z = (torch.zeros(8, dtype=torch.float64, device="cuda") for _ in range(3))
    with pytest.raises(M.MoltError) as ei:
        M.molt_wave_step_noalloc(d, x, y, z, from_rest=0)
    assert ei.value.status == M.MOLT_EINVAL
    d = _problem(1, M.BC_PERIODIC, 64)[0]
    u = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MoltError) as ei:
        M.molt_wave_step_noalloc(d, u, None, u, from_rest=1)
    assert ei.value.status == M.MOLT_EINVAL
