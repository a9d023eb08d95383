"""GPU parity of the flux-split advection-diffusion step (Sec. 2.5) against
the FP64 oracle: linear and Burgers fluxes, forward Euler and SSP-RK3,
P = 1..3, linear and WENO-Z weights, FP64 / mixed / FP32, 1-D to 3-D
ragged and exact-fit grids; exact mass conservation; rejected setups."""
import math

import numpy as np
import pytest

from oracle import schemes
from paper_2007_03041_gb300 import molt as M
from paper_2007_03041_gb300 import workloads
from tests.gpu_util import need_gpu, rel_l2, state_dtype, to_dev, tol_for, assert_grid_parity

pytestmark = pytest.mark.gpu


def _field(shape_np, seed):
    g = workloads.rng(seed)
    out = 0.3 * np.ones(shape_np)
    for ax, n in enumerate(shape_np):
        x = 2 * np.pi * np.arange(n) / n
        sh = [1] * len(shape_np)
        sh[ax] = n
        out = out + g.uniform(0.2, 0.5) * np.sin(x + g.uniform(0, 6)).reshape(sh)
    return out


CASES = [
    # numpy shape, flux, rk3, P, prec, weights, npts, kappa, beta, c
    ((80, 96), M.FLUX_LINEAR, False, 1, M.PREC_F64, M.W_LINEAR, 6, 0.05, 0.3, 1.0),
    ((64, 128), M.FLUX_LINEAR, True, 3, M.PREC_F64, M.W_LINEAR, 6, 0.05, 0.3, 1.0),
    ((80, 96), M.FLUX_BURGERS, False, 1, M.PREC_F32_F64UPDATE, M.W_LINEAR, 6, 0.02, 0.6, 1.6),
    ((64, 128), M.FLUX_BURGERS, True, 2, M.PREC_F32, M.W_LINEAR, 3, 0.0, 0.3, 1.6),
    ((300,), M.FLUX_BURGERS, False, 1, M.PREC_F32, M.W_WENOZ, 5, 0.01, 0.6, 1.6),
    ((64, 96), M.FLUX_BURGERS, True, 1, M.PREC_F64, M.W_WENOZ, 5, 0.01, 0.5, 1.6),
    ((20, 24, 28), M.FLUX_LINEAR, False, 1, M.PREC_F32_F64UPDATE, M.W_LINEAR, 6, 0.05, 0.3, 1.0),
]


@pytest.mark.parametrize("case", CASES, ids=[str(i) for i in range(len(CASES))])
def test_advdiff_steps_match_oracle(case):
    need_gpu()
    import torch
    shape, flux, rk3, P, prec, weights, npts, kappa, beta, c = case
    nd = len(shape)
    shape_xyz = tuple(reversed(shape))
    vel = (0.7, -0.4, 0.25)[:nd]
    hs_xyz = [2 * np.pi / n for n in shape_xyz]
    dt = 0.5 * min(hs_xyz) / c
    u0 = _field(shape, 40 + nd)
    if prec == M.PREC_F32:
        u0 = u0.astype(np.float32).astype(np.float64)
    d = M.make_desc(shape_xyz, lo=[0.0] * nd, hi=[2 * np.pi] * nd, P=P, quad_points=npts, weights=weights, beta=beta,
                    pde=M.PDE_ADVDIFF, c=c, diffusivity=kappa, dt=dt, prec=prec, velocity=vel, flux=flux,
                    integrator=M.INT_DEFAULT if rk3 else M.INT_EULER)
    ctx = M.molt_create(d)
    steps = 3
    try:
        u = to_dev(u0, state_dtype(prec))
        t = M.molt_step(ctx, u, None, nsteps=steps, t=[0.0])
        got = u.double().cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    kind = schemes.FLUX_BURGERS if flux == M.FLUX_BURGERS else schemes.FLUX_LINEAR
    wname = "wenoz" if weights == M.W_WENOZ else "linear"
    want = u0
    for _ in range(steps):
        want = schemes.advdiff_step(want, hs_xyz[::-1], dt, kind, vel[::-1], c, kappa, beta, npts, P, rk3, wname)
    assert_grid_parity(got, want, tol_for(prec), what=str(case))
    assert abs(t[0] - steps * dt) < 1e-12


def test_burgers_conserves_mass_on_the_gpu():
    need_gpu()
    import torch
    n = 256
    h = 2 * np.pi / n
    u0 = _field((n, n), 7)
    d = M.make_desc((n, n), lo=[0, 0], hi=[2 * np.pi] * 2, P=1, quad_points=6, beta=0.6, pde=M.PDE_ADVDIFF, c=1.6,
                    diffusivity=0.01, dt=0.5 * h / 1.6, prec=M.PREC_F64, flux=M.FLUX_BURGERS,
                    integrator=M.INT_EULER)
    ctx = M.molt_create(d)
    try:
        u = to_dev(u0, torch.float64)
        M.molt_step(ctx, u, None, nsteps=20, t=[0.0])
        m = float(u.sum())
    finally:
        M.molt_destroy(ctx)
    assert abs(m - u0.sum()) < 1e-11 * np.abs(u0).sum()


def test_advdiff_rejects_unsupported_setups():
    need_gpu()
    base = dict(P=1, pde=M.PDE_ADVDIFF, dt=0.01, prec=M.PREC_F64, flux=M.FLUX_BURGERS)
    for kw in (dict(c=1.0, bc=[M.BC_DIRICHLET] * 2), dict(c=0.0), dict(c=1.0, diffusivity=-1.0),
               dict(c=1.0, weights=M.W_WENOZ, quad_points=5, prec=M.PREC_F32_F64UPDATE)):
        args = dict(base)
        args.update(kw)
        with pytest.raises(M.MoltError):
            M.molt_create(M.make_desc((64, 64), **args))
