"""molt_step on non-uniform axes against the FP64 oracle's time integrators
with the same nodes (the ``grids`` of ``oracle.schemes``): the wave
leapfrog in mixed precision (2-D with a periodic and a Dirichlet
non-uniform axis; 3-D with a strided Dirichlet z axis), the SSP-RK3 heat
step in FP64 and mixed precision, the advection-diffusion step (Burgers
and linear flux) and the Hamilton-Jacobi step (forward Euler with WENO-Z,
SSP-RK3 with the linear rule; lagged adaptive dt) on stretched periodic
axes."""
import numpy as np
import pytest

from oracle import schemes
from paper_2007_03041_gb300 import molt as M
from paper_2007_03041_gb300 import workloads
from tests.gpu_util import assert_parity, max_for, need_gpu, state_dtype, to_dev, tol_for

pytestmark = pytest.mark.gpu


def _nodes(n, L, amp=0.3):
    xi = L * np.arange(n) / n
    return xi + amp * (L / (2 * np.pi)) * np.sin(2 * np.pi * xi / L)


def _dir_nodes(n, L, amp=0.3):
    t = np.linspace(0.0, 1.0, n)
    x = L * (t + amp * np.sin(2 * np.pi * t) / (2 * np.pi))
    x[0], x[-1] = 0.0, L
    return x


def _zero_dirichlet_faces(u, np_axes):
    for ax in np_axes:
        idx = [slice(None)] * u.ndim
        idx[ax] = 0
        u[tuple(idx)] = 0.0
        idx[ax] = -1
        u[tuple(idx)] = 0.0
    return u


def _bump(shape, seed):
    """Smooth data plus a little noise (every mode of the short lines)."""
    g = np.meshgrid(*[np.linspace(0, 1, n) for n in shape], indexing="ij")
    r2 = sum((gi - 0.45) ** 2 for gi in g)
    return np.exp(-r2 / 0.05) + 0.02 * workloads.rng(seed).standard_normal(shape)


@pytest.mark.parametrize("prec", [M.PREC_F32_F64UPDATE, M.PREC_F64])
def test_wave_2d_periodic_and_dirichlet_nonuniform_axes(prec):
    need_gpu()
    import torch
    nx, ny, L = 64, 48, 1.0
    xs, ys = _nodes(nx, L), _dir_nodes(ny, L, amp=0.4)
    h = L / nx
    dt = 2 * h
    u0 = _zero_dirichlet_faces(_bump((ny, nx), 3), [0])
    d = M.make_desc((nx, ny), bc=[M.BC_PERIODIC, M.BC_DIRICHLET], lo=[0, 0], hi=[L, L], P=2, quad_points=6,
                    beta=0.8, pde=M.PDE_WAVE, c=1.0, dt=dt, prec=prec)
    steps = 6
    ctx = M.molt_create(d)
    try:
        M.molt_set_grid_axis(ctx, 0, 0, xs)
        M.molt_set_grid_axis(ctx, 0, 1, ys)
        u = to_dev(u0, torch.float64)
        up = torch.zeros_like(u)
        t = M.molt_step(ctx, u, up, nsteps=steps, t=[0.0])
        got = u.cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    grids = ((ys, None), (xs, L))
    bc = ["dirichlet", "periodic"]
    prev, cur = None, u0
    for k in range(steps):
        nxt = schemes.wave_step(cur, prev, [h, h], dt, 1.0, 0.8, bc, 6, 2, from_rest=(k == 0), grids=grids)
        prev, cur = cur, nxt
    assert abs(t[0] - steps * dt) < 1e-12
    for ax in (0, 1):
        assert_parity(got, cur, tol_for(prec), max_for(prec), line_axis=ax, what="wave 2-D")


def test_wave_3d_with_a_strided_dirichlet_nonuniform_axis():
    need_gpu()
    import torch
    nx, ny, nz, L = 24, 20, 28, 1.0
    zs = _dir_nodes(nz, L)
    h = L / nx
    dt = 2 * h
    u0 = _zero_dirichlet_faces(_bump((nz, ny, nx), 4), [0])
    d = M.make_desc((nx, ny, nz), bc=[M.BC_PERIODIC, M.BC_PERIODIC, M.BC_DIRICHLET], lo=[0] * 3, hi=[L] * 3, P=2,
                    quad_points=6, beta=0.8, pde=M.PDE_WAVE, c=1.0, dt=dt, prec=M.PREC_F32_F64UPDATE)
    steps = 4
    ctx = M.molt_create(d)
    try:
        M.molt_set_grid_axis(ctx, 0, 2, zs)
        u = to_dev(u0, torch.float64)
        up = torch.zeros_like(u)
        M.molt_step(ctx, u, up, nsteps=steps, t=[0.0])
        got = u.cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    grids = ((zs, None), None, None)
    bc = ["dirichlet", "periodic", "periodic"]
    prev, cur = None, u0
    for k in range(steps):
        nxt = schemes.wave_step(cur, prev, [L / (nz - 1), L / ny, L / nx], dt, 1.0, 0.8, bc, 6, 2,
                                from_rest=(k == 0), grids=grids)
        prev, cur = cur, nxt
    assert_parity(got, cur, tol_for(M.PREC_F32_F64UPDATE), max_for(M.PREC_F32_F64UPDATE), line_axis=0,
                  what="wave 3-D")


@pytest.mark.parametrize("prec", [M.PREC_F64, M.PREC_F32_F64UPDATE])
def test_heat_rk3_on_a_dirichlet_nonuniform_axis(prec):
    need_gpu()
    import torch
    nx, ny, L = 72, 40, 1.0
    xs = _dir_nodes(nx, L, amp=0.4)
    hy = L / ny
    dt = 0.5 * hy * hy * 4
    u0 = _zero_dirichlet_faces(_bump((ny, nx), 5), [1])
    d = M.make_desc((nx, ny), bc=[M.BC_DIRICHLET, M.BC_PERIODIC], lo=[0, 0], hi=[L, L], P=3, quad_points=6,
                    beta=0.6, pde=M.PDE_HEAT, diffusivity=1.0, dt=dt, prec=prec)
    steps = 3
    ctx = M.molt_create(d)
    try:
        M.molt_set_grid_axis(ctx, 0, 0, xs)
        u = to_dev(u0, torch.float64)
        M.molt_step(ctx, u, None, nsteps=steps, t=[0.0])
        got = u.cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    want = u0
    for _ in range(steps):
        want = schemes.heat_step(want, [hy, L / (nx - 1)], dt, 1.0, 0.6, ["periodic", "dirichlet"], 6, 3,
                                 grids=(None, (xs, None)))
    for ax in (0, 1):
        assert_parity(got, want, tol_for(prec), max_for(prec), line_axis=ax, what="heat")


@pytest.mark.parametrize("case", [("burgers", True, 3, M.PREC_F64), ("linear", False, 1, M.PREC_F32),
                                  ("burgers", True, 2, M.PREC_F32_F64UPDATE)])
def test_advection_diffusion_on_stretched_periodic_axes(case):
    need_gpu()
    kind, rk3, P, prec = case
    nx, ny, L = 80, 48, 2 * np.pi
    xs, ys = _nodes(nx, L), _nodes(ny, L, amp=0.4)
    hx = L / nx
    c, kappa, beta = 1.6, 0.02, 0.6
    dt = 0.5 * hx / c
    vel = (0.7, -0.4)
    u0 = 1.0 + 0.4 * np.sin(ys)[:, None] * np.cos(xs)[None, :] + 0.02 * workloads.rng(6).standard_normal((ny, nx))
    if prec == M.PREC_F32:
        u0 = u0.astype(np.float32).astype(np.float64)
    d = M.make_desc((nx, ny), lo=[0, 0], hi=[L, L], P=P, quad_points=6, beta=beta, pde=M.PDE_ADVDIFF, c=c,
                    diffusivity=kappa, dt=dt, prec=prec, velocity=vel,
                    flux=M.FLUX_BURGERS if kind == "burgers" else M.FLUX_LINEAR,
                    integrator=M.INT_DEFAULT if rk3 else M.INT_EULER)
    steps = 3
    ctx = M.molt_create(d)
    try:
        M.molt_set_grid_axis(ctx, 0, 0, xs)
        M.molt_set_grid_axis(ctx, 0, 1, ys)
        u = to_dev(u0, state_dtype(prec))
        M.molt_step(ctx, u, None, nsteps=steps, t=[0.0])
        got = u.double().cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    want = u0
    for _ in range(steps):
        want = schemes.advdiff_step(want, [L / ny, hx], dt, kind, vel[::-1], c, kappa, beta, 6, P, rk3,
                                    grids=((ys, L), (xs, L)))
    for ax in (0, 1):
        assert_parity(got, want, tol_for(prec), max_for(prec), line_axis=ax, what="advection-diffusion")


def _min_cell(x, L):
    """The smallest cell of a periodic axis (the wrap cell included)."""
    return float(min(np.diff(x).min(), L - (x[-1] - x[0])))


@pytest.mark.parametrize("case", [("wenoz", M.PREC_F32, M.INT_EULER), ("wenoz", M.PREC_F64, M.INT_EULER),
                                  ("linear", M.PREC_F64, M.INT_RK3)])
def test_hamilton_jacobi_on_stretched_periodic_axes(case):
    """H = |grad u|^2/2 with lagged adaptive dt on a stretched grid: the step
    runs from the one-sided sums of both axes (the non-uniform sweep) and the
    pointwise stage kernel; alpha and dt take each axis's smallest cell, as
    the oracle does.  Forward Euler (P = 1) and SSP-RK3 (P = 2)."""
    need_gpu()
    import torch
    weights, prec, integ = case
    nx, ny, L = 96, 80, 2 * np.pi
    xs, ys = _nodes(nx, L), _nodes(ny, L, amp=0.4)
    u0 = (-np.cos(ys)[:, None] - np.cos(xs)[None, :] + 1e-3 * workloads.rng(8).standard_normal((ny, nx)))
    if prec == M.PREC_F32:
        u0 = u0.astype(np.float32).astype(np.float64)
    rk3 = integ == M.INT_RK3
    P = 2 if rk3 else 1
    npts = 5 if weights == "wenoz" else 6
    d = M.make_desc((nx, ny), lo=[0, 0], hi=[L, L], P=P, quad_points=npts,
                    weights=M.W_WENOZ if weights == "wenoz" else M.W_LINEAR, beta=1.0 if not rk3 else 0.3,
                    pde=M.PDE_HJ, cfl=1.5 if not rk3 else 0.5, dt=0.0, prec=prec, integrator=integ)
    steps = 3
    ctx = M.molt_create(d)
    try:
        M.molt_set_grid_axis(ctx, 0, 0, xs)
        M.molt_set_grid_axis(ctx, 0, 1, ys)
        u = to_dev(u0, state_dtype(prec))
        t = M.molt_step(ctx, u, None, nsteps=steps, t=[0.0])
        got = u.double().cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    grids = ((ys, L), (xs, L))
    dxs = [_min_cell(ys, L), _min_cell(xs, L)]
    cfl, beta = (0.5, 0.3) if rk3 else (1.5, 1.0)
    uu, tt = u0, 0.0
    if rk3:
        sp = schemes.hj_initial_speeds_P(uu, dxs, cfl, beta, npts, weights, P, grids=grids)
        for _ in range(steps):
            uu, dt, sp = schemes.hj_step_rk3(uu, dxs, sp, tt, cfl, beta, npts, weights, P, grids=grids)
            tt += dt
    else:
        sp = schemes.hj_initial_speeds(uu, dxs, cfl, beta, npts, weights, grids=grids)
        for _ in range(steps):
            uu, dt, sp = schemes.hj_step(uu, dxs, sp, cfl, beta, npts, weights, grids=grids)
            tt += dt
    for ax in (0, 1):
        assert_parity(got, uu, tol_for(prec), max_for(prec), line_axis=ax, what="HJ %s" % str(case))
    assert abs(t[0] - tt) < (1e-12 if prec == M.PREC_F64 else 1e-5) * tt
