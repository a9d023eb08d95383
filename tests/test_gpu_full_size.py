"""Parity at the full workload sizes, in the launch configuration the bench
times (molt_step with the persistent TMA sweeps, the graph-captured batched
step), on outputs the oracle can compute one by one:

* 3-D wave 512^3 (Dirichlet, P=2, 6-point rule, mixed precision): the start
  step u^1 at sampled points from the three lines through each point, and
  the first leapfrog step u^2 at a few points from the lines of u^1 through
  them;
* 2-D heat 256^2 (FP64, P=3, 3-point rule, 10 and 100 steps) and the 64 batched
  heat problems of sides 128..2048: against the closed-form discrete
  solution (every Fourier mode of the initial state evolves by the RK3
  polynomial of its exact discrete symbol), which holds at any size;
* Hamilton-Jacobi 4096^2 (WENO-Z) and 8192^2 (learned weights with an
  input-independent network): the first step's increment at sampled points
  from the x and y lines through them, and the lagged time step bound.
"""
import math

import numpy as np
import pytest

from oracle import mlp, schemes, stability, sweep
from oracle.quadrature import QuadratureRule
from paper_2007_03041_gb300 import molt as M
from paper_2007_03041_gb300 import workloads
from tests.gpu_util import TOL_F32, TOL_F64, need_gpu, rel_l2, assert_grid_parity

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _rk3(z):
    return 1.0 + z + z * z / 2.0 + z ** 3 / 6.0


def _modal_heat(n, seed, nsteps, beta=0.6, npts=3, P=3, points=None):
    """Closed-form discrete solution of the periodic heat step (dt = h/2) at
    grid points (iy, ix): sum_m a_m R(z_m)^nsteps cos(theta_x ix + theta_y iy)."""
    k, a = workloads.heat_mode_params(seed)
    h = 1.0 / n
    nu = beta / math.sqrt(h / 2) * h
    iy, ix = points
    out = np.zeros(len(ix))
    for (kx, ky), am in zip(k, a):
        tx, ty = 2 * np.pi * kx / n, 2 * np.pi * ky / n
        z = -beta ** 2 * (stability.partial_sum_symbol(tx, nu, "0", npts, P).real
                          + stability.partial_sum_symbol(ty, nu, "0", npts, P).real)
        out += am * _rk3(z) ** nsteps * np.cos(tx * ix + ty * iy)
    return out


def _sample_points(n, count, seed):
    g = workloads.rng(seed)
    pts = g.integers(0, n, size=(count, 2))
    pts[:4] = [[0, 0], [n - 1, n - 1], [0, n - 1], [n - 1, 0]]
    return pts[:, 0], pts[:, 1]


def test_heat_256_fp64_matches_closed_form():
    """10 steps (the slowest mode keeps 2% of its amplitude): relative L2;
    100 steps (every mode has decayed to the FP64 rounding level of the
    initial amplitude): absolute, against the initial amplitude."""
    need_gpu()
    import torch
    n = 256
    d = M.make_desc((n, n), P=3, quad_points=3, beta=0.6, pde=M.PDE_HEAT, dt=0.5 / n, prec=M.PREC_F64)
    ctx = M.molt_create(d)
    try:
        u0 = workloads.heat_modes(n)
        u = torch.tensor(u0, dtype=torch.float64, device="cuda")
        t = M.molt_step(ctx, u, None, nsteps=10, t=[0.0])
        got10 = u.cpu().numpy()
        M.molt_step(ctx, u, None, nsteps=90, t=t)
        got100 = u.cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    iy, ix = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    pts = (iy.ravel(), ix.ravel())
    assert_grid_parity(got10, _modal_heat(n, workloads.SEED_HEAT, 10, points=pts).reshape(n, n), TOL_F64)
    want100 = _modal_heat(n, workloads.SEED_HEAT, 100, points=pts).reshape(n, n)
    assert np.abs(got100 - want100).max() < TOL_F64 * np.abs(u0).max()


def test_batched_64_full_sizes_match_closed_form():
    need_gpu()
    import torch
    sides = workloads.batched_sides()
    descs = [M.make_desc((n, n), P=3, quad_points=3, beta=0.6, pde=M.PDE_HEAT, dt=0.5 / n,
                         prec=M.PREC_F32_F64UPDATE) for n in sides]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = M.molt_create(descs, stream=s)
        try:
            us = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in workloads.batched_heat(sides=sides)]
            M.molt_step(ctx, us, None, nsteps=3, t=[0.0] * len(us))
            s.synchronize()
            shapes = [M.molt_batch_tile_shape(ctx, i, 0) for i in range(len(sides))]
            got = [x.cpu().numpy() for x in us]
        finally:
            M.molt_destroy(ctx)
    assert all(E in (4, 8, 16) for E, _, _ in shapes)    # the batched kernel ran
    for i, (n, g) in enumerate(zip(sides, got)):
        iy, ix = _sample_points(n, 512, 100 + i)
        want = _modal_heat(n, 3000 + i, 3, points=(iy, ix))
        assert_grid_parity(g[iy, ix], want, TOL_F32, what=str((i, n)), ends=False)


def _wave_lines(u, pts):
    """Lines through the points (k, j, i) of a [z][y][x] array, per axis."""
    k, j, i = pts
    return [u[k, j, :], u[k, :, i], u[:, j, i].T]


def _wave_S(lines, alpha, h):
    return [sweep.partial_sum(L, 1, alpha, h, "0", "dirichlet", 6, 2) for L in lines]


def test_wave_512_start_and_leapfrog_steps_at_sampled_points():
    need_gpu()
    import torch
    n, beta = 512, 0.8
    h = 1.0 / (n - 1)
    dt = 2 * h
    alpha = beta / dt
    u0 = workloads.wave_bumps(n)
    d = M.make_desc((n, n, n), bc=[M.BC_DIRICHLET] * 3, P=2, quad_points=6, beta=beta, pde=M.PDE_WAVE, c=1.0,
                    dt=dt, prec=M.PREC_F32_F64UPDATE)
    ctx = M.molt_create(d)
    try:
        u = torch.tensor(u0, device="cuda")
        up = torch.empty_like(u)
        t = M.molt_step(ctx, u, up, nsteps=1, t=[0.0])
        u1 = u.cpu().numpy()
        M.molt_step(ctx, u, up, nsteps=1, t=t)
        u2 = u.cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    # u^1 at sampled points: half near the bump centres, half anywhere
    g = workloads.rng(77)
    cen, _ = workloads.wave_bump_params()
    near = np.clip(np.round(cen[g.integers(0, len(cen), 96)] * (n - 1)).astype(int)
                   + g.integers(-6, 7, size=(96, 3)), 0, n - 1)
    anyw = g.integers(0, n, size=(96, 3))
    P3 = np.concatenate([near, anyw])
    pts = (P3[:, 2], P3[:, 1], P3[:, 0])            # (k, j, i) = (z, y, x)
    S = _wave_S(_wave_lines(u0, pts), alpha, h)
    k, j, i = pts
    idx = [i, j, k]
    want1 = u0[pts] - 0.5 * beta ** 2 * sum(S[a][np.arange(len(i)), idx[a]] for a in range(3))
    assert_grid_parity(u1[pts], want1, TOL_F32, ends=False)
    # u^2 at two points near bump centres: u^1 on the three lines through each
    # point from the lines of u^0 through every point of those lines
    for p in range(2):
        kk, jj, ii = k[p], j[p], i[p]
        lines1 = []
        for axis in range(3):
            if axis == 0:
                line_pts = (np.full(n, kk), np.full(n, jj), np.arange(n))
            elif axis == 1:
                line_pts = (np.full(n, kk), np.arange(n), np.full(n, ii))
            else:
                line_pts = (np.arange(n), np.full(n, jj), np.full(n, ii))
            Sl = _wave_S(_wave_lines(u0, line_pts), alpha, h)
            lk, lj, li = line_pts
            lidx = [li, lj, lk]
            lines1.append(u0[line_pts] - 0.5 * beta ** 2 * sum(Sl[a][np.arange(n), lidx[a]] for a in range(3)))
        S1 = [sweep.partial_sum(L[None, :], 1, alpha, h, "0", "dirichlet", 6, 2)[0] for L in lines1]
        want2 = 2 * lines1[0][ii] - u0[kk, jj, ii] - beta ** 2 * (S1[0][ii] + S1[1][jj] + S1[2][kk])
        scale = np.abs(u1).max()
        assert abs(u2[kk, jj, ii] - want2) < TOL_F32 * scale, (p, u2[kk, jj, ii], want2)
        np.testing.assert_allclose(u1[kk, jj, :], lines1[0], atol=TOL_F32 * scale)


def _hj_first_step(n, seed, weights, blob=None, fn=None, wname="wenoz", samples=384):
    import torch
    h = 2 * math.pi / n
    u0 = workloads.hj_initial(n, seed=seed).astype(np.float32)
    d = M.make_desc((n, n), lo=[0, 0], hi=[2 * math.pi] * 2, P=1, quad_points=5, weights=weights, beta=1.0,
                    pde=M.PDE_HJ, cfl=1.5, dt=0.0, prec=M.PREC_F32)
    ctx = M.molt_create(d)
    try:
        if blob is not None:
            M.molt_set_mlp(ctx, blob)
        u = torch.tensor(u0, device="cuda")
        t = M.molt_step(ctx, u, None, nsteps=1, t=[0.0])
        u1 = u.cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    dt = t[0]
    iy, ix = _sample_points(n, samples, 5)
    alpha = 1.0 / (1.5 * h)
    u064 = u0.astype(np.float64)
    ders = []
    for lines, pos in ((u064[iy, :], ix), (u064[:, ix].T, iy)):
        dm = alpha * sweep.partial_sum(lines, 1, alpha, h, "R", "periodic", 5, 1, wname, fn)
        dp = -alpha * sweep.partial_sum(lines, 1, alpha, h, "L", "periodic", 5, 1, wname, fn)
        r = np.arange(len(pos))
        ders.append((dm[r, pos], dp[r, pos]))
    Hh, speeds = schemes.hj_hamiltonian(ders)
    inc_gpu = u1[iy, ix].astype(np.float64) - u064[iy, ix]
    inc_want = -dt * Hh
    # the state is FP32 (rounding 6e-8 of |u| ~ 2, against increments ~1e-3)
    assert_grid_parity(inc_gpu, inc_want, 1e-3, ends=False)
    assert_grid_parity(u1[iy, ix], u064[iy, ix] + inc_want, TOL_F32, ends=False)
    # lagged time step of the first step: dt = CFL h / max over the grid of
    # the speeds of u^0 <= CFL h / (max over the samples)
    assert 0 < dt <= 1.5 * h / max(speeds) * (1 + 1e-6)


def test_hj_4096_wenoz_first_step_at_sampled_points():
    need_gpu()
    _hj_first_step(4096, workloads.SEED_HJ, M.W_WENOZ)


def test_hj_8192_learned_first_step_at_sampled_points():
    need_gpu()
    import torch
    nu = 1.0 / 1.5
    d = M.molt_weno_linear_weights(nu)
    theta = np.zeros(mlp.NPARAMS)
    P = mlp.unpack(theta)
    P["b3"] = np.log(np.asarray(d))
    theta = mlp.pack(P).astype(np.float32)
    th = torch.tensor(theta, device="cuda")
    blob = torch.empty(M.MLP_BLOB_BYTES, dtype=torch.uint8, device="cuda")
    M.molt_mlp_pack(th, blob)
    fn = mlp.learned_weight_fn(theta.astype(np.float64), QuadratureRule(nu, 5), emulate_bf16=True)
    _hj_first_step(8192, workloads.SEED_HJ_LARGE, M.W_LEARNED, blob, fn, "learned", samples=96)
