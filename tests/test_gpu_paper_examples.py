"""GPU parity for the test problems of Sec. 5.1 (P = 1, 6-point linear
quadrature, first order in time): the Hamilton-Jacobi step with the linear
(Example 1) and (h0 + a.grad u)^2/2 (Example 3) Hamiltonians and a source
term, and the forward-Euler heat step (Example 2) -- against the FP64 oracle
step by step on small ragged and exact-fit grids, and at the paper's 5277^2
grid against the closed-form discrete solutions, the exact solutions and the
L-infinity errors the paper prints."""
import math
import os
import pathlib

import numpy as np
import pytest

from oracle import schemes, stability
from paper_2007_03041_gb300 import molt as M
from paper_2007_03041_gb300 import workloads
from tests.gpu_util import TOL_F32, TOL_F64, need_gpu, rel_l2, state_dtype, to_dev, tol_for, assert_grid_parity

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.txt")
ORACLE_H = {M.H_HALF_SQ: schemes.H_HALF_SQ, M.H_LINEAR: schemes.H_LINEAR, M.H_AFFINE_SQ: schemes.H_AFFINE_SQ}


def _paper_numbers():
    out = {}
    for line in pathlib.Path(GOLDEN).read_text().splitlines():
        line = line.split("#")[0].split()
        if len(line) == 2:
            out[line[0]] = float(line[1])
    return out


def _smooth(nx, ny, seed):
    g = workloads.rng(seed)
    x = 2 * np.pi * np.arange(nx) / nx
    y = 2 * np.pi * np.arange(ny) / ny
    a = g.uniform(-1, 1, 4)
    return (a[0] * np.sin(x + a[1])[None, :] * np.cos(2 * y + a[2])[:, None] + 0.3 * a[3] * np.cos(3 * x)[None, :]
            + 0.2 * np.sin(y)[:, None])


def _hj_desc(shape, ham, vel, h0, prec, cfl=1.0):
    nd = len(shape)
    return M.make_desc(shape, lo=[0.0] * nd, hi=[2 * np.pi] * nd, P=1, quad_points=6, weights=M.W_LINEAR, beta=1.0,
                       pde=M.PDE_HJ, cfl=cfl, dt=0.0, prec=prec, hamiltonian=ham, velocity=vel, h0=h0)


HJ_CASES = [(M.H_LINEAR, (1.0, 1.0), 0.0, False), (M.H_LINEAR, (-1.0, 0.5), 0.0, True),
            (M.H_AFFINE_SQ, (1.0, 1.0), 1.0, True), (M.H_AFFINE_SQ, (-0.7, 0.3), -0.4, False),
            (M.H_HALF_SQ, (0.0, 0.0), 0.0, True)]


@pytest.mark.parametrize("prec", [M.PREC_F64, M.PREC_F32])
@pytest.mark.parametrize("shape", [(96, 80), (128, 64), (300, 1)])
@pytest.mark.parametrize("ham,vel,h0,with_source", HJ_CASES)
def test_hj_hamiltonians_and_source_match_oracle(ham, vel, h0, with_source, shape, prec):
    need_gpu()
    import torch
    nx, ny = shape
    dims = (nx,) if ny == 1 else (nx, ny)
    u0 = _smooth(nx, ny, 11)
    src = np.stack([_smooth(nx, ny, 12 + k) for k in range(3)]) if with_source else None
    if ny == 1:
        u0 = u0[0]
        src = src[:, 0] if src is not None else None
        vel = vel[:1]
    dt_ = state_dtype(prec)
    if prec == M.PREC_F32:
        u0 = u0.astype(np.float32).astype(np.float64)
        src = src.astype(np.float32).astype(np.float64) if src is not None else None
    ctx = M.molt_create(_hj_desc(dims, ham, vel, h0, prec))
    steps = 3
    try:
        if src is not None:
            M.molt_set_source(ctx, 0, to_dev(src, dt_))
        u = to_dev(u0, dt_)
        got, ts = [], []
        t = [0.25]
        for _ in range(steps):
            t = M.molt_step(ctx, u, None, nsteps=1, t=t)
            got.append(u.double().cpu().numpy())
            ts.append(t[0])
    finally:
        M.molt_destroy(ctx)
    hs = [2 * np.pi / n for n in dims][::-1]          # numpy axis order
    kw = dict(cfl=1.0, beta=1.0, npts=6, weights="linear", hamiltonian=ORACLE_H[ham], a=tuple(vel)[::-1], h0=h0)
    uu = u0
    sp = schemes.hj_initial_speeds(uu, hs, **kw)
    tt = 0.25
    for k in range(steps):
        uu, dt, sp = schemes.hj_step(uu, hs, sp, source=src, t=tt, **kw)
        tt += dt
        assert_grid_parity(got[k], uu, tol_for(prec), what=str(k))
        assert abs(ts[k] - tt) < (1e-10 if prec == M.PREC_F64 else 1e-5) * tt, k


@pytest.mark.parametrize("prec", [M.PREC_F64, M.PREC_F32_F64UPDATE])
@pytest.mark.parametrize("shape,P,npts", [((96, 80), 1, 6), ((128, 64), 2, 3), ((200,), 1, 6)])
def test_heat_forward_euler_matches_oracle(shape, P, npts, prec):
    need_gpu()
    import torch
    nx = shape[0]
    ny = shape[1] if len(shape) > 1 else 1
    u0 = _smooth(nx, ny, 21)
    if ny == 1:
        u0 = u0[0]
    h = 2 * np.pi / nx
    nd = len(shape)
    d = M.make_desc(shape, lo=[0.0] * nd, hi=[2 * np.pi] * nd, P=P, quad_points=npts, beta=1.0, pde=M.PDE_HEAT,
                    dt=h, prec=prec, integrator=M.INT_EULER)
    ctx = M.molt_create(d)
    try:
        u = to_dev(u0, torch.float64)
        M.molt_step(ctx, u, None, nsteps=3, t=[0.0])
        got = u.cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    hs = [2 * np.pi / n for n in shape][::-1]
    uu = u0
    for _ in range(3):
        uu = schemes.heat_euler_step(uu, hs, h, beta=1.0, npts=npts, P=P)
    assert_grid_parity(got, uu, tol_for(prec))


def test_invalid_hamiltonian_integrator_and_source_are_rejected():
    need_gpu()
    import torch
    with pytest.raises(M.MoltError):
        M.molt_create(_hj_desc((64, 64), 7, (1.0, 1.0), 0.0, M.PREC_F64))
    bad = M.make_desc((64, 64, 64), P=2, pde=M.PDE_WAVE, dt=0.01, prec=M.PREC_F64, integrator=M.INT_EULER)
    with pytest.raises(M.MoltError):
        M.molt_create(bad)
    heat = M.make_desc((64, 64), P=1, pde=M.PDE_HEAT, dt=0.01, prec=M.PREC_F64)
    ctx = M.molt_create(heat)
    try:
        with pytest.raises(M.MoltError):
            M.molt_set_source(ctx, 0, torch.zeros((1, 64, 64), dtype=torch.float64, device="cuda"))
    finally:
        M.molt_destroy(ctx)
    ctx = M.molt_create(_hj_desc((64, 64), M.H_AFFINE_SQ, (1.0, 1.0), 1.0, M.PREC_F64))
    try:
        with pytest.raises(M.MoltError):
            M.molt_set_source(ctx, 0, torch.zeros((6, 64, 64), dtype=torch.float64, device="cuda"))
        M.molt_set_source(ctx, 0, None)
    finally:
        M.molt_destroy(ctx)


# ---------------------------------------------------------------- 5277^2

N_PAPER = 5277


def _sample(n, count, seed):
    g = workloads.rng(seed)
    pts = g.integers(0, n, size=(count, 2))
    pts[:2] = [[0, 0], [n - 1, n - 1]]
    return pts[:, 0], pts[:, 1]


def _advection_modes_at(n, steps, iy, ix):
    """Closed-form discrete solution of Example 1 (a = (1, 1), CFL 1, beta 1)
    at the points (iy, ix): each mode of u0 times G^steps, G = 1 - (d_R(th_x) + d_R(th_y))."""
    h = 2 * math.pi / n
    modes = {(0, 0): 0.25, (1, 0): -0.125, (-1, 0): -0.125, (0, 1): -0.125, (0, -1): -0.125,
             (1, 1): 1 / 16, (1, -1): 1 / 16, (-1, 1): 1 / 16, (-1, -1): 1 / 16}
    out = np.zeros(len(ix), dtype=complex)
    for (kx, ky), am in modes.items():
        G = 1 - ((1 - stability.symbol(kx * h, 1.0, "R", 6)) + (1 - stability.symbol(ky * h, 1.0, "R", 6)))
        out += am * G ** steps * np.exp(1j * (kx * ix + ky * iy) * h)
    return out.real


@pytest.mark.slow
def test_example1_advection_5277():
    need_gpu()
    import torch
    n = N_PAPER
    ctx = M.molt_create(_hj_desc((n, n), M.H_LINEAR, (1.0, 1.0), 0.0, M.PREC_F64))
    try:
        u = torch.tensor(workloads.advection_initial(n), device="cuda")
        t = M.molt_step(ctx, u, None, nsteps=n, t=[0.0])
        exact = torch.tensor(workloads.advection_solution(n, t[0]), device="cuda")
        linf = float((u - exact).abs().max())
        iy, ix = _sample(n, 256, 31)
        got = u[torch.tensor(iy, device="cuda"), torch.tensor(ix, device="cuda")].cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    assert abs(t[0] - 2 * math.pi) < 1e-9
    np.testing.assert_allclose(got, _advection_modes_at(n, n, iy, ix), rtol=0, atol=1e-10)
    ref = _paper_numbers()["linf_5277_advection"]
    assert ref / 1.5 < linf < ref * 1.5, linf


@pytest.mark.slow
def test_example2_diffusion_5277():
    need_gpu()
    import torch
    n = N_PAPER
    h = 2 * math.pi / n
    steps = round(1.0 / h)
    d = M.make_desc((n, n), lo=[0, 0], hi=[2 * math.pi] * 2, P=1, quad_points=6, beta=1.0, pde=M.PDE_HEAT,
                    dt=h, prec=M.PREC_F64, integrator=M.INT_EULER)
    ctx = M.molt_create(d)
    try:
        u = torch.tensor(workloads.diffusion_initial(n), device="cuda")
        M.molt_step(ctx, u, None, nsteps=steps, t=[0.0])
        u0 = torch.tensor(workloads.diffusion_initial(n), device="cuda")
        nu = h / math.sqrt(h)
        G = 1 - stability.partial_sum_symbol(h, nu, "0", 6, 1).real
        closed = float((u - G ** steps * u0).abs().max())
        linf = float((u - math.exp(-steps * h) * u0).abs().max())
    finally:
        M.molt_destroy(ctx)
    assert closed < 1e-11
    ref = _paper_numbers()["linf_5277_diffusion"]
    assert ref / 1.5 < linf < ref * 1.5, linf


def _manufactured_run(n, T, prec=M.PREC_F64):
    import torch
    ctx = M.molt_create(_hj_desc((n, n), M.H_AFFINE_SQ, (1.0, 1.0), 1.0, prec))
    try:
        M.molt_set_source(ctx, 0, torch.tensor(workloads.manufactured_hj_source(n), device="cuda",
                                               dtype=state_dtype(prec)))
        u = torch.zeros((n, n), dtype=state_dtype(prec), device="cuda")
        t = [0.0]
        steps = 0
        while t[0] < T:
            t = M.molt_step(ctx, u, None, nsteps=1, t=t)
            steps += 1
        exact = torch.tensor(workloads.manufactured_hj_solution(n, t[0]), device="cuda")
        linf = float((u.double() - exact).abs().max())
        return u.double().cpu().numpy(), t[0], steps, linf
    finally:
        M.molt_destroy(ctx)


@pytest.mark.slow
def test_example3_manufactured_hj_matches_oracle_and_converges():
    need_gpu()
    # the whole run against the oracle at 256^2 (about 40 lagged steps)
    n = 256
    u, t, steps, _ = _manufactured_run(n, 0.5)
    h = 2 * math.pi / n
    kw = dict(cfl=1.0, npts=6, weights="linear", hamiltonian=schemes.H_AFFINE_SQ, a=(1.0, 1.0), h0=1.0)
    F = workloads.manufactured_hj_source(n)
    uu = np.zeros((n, n))
    sp = schemes.hj_initial_speeds(uu, [h, h], **kw)
    tt = 0.0
    for _ in range(steps):
        uu, dt, sp = schemes.hj_step(uu, [h, h], sp, source=F, t=tt, **kw)
        tt += dt
    assert abs(t - tt) < 1e-10 * tt
    assert_grid_parity(u, uu, 1e-11)
    # first-order convergence in the grid
    errs = [_manufactured_run(m, 0.5)[3] for m in (512, 1024, 2048)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(0.85 < r < 1.3 for r in rates), (errs, rates)


@pytest.mark.slow
def test_example3_manufactured_hj_5277():
    need_gpu()
    _, t, _, linf = _manufactured_run(N_PAPER, 0.5)
    assert 0.5 <= t < 0.51
    ref = _paper_numbers()["linf_5277_hj"]
    assert ref / 2 < linf < ref * 2, linf


@pytest.mark.parametrize("prec", [M.PREC_F32, M.PREC_F32_F64UPDATE])
@pytest.mark.parametrize("npts", [3, 5, 6])
def test_fp32_sweeps_keep_constants_in_the_kernel_of_D(npts, prec):
    """sum_l c_l = 1 - q (App. C moments) makes D[const] = 0.  The FP32
    sweeps run their recurrences with q rounded to FP32; their weights and
    boundary constants are fitted to that q, so D[const] stays at the FP32
    rounding floor of the sweep (measured up to 9.5e-7 relative, about 16
    ulps, from the local sums and carries) for small nu as well; with the
    weights rounded one by one it would be off by (q - q32)/(1 - q) on top,
    up to 3e-6 at nu = 0.01."""
    need_gpu()
    import torch
    n = 1000
    h = 1.0 / n
    worst = 0.0
    for nu in (0.01, 0.013, 0.02, 0.031, 0.047, 0.07, 0.11, 0.3):
        for bc in (M.BC_PERIODIC, M.BC_DIRICHLET):
            d = M.make_desc((n,), bc=[bc], quad_points=npts, prec=prec)
            hh = 1.0 / (n if bc == M.BC_PERIODIC else n - 1)
            ctx = M.molt_create(d)
            try:
                dt_ = state_dtype(prec)
                x = torch.full((n,), 0.75, dtype=dt_, device="cuda")
                out = torch.empty_like(x)
                M.molt_apply_D(ctx, 0, 0, M.OP_0 if bc == M.BC_DIRICHLET else M.OP_R, 1, nu / hh, x, out)
                o = out.double().cpu().numpy()
            finally:
                M.molt_destroy(ctx)
            # constants: J = (1 - q) v, I_R = (1 - q^i) v, and the periodic
            # closure or the Dirichlet solve (A = B = v/2) give L^{-1} v = v
            worst = max(worst, float(np.abs(o).max()) / 0.75)
    assert worst < 1.5e-6, worst


RK3_CASES = [(M.H_LINEAR, (1.0, -0.5), 0.0, False, 3, M.W_LINEAR, 6), (M.H_AFFINE_SQ, (1.0, 1.0), 1.0, True, 3, M.W_LINEAR, 6),
             (M.H_HALF_SQ, (0.0, 0.0), 0.0, False, 2, M.W_WENOZ, 5)]


@pytest.mark.parametrize("prec", [M.PREC_F64, M.PREC_F32])
@pytest.mark.parametrize("shape", [(96, 80), (128, 1)])
@pytest.mark.parametrize("ham,vel,h0,with_source,P,weights,npts", RK3_CASES)
def test_hj_rk3_matches_oracle(ham, vel, h0, with_source, P, weights, npts, shape, prec):
    """SSP-RK3 with P-term one-sided sums (Sec. 2.5) against the oracle, step by step."""
    need_gpu()
    import torch
    nx, ny = shape
    dims = (nx,) if ny == 1 else (nx, ny)
    u0 = _smooth(nx, ny, 13)
    src = np.stack([_smooth(nx, ny, 22 + k) for k in range(3)]) if with_source else None
    if ny == 1:
        u0 = u0[0]
        src = src[:, 0] if src is not None else None
        vel = vel[:1]
    dt_ = state_dtype(prec)
    if prec == M.PREC_F32:
        u0 = u0.astype(np.float32).astype(np.float64)
        src = src.astype(np.float32).astype(np.float64) if src is not None else None
    nd = len(dims)
    d = M.make_desc(dims, lo=[0.0] * nd, hi=[2 * np.pi] * nd, P=P, quad_points=npts, weights=weights, beta=0.3,
                    pde=M.PDE_HJ, cfl=1.0, dt=0.0, prec=prec, hamiltonian=ham, velocity=vel, h0=h0,
                    integrator=M.INT_RK3)
    ctx = M.molt_create(d)
    steps = 3
    try:
        if src is not None:
            M.molt_set_source(ctx, 0, to_dev(src, dt_))
        u = to_dev(u0, dt_)
        got, ts = [], []
        t = [0.1]
        for _ in range(steps):
            t = M.molt_step(ctx, u, None, nsteps=1, t=t)
            got.append(u.double().cpu().numpy())
            ts.append(t[0])
    finally:
        M.molt_destroy(ctx)
    hs = [2 * np.pi / n for n in dims][::-1]
    wname = "wenoz" if weights == M.W_WENOZ else "linear"
    kw = dict(cfl=1.0, beta=0.3, npts=npts, weights=wname, P=P, hamiltonian=ORACLE_H[ham], a=tuple(vel)[::-1], h0=h0)
    uu = u0
    sp = schemes.hj_initial_speeds_P(uu, hs, **kw)
    tt = 0.1
    for k in range(steps):
        uu, dt, sp = schemes.hj_step_rk3(uu, hs, sp, t=tt, source=src, **kw)
        tt += dt
        assert_grid_parity(got[k], uu, tol_for(prec), what=str(k))
        assert abs(ts[k] - tt) < (1e-10 if prec == M.PREC_F64 else 1e-5) * tt, k
