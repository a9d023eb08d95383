"""GPU parity of the persistent TMA-fed sweep kernel (exact-fit lines whose
arrays meet the tensor-copy alignment rules) against the oracle, and against
the plain one-tile-per-CTA kernel on the same inputs."""
import numpy as np
import pytest

from oracle import schemes, sweep
from paper_2007_03041_gb300 import molt as M
from paper_2007_03041_gb300 import workloads
from tests.gpu_util import need_gpu, rel_l2, np_axis, to_dev, tol_for, state_dtype, assert_grid_parity

pytestmark = pytest.mark.gpu

OPS = {M.OP_L: "L", M.OP_R: "R", M.OP_0: "0"}
BCS = {M.BC_PERIODIC: "periodic", M.BC_DIRICHLET: "dirichlet"}


def apply_both(shape_np, axis, op, P, nu, bc, npts, prec, weights=M.W_LINEAR):
    import torch
    need_gpu()
    ndim = len(shape_np)
    shape_xyz = tuple(reversed(shape_np))
    d = M.make_desc(shape_xyz, bc=[bc] * ndim, P=P, quad_points=npts, weights=weights, prec=prec)
    g = np.random.default_rng(21)
    u = g.standard_normal(shape_np)
    n_ax = shape_xyz[axis]
    N = n_ax if bc == M.BC_PERIODIC else n_ax - 1
    h = 1.0 / N
    alpha = nu / h
    outs = []
    ctx = M.molt_create(d)
    try:
        uin = to_dev(u, state_dtype(prec))
        for tma in (1, 0):
            M.molt_set_option(ctx, M.OPT_TMA, tma)
            out = torch.empty_like(uin)
            M.molt_apply_D(ctx, 0, axis, op, P, alpha, uin, out)
            torch.cuda.synchronize()
            outs.append(out.double().cpu().numpy())
    finally:
        M.molt_destroy(ctx)
    u_in = u.astype(np.float32).astype(np.float64) if prec == M.PREC_F32 else u
    wname = "wenoz" if weights == M.W_WENOZ else "linear"
    want = sweep.partial_sum(u_in, np_axis(ndim, axis), alpha, h, OPS[op], BCS[bc], npts, P, wname)
    return outs[0], outs[1], want


CASES = [((512, 16, 32), 2), ((32, 512, 16), 1), ((4, 8, 1024), 0), ((16, 512), 1), ((8, 512), 0)]


@pytest.mark.parametrize("prec", [M.PREC_F32, M.PREC_F32_F64UPDATE, M.PREC_F64])
@pytest.mark.parametrize("bc", [M.BC_PERIODIC, M.BC_DIRICHLET])
def test_tma_sweep_matches_oracle_and_plain(prec, bc):
    for shape, axis in CASES:
        tma, plain, want = apply_both(shape, axis, M.OP_0, 2, 0.4, bc, 6, prec)
        assert_grid_parity(tma, want, tol_for(prec), what=str((shape, axis)))
        assert_grid_parity(plain, want, tol_for(prec), what=str((shape, axis)))
        assert_grid_parity(tma, plain, 1e-13 * (1 if prec == M.PREC_F64 else 1e6), what=str((shape, axis)))


# Long strided lines whose tiles hold fewer than 16 bytes of lines (one or two
# FP32 lines, one FP64 line): the TMA box is widened to a 16-byte-aligned
# column group and the tile's lines are picked out of it.
LONG = [((4096, 1280), 1, M.PREC_F32), ((8192, 40), 1, M.PREC_F32), ((4096, 2, 640), 2, M.PREC_F32),
        ((8192, 10), 1, M.PREC_F64)]


@pytest.mark.parametrize("shape,axis,prec", LONG)
def test_tma_long_strided_lines_with_narrow_tiles(shape, axis, prec):
    tma, plain, want = apply_both(shape, axis, M.OP_0, 1, 0.5, M.BC_PERIODIC, 6, prec)
    assert_grid_parity(tma, want, tol_for(prec))
    assert_grid_parity(plain, want, tol_for(prec))
    assert_grid_parity(tma, plain, 1e-13 * (1 if prec == M.PREC_F64 else 1e6))


@pytest.mark.parametrize("op", [M.OP_L, M.OP_R])
def test_tma_wenoz_one_sided(op):
    tma, plain, want = apply_both((64, 512), 0, op, 1, 2.0 / 3.0, M.BC_PERIODIC, 5, M.PREC_F32, M.W_WENOZ)
    assert_grid_parity(tma, want, 1e-5)
    assert_grid_parity(plain, want, 1e-5)


def test_wave_step_anisotropic_uses_tma_on_long_axis():
    import torch
    need_gpu()
    nz, ny, nx = 512, 16, 16
    hs = [1.0 / (nx - 1), 1.0 / (ny - 1), 1.0 / (nz - 1)]
    dt = 2 * min(hs)
    u0 = workloads.random_lines((nz, ny, nx), seed=3)
    workloads.zero_boundary(u0)
    d = M.make_desc((nx, ny, nz), bc=[M.BC_DIRICHLET] * 3, P=2, quad_points=6, beta=0.8, pde=M.PDE_WAVE,
                    c=1.0, dt=dt, prec=M.PREC_F32_F64UPDATE)
    ctx = M.molt_create(d)
    try:
        u = to_dev(u0, torch.float64)
        up = torch.zeros_like(u)
        M.molt_step(ctx, u, up, nsteps=3, t=[0.0])
        got = u.cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    # numpy axis order (z, y, x) -> spacings (hz, hy, hx)
    dxs = [hs[2], hs[1], hs[0]]
    prev, cur = None, u0
    for k in range(3):
        nxt = schemes.wave_step(cur, prev, dxs, dt, 1.0, 0.8, ["dirichlet"] * 3, 6, 2, from_rest=(k == 0))
        prev, cur = cur, nxt
    assert_grid_parity(got, cur, 1e-5)


def test_hj_512_tma_matches_oracle():
    import torch
    need_gpu()
    n = 512
    h = 2 * np.pi / n
    u0 = workloads.hj_initial(n)
    d = M.make_desc((n, n), lo=[0, 0], hi=[2 * np.pi] * 2, P=1, quad_points=5, weights=M.W_WENOZ, beta=1.0,
                    pde=M.PDE_HJ, cfl=1.5, prec=M.PREC_F32)
    ctx = M.molt_create(d)
    try:
        u = to_dev(u0, torch.float32)
        t = M.molt_step(ctx, u, None, nsteps=3, t=[0.0])
        got = u.double().cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    uu = u0.astype(np.float32).astype(np.float64)
    speeds = schemes.hj_initial_speeds(uu, [h, h])
    tt = 0.0
    for _ in range(3):
        uu, dtk, speeds = schemes.hj_step(uu, [h, h], speeds)
        tt += dtk
    assert_grid_parity(got, uu, 1e-5)
    assert abs(t[0] - tt) < 1e-4 * tt


def test_heat_mixed_512_tma_matches_oracle():
    import torch
    need_gpu()
    n = 512
    h = 1.0 / n
    dt = h / 2
    u0 = workloads.heat_modes(n)
    d = M.make_desc((n, n), P=3, quad_points=3, beta=0.6, pde=M.PDE_HEAT, dt=dt, prec=M.PREC_F32_F64UPDATE)
    ctx = M.molt_create(d)
    try:
        u = to_dev(u0, torch.float64)
        M.molt_step(ctx, u, None, nsteps=2, t=[0.0])
        got = u.cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    want = u0
    for _ in range(2):
        want = schemes.heat_step(want, [h, h], dt, 1.0, 0.6, None, 3, 3)
    assert_grid_parity(got, want, 1e-5)
