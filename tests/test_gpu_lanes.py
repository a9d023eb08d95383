"""GPU parity of the line-per-lane FP32 sweeps (one lane per line, one warp
per 16-point segment, difference form of the recurrences) and of the
warp-per-line x sweeps (one lane per 16-point segment) against the FP64
oracle: every axis, both boundary types, the three operators, the 3/5/6-point
rules, P = 1 and 2, lines of 16 to 512 points, decays with a short look-back
(nu = 0.4: terms below 2^-40 dropped after 5 segments) and without truncation
(nu = 0.05: every segment), element by element and at the line ends."""
import numpy as np
import pytest

from oracle import sweep, schemes
from paper_2007_03041_gb300 import molt as M
from paper_2007_03041_gb300 import workloads
from tests.gpu_util import need_gpu, np_axis, to_dev, assert_parity, TOL_F32, MAX_F32

pytestmark = pytest.mark.gpu

BCS = {M.BC_PERIODIC: "periodic", M.BC_DIRICHLET: "dirichlet"}
OPS = {M.OP_L: "L", M.OP_R: "R", M.OP_0: "0"}


def _shape_for(axis, n):
    """numpy shape (z, y, x) whose lines along `axis` have n points and fill
    whole 32-line tiles."""
    return {0: (4, 8, n), 1: (3, n, 32), 2: (n, 2, 64)}[axis]


def _apply(u, axis, op, P, alpha, bc, npts, lanes, inplace=False, lanes_launches=None, xlines=1):
    """S_P along `axis` through molt_apply_D (FP32 state); appends to
    `lanes_launches` how many (line-per-lane, warp-per-line) launches ran."""
    import torch
    shape_xyz = tuple(reversed(u.shape))
    d = M.make_desc(shape_xyz, bc=[bc] * 3, P=P, quad_points=npts, prec=M.PREC_F32)
    ctx = M.molt_create(d)
    try:
        M.molt_set_option(ctx, M.OPT_LANES, lanes)
        M.molt_set_option(ctx, M.OPT_XLINES, xlines)
        M.molt_set_option(ctx, M.OPT_PROFILE, 1)
        x = to_dev(u, torch.float32)
        out = x if inplace else torch.empty_like(x)
        M.molt_apply_D(ctx, 0, axis, op, P, alpha, x, out)
        torch.cuda.synchronize()
        _, nl = M.molt_profile_read(ctx, M.KERNEL_LANES_STORE)
        _, nx = M.molt_profile_read(ctx, M.KERNEL_XLINES_STORE)
        if lanes_launches is not None:
            lanes_launches.append((nl, nx))
        return out.double().cpu().numpy()
    finally:
        M.molt_destroy(ctx)


def _case(axis, n, bc, seed):
    g = np.random.default_rng(seed)
    u = g.standard_normal(_shape_for(axis, n))
    # a smooth part as well: D of smooth data is small, the relative bound tighter
    x = np.arange(n) / n
    sh = [1, 1, 1]
    sh[np_axis(3, axis)] = n
    u = 0.5 * u + np.sin(2 * np.pi * 3 * x).reshape(sh)
    return u.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("bc", [M.BC_PERIODIC, M.BC_DIRICHLET])
@pytest.mark.parametrize("op", [M.OP_0, M.OP_R, M.OP_L])
def test_lanes_apply_D_matches_oracle(axis, bc, op):
    need_gpu()
    for n, npts, P, nu in ((512, 6, 2, 0.4), (512, 3, 1, 0.05), (48, 5, 2, 0.4), (16, 6, 1, 1.3), (128, 6, 2, 0.05)):
        u = _case(axis, n, bc, seed=n + axis)
        N = n if bc == M.BC_PERIODIC else n - 1
        h = 1.0 / N
        alpha = nu / h
        want = sweep.partial_sum(u, np_axis(3, axis), alpha, h, OPS[op], BCS[bc], npts, P)
        # x lines: the warp-per-line kernel and the line-per-lane tiles
        for xl in ((1, 0) if axis == 0 else (1,)):
            got = _apply(u, axis, op, P, alpha, bc, npts, lanes=2, xlines=xl)
            assert_parity(got, want, TOL_F32, MAX_F32, line_axis=np_axis(3, axis),
                          what="axis %d n %d npts %d P %d nu %g xlines %d" % (axis, n, npts, P, nu, xl))


def test_lanes_kernel_runs_and_agrees_with_the_scan_kernel():
    """The auto choice takes the warp-per-line kernel for x lines and the
    line-per-lane kernel for y and z lines at nu = 0.4 (the line-per-lane
    tiles for x lines too with MOLT_OPT_XLINES off, the scan kernel with
    MOLT_OPT_LANES off); all agree to FP32 rounding."""
    need_gpu()
    n = 512
    for axis in (0, 1, 2):
        u = _case(axis, n, M.BC_DIRICHLET, seed=7 + axis)
        alpha = 0.4 * (n - 1)
        la, lb, lc = [], [], []
        a = _apply(u, axis, M.OP_0, 2, alpha, M.BC_DIRICHLET, 6, lanes=1, lanes_launches=la)
        b = _apply(u, axis, M.OP_0, 2, alpha, M.BC_DIRICHLET, 6, lanes=0, lanes_launches=lb)
        c = _apply(u, axis, M.OP_0, 2, alpha, M.BC_DIRICHLET, 6, lanes=1, lanes_launches=lc, xlines=0)
        assert la == [(0, 1) if axis == 0 else (1, 0)] and lb == [(0, 0)] and lc == [(1, 0)], (axis, la, lb, lc)
        assert_parity(a, b, 2e-6, 1e-5, line_axis=np_axis(3, axis), what="lanes vs scan axis %d" % axis)
        assert_parity(c, b, 2e-6, 1e-5, line_axis=np_axis(3, axis), what="tiles vs scan axis %d" % axis)


def test_lanes_in_place_and_constants():
    need_gpu()
    n = 256
    for axis in (0, 1, 2):
        u = _case(axis, n, M.BC_PERIODIC, seed=3)
        alpha = 0.4 * n
        got = _apply(u, axis, M.OP_0, 2, alpha, M.BC_PERIODIC, 6, lanes=2, inplace=True)
        want = sweep.partial_sum(u, np_axis(3, axis), alpha, 1.0 / n, "0", "periodic", 6, 2)
        assert_parity(got, want, TOL_F32, MAX_F32, line_axis=np_axis(3, axis), what="in place axis %d" % axis)
        # D of a constant is zero exactly in the difference form
        c = np.full(_shape_for(axis, n), 1.25)
        got = _apply(c, axis, M.OP_0, 2, alpha, M.BC_PERIODIC, 6, lanes=2)
        assert np.abs(got).max() == 0.0


@pytest.mark.parametrize("n", [64, 96])
def test_wave_step_on_lanes_kernels_matches_oracle(n):
    """3-D wave, Dirichlet, FP32 sweeps + FP64 update, P = 2, dt = 2h
    (nu = 0.4): every sweep takes the line-per-lane kernel; 10 steps (from
    rest, then leapfrog, ending on the in-place variant that keeps u the
    newest state) against the oracle, element by element and at the line
    ends."""
    need_gpu()
    import torch
    h = 1.0 / (n - 1)
    dt = 2 * h
    u0 = workloads.wave_bumps(n)
    d = M.make_desc((n, n, n), bc=[M.BC_DIRICHLET] * 3, P=2, quad_points=6, beta=0.8, pde=M.PDE_WAVE,
                    c=1.0, dt=dt, prec=M.PREC_F32_F64UPDATE)
    ctx = M.molt_create(d)
    try:
        u = to_dev(u0, torch.float64)
        up = torch.zeros_like(u)
        M.molt_set_option(ctx, M.OPT_PROFILE, 1)
        M.molt_step(ctx, u, up, nsteps=1, t=[0.0])
        _, nset = M.molt_profile_read(ctx, M.KERNEL_XLINES_ACC_SET)
        _, nadd = M.molt_profile_read(ctx, M.KERNEL_LANES_ACC_ADD)
        _, nfin = M.molt_profile_read(ctx, M.KERNEL_LANES_WAVE_FINAL)
        _, nupd = M.molt_profile_read(ctx, M.KERNEL_UPDATE)
        M.molt_set_option(ctx, M.OPT_PROFILE, 0)
        # x on the warp-per-line kernel, y and z on the line-per-lane kernel,
        # then the FP64 update kernel
        assert (nset, nadd, nfin, nupd) == (1, 2, 0, 1), (nset, nadd, nfin, nupd)
        M.molt_step(ctx, u, up, nsteps=9, t=[dt])
        got, gotp = u.cpu().numpy(), up.cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    bc = ["dirichlet"] * 3
    prev, cur = None, u0
    for k in range(10):
        nxt = schemes.wave_step(cur, prev, [h] * 3, dt, 1.0, 0.8, bc, 6, 2, from_rest=(k == 0))
        prev, cur = cur, nxt
    for ax in range(3):
        assert_parity(got, cur, TOL_F32, MAX_F32, line_axis=ax, what="u^10 lines along numpy axis %d" % ax)
    assert_parity(gotp, prev, TOL_F32, MAX_F32, what="u^9")
