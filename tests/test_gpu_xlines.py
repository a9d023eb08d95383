"""GPU parity of the warp-per-line FP32 x sweeps (csrc/sweep_xlines.cuh)
against the FP64 oracle, on the shapes the line-per-lane tiles do not take:
several lines per warp (lines of 16..256 points, 32/S lines to a warp), one
line per warp with idle lanes (S not a power of two), line counts that fill
no whole warp or tile, in place, decays whose boundary constants reach every
segment (nu = 0.05 on short lines: the segments near both ends of a line are
the same ones), and the zero of D on constants.  Element by element and at
the line ends (Sec. 2.1-2.4)."""
import numpy as np
import pytest

from oracle import sweep
from paper_2007_03041_gb300 import molt as M
from tests.gpu_util import need_gpu, to_dev, assert_parity, TOL_F32, MAX_F32

pytestmark = pytest.mark.gpu

BCS = {M.BC_PERIODIC: "periodic", M.BC_DIRICHLET: "dirichlet"}
OPS = {M.OP_L: "L", M.OP_R: "R", M.OP_0: "0"}


def _apply_x(u, op, P, alpha, bc, npts, inplace=False, lanes=2):
    """S_P along x through molt_apply_D (FP32 state); returns (result, number
    of warp-per-line launches)."""
    import torch
    d = M.make_desc(tuple(reversed(u.shape)), bc=[bc] * 3, P=P, quad_points=npts, prec=M.PREC_F32)
    ctx = M.molt_create(d)
    try:
        M.molt_set_option(ctx, M.OPT_LANES, lanes)
        M.molt_set_option(ctx, M.OPT_PROFILE, 1)
        x = to_dev(u, torch.float32)
        out = x if inplace else torch.empty_like(x)
        M.molt_apply_D(ctx, 0, 0, op, P, alpha, x, out)
        torch.cuda.synchronize()
        _, nx = M.molt_profile_read(ctx, M.KERNEL_XLINES_STORE)
        return out.double().cpu().numpy(), nx
    finally:
        M.molt_destroy(ctx)


def _case(shape, seed):
    g = np.random.default_rng(seed)
    n = shape[-1]
    u = 0.5 * g.standard_normal(shape) + np.sin(2 * np.pi * 3 * np.arange(n) / n)
    return u.astype(np.float32).astype(np.float64)


def _check(u, op, P, nu, bc, npts, inplace=False, what=""):
    n = u.shape[-1]
    N = n if bc == M.BC_PERIODIC else n - 1
    h = 1.0 / N
    alpha = nu / h
    got, nx = _apply_x(u, op, P, alpha, bc, npts, inplace=inplace)
    assert nx == 1, (what, nx)
    want = sweep.partial_sum(u, 2, alpha, h, OPS[op], BCS[bc], npts, P)
    assert_parity(got, want, TOL_F32, MAX_F32, line_axis=2, what=what)


@pytest.mark.parametrize("bc", [M.BC_PERIODIC, M.BC_DIRICHLET])
@pytest.mark.parametrize("op", [M.OP_0, M.OP_R, M.OP_L])
def test_xlines_packed_lines_match_oracle(bc, op):
    """Lines of 16..256 points, 32/S of them to a warp, 21 lines (the last
    warp's group is partly empty)."""
    need_gpu()
    for n, npts, P, nu in ((16, 6, 2, 0.4), (32, 5, 1, 0.4), (64, 6, 2, 0.05), (128, 3, 2, 0.4), (256, 6, 1, 1.3)):
        u = _case((3, 7, n), seed=n + op)
        _check(u, op, P, nu, bc, npts, what="n %d npts %d P %d nu %g" % (n, npts, P, nu))


@pytest.mark.parametrize("bc", [M.BC_PERIODIC, M.BC_DIRICHLET])
def test_xlines_one_line_per_warp_with_idle_lanes(bc):
    """S = 3, 5, 31 segments: one line to a warp, lanes S..31 idle; 6 lines."""
    need_gpu()
    for n, P, nu in ((48, 2, 0.4), (80, 1, 0.05), (496, 2, 0.4)):
        u = _case((2, 3, n), seed=n)
        _check(u, M.OP_0, P, nu, bc, 6, what="n %d P %d nu %g" % (n, P, nu))


def test_xlines_constants_reach_every_segment():
    """nu = 0.05 on 32- and 48-point lines: the boundary constants reach
    every segment, and the lanes near one end are near the other too (both
    constants on one lane)."""
    need_gpu()
    for n in (32, 48):
        for bc in (M.BC_PERIODIC, M.BC_DIRICHLET):
            u = _case((2, 3, n), seed=5 * n + bc)
            _check(u, M.OP_0, 2, 0.05, bc, 6, what="n %d bc %d" % (n, bc))


def test_xlines_in_place_ragged_and_constants():
    need_gpu()
    for n in (64, 512):
        u = _case((1, 37, n), seed=11)
        _check(u, M.OP_0, 2, 0.4, M.BC_PERIODIC, 6, inplace=True, what="in place n %d" % n)
        # D of a constant is zero exactly in the difference form
        got, _ = _apply_x(np.full((1, 37, n), -0.75), M.OP_0, 2, 0.4 * n, M.BC_PERIODIC, 6)
        assert np.abs(got).max() == 0.0
