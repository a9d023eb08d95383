"""GPU parity of molt_apply_D (one sweep kernel launch) against the oracle:
S_P = sum_{p<=P} D_op^p along each axis, every boundary type, quadrature,
weight rule and precision, on ragged sizes that span several warps/tiles."""
import math

import numpy as np
import pytest

from oracle import sweep
from paper_2007_03041_gb300 import molt as M
from tests.gpu_util import assert_parity, max_for, need_gpu, rel_l2, np_axis, to_dev, tol_for, state_dtype

pytestmark = pytest.mark.gpu

BCS = {M.BC_PERIODIC: "periodic", M.BC_DIRICHLET: "dirichlet"}
OPS = {M.OP_L: "L", M.OP_R: "R", M.OP_0: "0"}


def run_apply(shape_np, axis, op, P, nu, bc, npts, prec, weights=M.W_LINEAR, seed=0, inplace=False):
    need_gpu()
    import torch
    ndim = len(shape_np)
    shape_xyz = tuple(reversed(shape_np))
    bcs = [bc] * ndim
    d = M.make_desc(shape_xyz, bc=bcs, P=P, quad_points=npts, weights=weights, prec=prec)
    g = np.random.default_rng(seed)
    u = g.standard_normal(shape_np)
    if weights != M.W_LINEAR:
        # smooth data plus noise: nonlinear weights away from their linear values
        x = np.linspace(0, 2 * np.pi, shape_np[-1], endpoint=False)
        u = np.sin(x) + 0.1 * u
    n_ax = shape_xyz[axis]
    N = n_ax if bc == M.BC_PERIODIC else n_ax - 1
    h = 1.0 / N
    alpha = nu / h
    ctx = M.molt_create(d)
    try:
        dt = state_dtype(prec)
        uin = to_dev(u, dt)
        out = uin if inplace else torch.empty_like(uin)
        M.molt_apply_D(ctx, 0, axis, op, P, alpha, uin, out)
        torch.cuda.synchronize()
        got = out.double().cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    wname = {M.W_LINEAR: "linear", M.W_WENOZ: "wenoz"}[weights]
    u_in = u.astype(np.float32).astype(np.float64) if prec == M.PREC_F32 else u
    want = sweep.partial_sum(u_in, np_axis(ndim, axis), alpha, h, OPS[op], BCS[bc], npts, P, wname)
    return got, want


def check(got, want, prec, ndim, axis, what):
    """Relative L2, max-abs and the first and last 4 points of every line
    along the swept axis."""
    assert_parity(got, want, tol_for(prec), max_for(prec), line_axis=np_axis(ndim, axis), what=str(what))


@pytest.mark.parametrize("prec", [M.PREC_F64, M.PREC_F32_F64UPDATE, M.PREC_F32])
@pytest.mark.parametrize("bc", [M.BC_PERIODIC, M.BC_DIRICHLET])
@pytest.mark.parametrize("op", [M.OP_L, M.OP_R, M.OP_0])
@pytest.mark.parametrize("npts", [3, 5, 6])
def test_lines_1d(prec, bc, op, npts):
    for n, P, nu in ((7, 1, 0.4), (100, 2, 0.05), (513, 3, 0.9), (1000, 2, 0.02), (2053, 1, 0.3)):
        got, want = run_apply((n,), 0, op, P, nu, bc, npts, prec, seed=n)
        check(got, want, prec, 1, 0, (n, P, nu))


@pytest.mark.parametrize("prec", [M.PREC_F64, M.PREC_F32_F64UPDATE])
@pytest.mark.parametrize("bc", [M.BC_PERIODIC, M.BC_DIRICHLET])
def test_every_axis_2d_3d(prec, bc):
    for shape in ((37, 53), (9, 10, 11), (20, 3, 600)):
        for axis in range(len(shape)):
            got, want = run_apply(shape, axis, M.OP_0, 2, 0.37, bc, 6, prec, seed=axis + 10)
            check(got, want, prec, len(shape), axis, (shape, axis))


@pytest.mark.parametrize("prec", [M.PREC_F64, M.PREC_F32])
@pytest.mark.parametrize("op", [M.OP_L, M.OP_R])
def test_wenoz_weights(prec, op):
    for shape, axis in (((300,), 0), ((24, 130), 1), ((24, 130), 0)):
        got, want = run_apply(shape, axis, op, 1, 2.0 / 3.0, M.BC_PERIODIC, 5, prec, weights=M.W_WENOZ)
        check(got, want, prec, len(shape), axis, (shape, axis))


def test_tiny_and_degenerate_lines():
    for n in (1, 2, 3, 4):
        got, want = run_apply((n,), 0, M.OP_0, 2, 0.5, M.BC_PERIODIC, 6, M.PREC_F64)
        assert rel_l2(got, want) < 1e-12 or np.abs(want).max() < 1e-14, n
    for n in (2, 3, 5):
        got, want = run_apply((n,), 0, M.OP_0, 2, 0.5, M.BC_DIRICHLET, 6, M.PREC_F64)
        assert np.abs(got - want).max() < 1e-12, n


def test_longest_line_and_in_place():
    got, want = run_apply((8192,), 0, M.OP_0, 1, 0.01, M.BC_PERIODIC, 3, M.PREC_F32_F64UPDATE)
    check(got, want, M.PREC_F32_F64UPDATE, 1, 0, "8192 points")
    got, want = run_apply((16, 300), 1, M.OP_0, 2, 0.2, M.BC_DIRICHLET, 6, M.PREC_F64, inplace=True)
    check(got, want, M.PREC_F64, 2, 1, "in place")


def test_errors_are_reported():
    need_gpu()
    import torch
    d = M.make_desc((10,), P=0)
    with pytest.raises(M.MoltError) as ei:
        M.molt_create(d)
    assert ei.value.status == M.MOLT_EINVAL
    d = M.make_desc((9000,), P=1)
    ctx = M.molt_create(d)
    try:
        x = torch.zeros(9000, dtype=torch.float64, device="cuda")
        with pytest.raises(M.MoltError) as ei:
            M.molt_apply_D(ctx, 0, 0, M.OP_0, 1, 10.0, x, x)
        assert ei.value.status == M.MOLT_EUNSUPPORTED
        with pytest.raises(M.MoltError) as ei:
            M.molt_apply_D(ctx, 0, 1, M.OP_0, 1, 10.0, x, x)
        assert ei.value.status == M.MOLT_EINVAL
    finally:
        M.molt_destroy(ctx)


@pytest.mark.parametrize("bc", [M.BC_PERIODIC, M.BC_DIRICHLET])
def test_fp64_multiwarp_tile_shapes(bc):
    """FP64 sweeps take the fewest points per lane that fit a line exactly
    (4 or 8), so lines of 256..4096 points run 2-16 warps per line: contiguous
    and strided lines of those lengths against the oracle."""
    need_gpu()
    # numpy shapes; axis 0 = x (the last numpy axis, contiguous), 1 = y (strided)
    for shape, axis in (((256,), 0), ((512,), 0), ((1536,), 0), ((4096,), 0), ((256, 3), 1), ((512, 6), 1),
                        ((1024, 4), 1), ((4, 1024), 0)):
        for op in (M.OP_0, M.OP_R):
            got, want = run_apply(shape, axis, op, 2, 0.21, bc, 6, M.PREC_F64, seed=len(shape) + shape[0])
            check(got, want, M.PREC_F64, len(shape), axis, (shape, axis, op))
