"""GPU parity of sum_{p<=P} D^p along non-uniform axes (point-local
quadrature weights, the non-uniform case of Sec. 2.4) against the FP64
oracle: periodic and Dirichlet lines of several lengths, every operator and
rule, P = 1..3, FP64 / FP32 / mixed, contiguous and strided axes of 2-D and
3-D grids, in place; WENO-Z with point-local linear weights and smoothness
indicators; rejected setups."""
import numpy as np
import pytest

from oracle import nonuniform
from paper_2007_03041_gb300 import molt as M
from paper_2007_03041_gb300 import workloads
from tests.gpu_util import (MAX_F32, TOL_F32, assert_parity, max_for, need_gpu, rel_l2, state_dtype, to_dev,
                            tol_for, assert_grid_parity)

pytestmark = pytest.mark.gpu
OPS = {M.OP_L: "L", M.OP_R: "R", M.OP_0: "0"}


def _nodes(n, lo, L, amp=0.3):
    xi = L * np.arange(n) / n
    return lo + xi + amp * (L / (2 * np.pi)) * np.sin(2 * np.pi * xi / L)


def _dir_nodes(n, a, b, amp=0.3):
    """n nodes of a Dirichlet line, x_0 = a and x_{n-1} = b included, cells
    stretched by up to (1 +- amp)."""
    t = np.linspace(0.0, 1.0, n)
    x = a + (b - a) * (t + amp * np.sin(2 * np.pi * t) / (2 * np.pi))
    x[0], x[-1] = a, b
    return x


@pytest.mark.parametrize("prec", [M.PREC_F64, M.PREC_F32, M.PREC_F32_F64UPDATE])
@pytest.mark.parametrize("npts", [3, 5, 6])
def test_lines_1d(prec, npts):
    need_gpu()
    import torch
    lo, L = 0.5, 3.0
    for n, op, P in ((7, M.OP_0, 1), (100, M.OP_R, 2), (513, M.OP_L, 3), (1000, M.OP_0, 2), (2048, M.OP_R, 1)):
        x = _nodes(n, lo, L)
        alpha = 0.6 * n / L                      # nu ~ 0.6 on the average cell
        v = workloads.rng(n).standard_normal(n)
        if prec == M.PREC_F32:
            v = v.astype(np.float32).astype(np.float64)
        d = M.make_desc((n,), lo=[lo], hi=[lo + L], quad_points=npts, prec=prec)
        ctx = M.molt_create(d)
        try:
            M.molt_set_grid_axis(ctx, 0, 0, x)
            vin = to_dev(v, state_dtype(prec))
            out = torch.empty_like(vin)
            M.molt_apply_D(ctx, 0, 0, op, P, alpha, vin, out)
            got = out.double().cpu().numpy()
        finally:
            M.molt_destroy(ctx)
        want = nonuniform.partial_sum(v, x, L, alpha, OPS[op], npts, P)
        assert_parity(got, want, tol_for(prec), max_for(prec), line_axis=0, what="n=%d op=%s P=%d" % (n, op, P))


@pytest.mark.parametrize("prec", [M.PREC_F64, M.PREC_F32])
def test_both_axes_of_a_2d_grid_and_in_place(prec):
    need_gpu()
    import torch
    nx, ny, L = 96, 80, 2 * np.pi
    xs, ys = _nodes(nx, 0.0, L), _nodes(ny, 0.0, L, amp=0.4)
    u = workloads.rng(5).standard_normal((ny, nx))
    if prec == M.PREC_F32:
        u = u.astype(np.float32).astype(np.float64)
    d = M.make_desc((nx, ny), lo=[0, 0], hi=[L, L], quad_points=6, prec=prec)
    ctx = M.molt_create(d)
    try:
        M.molt_set_grid_axis(ctx, 0, 0, xs)
        M.molt_set_grid_axis(ctx, 0, 1, ys)
        uin = to_dev(u, state_dtype(prec))
        gx = torch.empty_like(uin)
        M.molt_apply_D(ctx, 0, 0, M.OP_0, 2, 9.0, uin, gx)
        gy = uin.clone()
        M.molt_apply_D(ctx, 0, 1, M.OP_R, 2, 7.0, gy, gy)         # in place
        gotx, goty = gx.double().cpu().numpy(), gy.double().cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    wantx = np.stack([nonuniform.partial_sum(u[j], xs, L, 9.0, "0", 6, 2) for j in range(ny)])
    wanty = np.stack([nonuniform.partial_sum(u[:, i], ys, L, 7.0, "R", 6, 2) for i in range(nx)], axis=1)
    assert_parity(gotx, wantx, tol_for(prec), max_for(prec), line_axis=1, what="x lines")
    assert_parity(goty, wanty, tol_for(prec), max_for(prec), line_axis=0, what="y lines")


def test_rejected_setups():
    need_gpu()
    import torch
    n, L = 64, 2.0
    d = M.make_desc((n, n), lo=[0, 0], hi=[L, L], prec=M.PREC_F64, pde=M.PDE_HEAT, dt=0.01)
    ctx = M.molt_create(d)
    try:
        with pytest.raises(M.MoltError):
            M.molt_set_grid_axis(ctx, 0, 0, _nodes(n - 1, 0.0, L))            # wrong count
        with pytest.raises(M.MoltError):
            M.molt_set_grid_axis(ctx, 0, 0, _nodes(n, 0.0, L)[::-1])          # not increasing
        with pytest.raises(M.MoltError):
            M.molt_set_grid_axis(ctx, 0, 0, np.linspace(0, 1.5 * L, n))      # wider than the period
        M.molt_set_grid_axis(ctx, 0, 1, _nodes(n, 0.0, L))
        M.molt_set_grid_axis(ctx, 0, 1, None)
        u = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        M.molt_step(ctx, u, None, nsteps=1, t=[0.0])
    finally:
        M.molt_destroy(ctx)
    dd = M.make_desc((3,), bc=[M.BC_DIRICHLET], lo=[0], hi=[L], prec=M.PREC_F64)
    ctx = M.molt_create(dd)
    try:
        with pytest.raises(M.MoltError):
            M.molt_set_grid_axis(ctx, 0, 0, _dir_nodes(3, 0.0, L))           # Dirichlet: n >= 4
    finally:
        M.molt_destroy(ctx)
    dw = M.make_desc((n,), lo=[0], hi=[L], prec=M.PREC_F32, quad_points=5, weights=M.W_LEARNED)
    ctx = M.molt_create(dw)
    try:
        M.molt_set_grid_axis(ctx, 0, 0, _nodes(n, 0.0, L))
        v = torch.zeros(n, dtype=torch.float32, device="cuda")
        with pytest.raises(M.MoltError):
            M.molt_apply_D(ctx, 0, 0, M.OP_0, 1, 5.0, v, v)                # learned weights
    finally:
        M.molt_destroy(ctx)


def test_longest_line_uses_sixteen_warps():
    """8192 points: 16 warps of 512 scan positions per line."""
    need_gpu()
    import torch
    n, lo, L = 8192, 0.0, 2 * np.pi
    x = _nodes(n, lo, L)
    v = workloads.rng(3).standard_normal(n).astype(np.float32).astype(np.float64)
    d = M.make_desc((n,), lo=[lo], hi=[lo + L], quad_points=6, prec=M.PREC_F32)
    ctx = M.molt_create(d)
    try:
        M.molt_set_grid_axis(ctx, 0, 0, x)
        vin = to_dev(v, torch.float32)
        out = torch.empty_like(vin)
        M.molt_apply_D(ctx, 0, 0, M.OP_0, 2, 0.6 * n / L, vin, out)
        got = out.double().cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    want = nonuniform.partial_sum(v, x, L, 0.6 * n / L, "0", 6, 2)
    assert_parity(got, want, TOL_F32, MAX_F32, line_axis=0, what="8192 points")


def _run_line(x, lo, L, v, op, P, alpha, prec, weights=M.W_LINEAR, npts=5):
    import torch
    n = len(x)
    d = M.make_desc((n,), lo=[lo], hi=[lo + L], quad_points=npts, prec=prec, weights=weights)
    ctx = M.molt_create(d)
    try:
        M.molt_set_grid_axis(ctx, 0, 0, x)
        vin = to_dev(v, state_dtype(prec))
        out = torch.empty_like(vin)
        M.molt_apply_D(ctx, 0, 0, op, P, alpha, vin, out)
        return out.double().cpu().numpy()
    finally:
        M.molt_destroy(ctx)


def test_wenoz_lines_1d():
    """WENO-Z with point-local d_r and smoothness indicators on rough data
    (every nonlinear weight active), each line length, operator and P, in
    FP64, FP32 and the mixed form."""
    need_gpu()
    lo, L = 0.5, 3.0
    for n, op, P in ((7, M.OP_0, 1), (100, M.OP_R, 2), (513, M.OP_L, 1), (1000, M.OP_0, 2)):
        x = _nodes(n, lo, L)
        alpha = 0.6 * n / L
        v = workloads.rng(40 + n).standard_normal(n).astype(np.float32).astype(np.float64)
        want = nonuniform.partial_sum(v, x, L, alpha, OPS[op], 5, P, "wenoz")
        for prec in (M.PREC_F64, M.PREC_F32, M.PREC_F32_F64UPDATE):
            got = _run_line(x, lo, L, v, op, P, alpha, prec, M.W_WENOZ)
            assert_parity(got, want, tol_for(prec), max_for(prec), line_axis=0,
                          what="n=%d op=%s P=%d prec=%d" % (n, op, P, prec))


def test_wenoz_keeps_a_jump_sharp_and_differs_from_the_linear_rule():
    """A square wave on a jagged grid: the GPU WENO-Z result matches the
    oracle's WENO-Z (FP64 bar) and not its linear rule, whose oscillations
    near the jumps the nonlinear weights remove."""
    need_gpu()
    n, lo, L = 400, 0.0, 2 * np.pi
    w = 1.0 + 0.6 * workloads.rng(9).uniform(-1, 1, n)
    x = np.concatenate([[0.0], np.cumsum(w)[:-1]]) * (L / w.sum())
    v = np.where((x > 1.0) & (x < 4.0), 1.0, 0.0)
    alpha = 0.8 * n / L
    want = nonuniform.partial_sum(v, x, L, alpha, "R", 5, 1, "wenoz")
    lin = nonuniform.partial_sum(v, x, L, alpha, "R", 5, 1)
    got = _run_line(x, lo, L, v, M.OP_R, 1, alpha, M.PREC_F64, M.W_WENOZ)
    assert_grid_parity(got, want, 1e-12)
    assert rel_l2(got, lin) > 1e-3


@pytest.mark.parametrize("prec", [M.PREC_F64, M.PREC_F32])
def test_wenoz_both_axes_of_a_2d_grid(prec):
    need_gpu()
    import torch
    nx, ny, L = 96, 80, 2 * np.pi
    xs, ys = _nodes(nx, 0.0, L), _nodes(ny, 0.0, L, amp=0.4)
    u = workloads.rng(6).standard_normal((ny, nx)).astype(np.float32).astype(np.float64)
    d = M.make_desc((nx, ny), lo=[0, 0], hi=[L, L], quad_points=5, prec=prec, weights=M.W_WENOZ)
    ctx = M.molt_create(d)
    try:
        M.molt_set_grid_axis(ctx, 0, 0, xs)
        M.molt_set_grid_axis(ctx, 0, 1, ys)
        uin = to_dev(u, state_dtype(prec))
        gx = torch.empty_like(uin)
        M.molt_apply_D(ctx, 0, 0, M.OP_L, 1, 9.0, uin, gx)
        gy = uin.clone()
        M.molt_apply_D(ctx, 0, 1, M.OP_0, 2, 7.0, gy, gy)         # in place, transposed lines
        gotx, goty = gx.double().cpu().numpy(), gy.double().cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    tx, wx = nonuniform.weights(xs, L, 9.0, 5), nonuniform.weno_tables(xs, L, 9.0, 5)
    ty, wy = nonuniform.weights(ys, L, 7.0, 5), nonuniform.weno_tables(ys, L, 7.0, 5)
    wantx = np.stack([nonuniform.partial_sum(u[j], xs, L, 9.0, "L", 5, 1, "wenoz", tx, wx) for j in range(ny)])
    wanty = np.stack([nonuniform.partial_sum(u[:, i], ys, L, 7.0, "0", 5, 2, "wenoz", ty, wy) for i in range(nx)],
                     axis=1)
    assert_parity(gotx, wantx, tol_for(prec), max_for(prec), line_axis=1, what="x lines")
    assert_parity(goty, wanty, tol_for(prec), max_for(prec), line_axis=0, what="y lines")


_DIR_CACHE = {}


def _dir_oracle(v, x, alpha, op, npts, P, weights="linear"):
    key = (len(x), float(x[1]), alpha, op, npts, P, weights, float(v[0]), float(v[-1]))
    if key not in _DIR_CACHE:
        _DIR_CACHE[key] = nonuniform.partial_sum(v, x, None, alpha, op, npts, P, weights)
    return _DIR_CACHE[key]


def _run_dir_line(x, v, op, P, alpha, prec, npts, weights=M.W_LINEAR):
    import torch
    n = len(x)
    d = M.make_desc((n,), bc=[M.BC_DIRICHLET], lo=[x[0]], hi=[x[-1]], quad_points=npts, prec=prec, weights=weights)
    ctx = M.molt_create(d)
    try:
        M.molt_set_grid_axis(ctx, 0, 0, x)
        vin = to_dev(v, state_dtype(prec))
        out = torch.empty_like(vin)
        M.molt_apply_D(ctx, 0, 0, op, P, alpha, vin, out)
        return out.double().cpu().numpy()
    finally:
        M.molt_destroy(ctx)


@pytest.mark.parametrize("prec", [M.PREC_F64, M.PREC_F32, M.PREC_F32_F64UPDATE])
@pytest.mark.parametrize("npts", [3, 5, 6])
def test_dirichlet_lines_1d(prec, npts):
    """Dirichlet lines, boundary nodes included: lengths 7 to 4096 (eight
    warps per line), each operator; in FP64 also a line with alpha (b - a) =
    3, where the two boundary constants couple through mu = e^{-3}, the
    shortest line a Dirichlet axis takes (4 nodes: every stencil reaches
    mirrored ghosts at both ends) and the longest (8192 nodes, 16 warps)."""
    need_gpu()
    a, b = 0.5, 3.5
    cases = [(7, M.OP_0, 1, 0.6), (100, M.OP_R, 2, 0.6), (513, M.OP_L, 3, 0.6), (1000, M.OP_0, 2, 0.6),
             (4096, M.OP_0, 1, 0.6), (300, M.OP_0, 3, 0.3)]
    if prec == M.PREC_F64:
        # alpha (b - a) = 3; the fewest nodes a Dirichlet line takes; the longest line (16 warps)
        cases += [(64, M.OP_0, 2, None), (64, M.OP_R, 1, None), (64, M.OP_L, 2, None), (4, M.OP_0, 2, 0.6),
                  (8192, M.OP_0, 1, 0.6)]
    for n, op, P, nu in cases:
        x = _dir_nodes(n, a, b)
        alpha = nu * (n - 1) / (b - a) if nu else 3.0 / (b - a)
        v = workloads.rng(70 + n).standard_normal(n).astype(np.float32).astype(np.float64)
        want = _dir_oracle(v, x, alpha, OPS[op], npts, P)
        got = _run_dir_line(x, v, op, P, alpha, prec, npts)
        assert_parity(got, want, tol_for(prec), max_for(prec), line_axis=0,
                      what="n=%d op=%s P=%d prec=%d" % (n, OPS[op], P, prec))


def test_dirichlet_wenoz_lines_1d():
    """WENO-Z on Dirichlet lines (the end points' rules are zero, the odd
    reflection feeds the ghost nodes of the smoothness indicators)."""
    need_gpu()
    a, b = 0.0, 2.0
    for n, op, P in ((7, M.OP_0, 1), (200, M.OP_R, 1), (513, M.OP_L, 2), (1000, M.OP_0, 1)):
        x = _dir_nodes(n, a, b, amp=0.4)
        alpha = 0.7 * (n - 1) / (b - a)
        v = workloads.rng(90 + n).standard_normal(n).astype(np.float32).astype(np.float64)
        want = _dir_oracle(v, x, alpha, OPS[op], 5, P, "wenoz")
        for prec in (M.PREC_F64, M.PREC_F32, M.PREC_F32_F64UPDATE):
            got = _run_dir_line(x, v, op, P, alpha, prec, 5, M.W_WENOZ)
            assert_parity(got, want, tol_for(prec), max_for(prec), line_axis=0,
                          what="n=%d op=%s P=%d prec=%d" % (n, OPS[op], P, prec))


@pytest.mark.parametrize("prec", [M.PREC_F64, M.PREC_F32])
def test_dirichlet_axes_of_2d_and_3d_grids(prec):
    """2-D: x Dirichlet (contiguous lines), y Dirichlet in place (transposed
    lines), and x periodic beside y Dirichlet; 3-D: strided y (periodic) and
    z (Dirichlet) lines."""
    need_gpu()
    import torch
    nx, ny, L = 96, 80, 2.0
    xd, yd, xp = _dir_nodes(nx, 0.0, L), _dir_nodes(ny, 0.0, L, amp=0.4), _nodes(nx, 0.0, L)
    u = workloads.rng(15).standard_normal((ny, nx)).astype(np.float32).astype(np.float64)
    for bcx, xs in ((M.BC_DIRICHLET, xd), (M.BC_PERIODIC, xp)):
        d = M.make_desc((nx, ny), bc=[bcx, M.BC_DIRICHLET], lo=[0, 0], hi=[L, L], quad_points=6, prec=prec)
        ctx = M.molt_create(d)
        try:
            M.molt_set_grid_axis(ctx, 0, 0, xs)
            M.molt_set_grid_axis(ctx, 0, 1, yd)
            uin = to_dev(u, state_dtype(prec))
            gx = torch.empty_like(uin)
            M.molt_apply_D(ctx, 0, 0, M.OP_0, 2, 40.0, uin, gx)
            gy = uin.clone()
            M.molt_apply_D(ctx, 0, 1, M.OP_0, 2, 30.0, gy, gy)
            gotx, goty = gx.double().cpu().numpy(), gy.double().cpu().numpy()
        finally:
            M.molt_destroy(ctx)
        Lx = None if bcx == M.BC_DIRICHLET else L
        wantx = nonuniform.partial_sum_axis(u, 1, xs, Lx, 40.0, "0", 6, 2)
        wanty = nonuniform.partial_sum_axis(u, 0, yd, None, 30.0, "0", 6, 2)
        assert_parity(gotx, wantx, tol_for(prec), max_for(prec), line_axis=1, what="x lines")
        assert_parity(goty, wanty, tol_for(prec), max_for(prec), line_axis=0, what="y lines")
    nx, ny, nz = 20, 18, 24
    ys, zs = _nodes(ny, 0.0, L), _dir_nodes(nz, 0.0, L)
    u3 = workloads.rng(16).standard_normal((nz, ny, nx)).astype(np.float32).astype(np.float64)
    d = M.make_desc((nx, ny, nz), bc=[M.BC_PERIODIC, M.BC_PERIODIC, M.BC_DIRICHLET], lo=[0] * 3, hi=[L] * 3,
                    quad_points=5, prec=prec)
    ctx = M.molt_create(d)
    try:
        M.molt_set_grid_axis(ctx, 0, 1, ys)
        M.molt_set_grid_axis(ctx, 0, 2, zs)
        uin = to_dev(u3, state_dtype(prec))
        gy, gz = torch.empty_like(uin), torch.empty_like(uin)
        M.molt_apply_D(ctx, 0, 1, M.OP_L, 2, 12.0, uin, gy)
        M.molt_apply_D(ctx, 0, 2, M.OP_0, 3, 10.0, uin, gz)
        goty, gotz = gy.double().cpu().numpy(), gz.double().cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    assert_parity(goty, nonuniform.partial_sum_axis(u3, 1, ys, L, 12.0, "L", 5, 2), tol_for(prec), max_for(prec),
                  line_axis=1, what="3-D y lines")
    assert_parity(gotz, nonuniform.partial_sum_axis(u3, 0, zs, None, 10.0, "0", 5, 3), tol_for(prec),
                  max_for(prec), line_axis=0, what="3-D z lines")
