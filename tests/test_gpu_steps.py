"""GPU parity of molt_step (the fused multi-axis passes and the time-integrator
epilogues) against the oracle's schemes, for every problem family."""
import math

import numpy as np
import pytest

from oracle import schemes
from paper_2007_03041_gb300 import molt as M
from paper_2007_03041_gb300 import workloads
from tests.gpu_util import need_gpu, rel_l2, to_dev, tol_for, state_dtype, assert_grid_parity

pytestmark = pytest.mark.gpu
TOL_F64_STEPS = 1e-12


@pytest.mark.parametrize("prec", [M.PREC_F64, M.PREC_F32_F64UPDATE])
@pytest.mark.parametrize("n", [64, 100])
def test_heat_rk3_2d(prec, n):
    need_gpu()
    import torch
    h = 1.0 / n
    dt = h / 2
    u0 = workloads.heat_modes(n)
    d = M.make_desc((n, n), P=3, quad_points=3, beta=0.6, pde=M.PDE_HEAT, diffusivity=1.0, dt=dt, prec=prec)
    ctx = M.molt_create(d)
    try:
        u = to_dev(u0, torch.float64)
        t = M.molt_step(ctx, u, None, nsteps=3, t=[0.0])
        got = u.cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    want = u0
    for _ in range(3):
        want = schemes.heat_step(want, [h, h], dt, 1.0, 0.6, None, 3, 3)
    assert_grid_parity(got, want, tol_for(prec))
    assert abs(t[0] - 3 * dt) < 1e-15


@pytest.mark.parametrize("nsteps", [1, 2, 3])
def test_wave_leapfrog_3d_dirichlet(nsteps):
    need_gpu()
    import torch
    n = 33
    h = 1.0 / (n - 1)
    dt = 2 * h
    u0 = workloads.wave_bumps(n)
    d = M.make_desc((n, n, n), bc=[M.BC_DIRICHLET] * 3, P=2, quad_points=6, beta=0.8, pde=M.PDE_WAVE,
                    c=1.0, dt=dt, prec=M.PREC_F32_F64UPDATE)
    ctx = M.molt_create(d)
    try:
        u = to_dev(u0, torch.float64)
        up = torch.full_like(u, float("nan"))   # ignored when starting from rest
        M.molt_step(ctx, u, up, nsteps=nsteps, t=[0.0])
        got, gotp = u.cpu().numpy(), up.cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    bc = ["dirichlet"] * 3
    prev, cur = None, u0
    for k in range(nsteps):
        nxt = schemes.wave_step(cur, prev, [h] * 3, dt, 1.0, 0.8, bc, 6, 2, from_rest=(k == 0))
        prev, cur = cur, nxt
    assert_grid_parity(got, cur, 1e-5)
    assert_grid_parity(gotp, prev, 1e-5)


def test_wave_continues_across_calls_and_fp64():
    need_gpu()
    import torch
    n = 21
    h = 1.0 / (n - 1)
    dt = 2 * h
    u0 = workloads.wave_bumps(n)
    for prec, tol in ((M.PREC_F64, 1e-12), (M.PREC_F32_F64UPDATE, 1e-5)):
        d = M.make_desc((n, n, n), bc=[M.BC_DIRICHLET] * 3, P=2, quad_points=6, beta=0.8, pde=M.PDE_WAVE,
                        c=1.0, dt=dt, prec=prec)
        ctx = M.molt_create(d)
        try:
            u = to_dev(u0, torch.float64)
            up = torch.zeros_like(u)
            t = M.molt_step(ctx, u, up, nsteps=1, t=[0.0])
            t = M.molt_step(ctx, u, up, nsteps=2, t=t)
            got = u.cpu().numpy()
        finally:
            M.molt_destroy(ctx)
        prev, cur = None, u0
        for k in range(3):
            nxt = schemes.wave_step(cur, prev, [h] * 3, dt, 1.0, 0.8, ["dirichlet"] * 3, 6, 2, from_rest=(k == 0))
            prev, cur = cur, nxt
        assert_grid_parity(got, cur, tol)
        assert abs(t[0] - 3 * dt) < 1e-14


@pytest.mark.parametrize("prec,weights", [(M.PREC_F32, M.W_WENOZ), (M.PREC_F64, M.W_WENOZ),
                                          (M.PREC_F32, M.W_LINEAR)])
def test_hj_lagged_adaptive_2d(prec, weights):
    need_gpu()
    import torch
    n = 128
    h = 2 * np.pi / n
    u0 = workloads.hj_initial(n)
    d = M.make_desc((n, n), lo=[0, 0], hi=[2 * np.pi] * 2, P=1, quad_points=5, weights=weights, beta=1.0,
                    pde=M.PDE_HJ, cfl=1.5, dt=0.0, prec=prec)
    ctx = M.molt_create(d)
    try:
        u = to_dev(u0, state_dtype(prec))
        t = M.molt_step(ctx, u, None, nsteps=2, t=[0.0])
        t = M.molt_step(ctx, u, None, nsteps=2, t=t)
        got = u.double().cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    wname = "wenoz" if weights == M.W_WENOZ else "linear"
    uu = u0.astype(np.float32).astype(np.float64) if prec == M.PREC_F32 else u0
    speeds = schemes.hj_initial_speeds(uu, [h, h], 1.5, 1.0, 5, wname)
    tt = 0.0
    for _ in range(4):
        uu, dt, speeds = schemes.hj_step(uu, [h, h], speeds, 1.5, 1.0, 5, wname)
        tt += dt
    assert_grid_parity(got, uu, tol_for(prec))
    assert abs(t[0] - tt) < (1e-12 if prec == M.PREC_F64 else 1e-4) * tt


def test_nonfinite_state_is_reported():
    need_gpu()
    import torch
    n = 32
    u0 = workloads.heat_modes(n)
    u0[3, 4] = np.inf
    d = M.make_desc((n, n), P=1, quad_points=3, beta=0.6, pde=M.PDE_HEAT, dt=0.5 / n, prec=M.PREC_F64)
    ctx = M.molt_create(d)
    try:
        u = to_dev(u0, torch.float64)
        with pytest.raises(M.MoltError) as ei:
            M.molt_step(ctx, u, None, nsteps=1, t=[0.0])
        assert ei.value.status == M.MOLT_ENONFINITE
    finally:
        M.molt_destroy(ctx)


@pytest.mark.slow
@pytest.mark.parametrize("nx,ny,prec,transposed", [(256, 4096, M.PREC_F32, True), (4096, 256, M.PREC_F32, False),
                                                    (64, 4096, M.PREC_F64, True)])
def test_hj_anisotropic_long_lines(nx, ny, prec, transposed):
    """Long y lines run the y pass on the transposed state (their tiles would
    hold fewer than 32 bytes of lines); long x lines do not.  FP64 dt: the
    speeds are one-sided derivatives alpha*D[u], whose FP64 rounding is
    amplified by the cancellation in D = u - L^{-1}u, so dt agrees to 1e-10
    relative."""
    need_gpu()
    import torch
    hx_, hy_ = 2 * np.pi / nx, 2 * np.pi / ny
    g = workloads.rng(9)
    x = 2 * np.pi * np.arange(nx) / nx
    y = 2 * np.pi * np.arange(ny) / ny
    u0 = -np.cos(x)[None, :] - np.cos(2 * y)[:, None] + 1e-3 * g.standard_normal((ny, nx))
    d = M.make_desc((nx, ny), lo=[0, 0], hi=[2 * np.pi] * 2, P=1, quad_points=5, weights=M.W_WENOZ, beta=1.0,
                    pde=M.PDE_HJ, cfl=1.5, dt=0.0, prec=prec)
    ctx = M.molt_create(d)
    try:
        u = to_dev(u0, state_dtype(prec))
        M.molt_set_option(ctx, M.OPT_PROFILE, 1)
        # three steps in two calls: the transposed form alternates the
        # state's layout and returns it in u after an odd count
        t = M.molt_step(ctx, u, None, nsteps=2, t=[0.0])
        got2 = u.double().cpu().numpy()
        t = M.molt_step(ctx, u, None, nsteps=1, t=t)
        _, ntr = M.molt_profile_read(ctx, M.KERNEL_TRANSPOSE)
        got = u.double().cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    # one for the speeds of u^0, two per step, one back after the odd run
    assert ntr == (8 if transposed else 0)
    uu = u0.astype(np.float32).astype(np.float64) if prec == M.PREC_F32 else u0
    dxs = [hy_, hx_]            # numpy axis order: y, x
    speeds = schemes.hj_initial_speeds(uu, dxs, 1.5, 1.0, 5, "wenoz")
    tt = 0.0
    for k in range(3):
        uu, dt, speeds = schemes.hj_step(uu, dxs, speeds, 1.5, 1.0, 5, "wenoz")
        tt += dt
        if k == 1:
            assert_grid_parity(got2, uu, tol_for(prec), what="after 2 steps")
    assert_grid_parity(got, uu, tol_for(prec), what="after 3 steps")
    assert abs(t[0] - tt) < (1e-10 if prec == M.PREC_F64 else 1e-4) * tt


def test_hj_linear_hamiltonian_on_long_y_lines():
    """H = a.grad u with a_x != a_y on long y lines (the transposed y pass):
    the transposed problem carries the swapped velocities."""
    need_gpu()
    import torch
    nx, ny = 128, 4096
    hx_, hy_ = 2 * np.pi / nx, 2 * np.pi / ny
    x = 2 * np.pi * np.arange(nx) / nx
    y = 2 * np.pi * np.arange(ny) / ny
    u0 = np.sin(x)[None, :] + 0.5 * np.cos(3 * y)[:, None]
    vel = (0.7, -1.3)
    d = M.make_desc((nx, ny), lo=[0, 0], hi=[2 * np.pi] * 2, P=1, quad_points=6, beta=1.0, pde=M.PDE_HJ, cfl=0.5,
                    dt=0.0, prec=M.PREC_F64, hamiltonian=M.H_LINEAR, velocity=vel)
    ctx = M.molt_create(d)
    try:
        u = to_dev(u0, torch.float64)
        M.molt_set_option(ctx, M.OPT_PROFILE, 1)
        t = M.molt_step(ctx, u, None, nsteps=3, t=[0.0])
        _, ntr = M.molt_profile_read(ctx, M.KERNEL_TRANSPOSE)
        got = u.cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    assert ntr == 8
    dxs = [hy_, hx_]
    a = [vel[1], vel[0]]        # numpy axis order
    uu = u0
    speeds = schemes.hj_initial_speeds(uu, dxs, 0.5, 1.0, 6, "linear", hamiltonian=schemes.H_LINEAR, a=a)
    tt = 0.0
    for _ in range(3):
        uu, dt, speeds = schemes.hj_step(uu, dxs, speeds, 0.5, 1.0, 6, "linear", hamiltonian=schemes.H_LINEAR, a=a)
        tt += dt
    assert_grid_parity(got, uu, TOL_F64_STEPS)
    assert abs(t[0] - tt) < 1e-10 * tt


@pytest.mark.parametrize("case", ["heat1d", "heat3d", "wave1d", "wave2d_periodic", "hj1d"])
def test_other_dimensions(case):
    """Every PDE in the other dimensions the descriptor allows, against the
    oracle's schemes (FP64 and mixed precision)."""
    need_gpu()
    import torch
    g = workloads.rng(12)
    if case.startswith("heat"):
        shape = (48,) if case == "heat1d" else (20, 24, 28)           # numpy order
        shape_xyz = tuple(reversed(shape))
        hs = [1.0 / s for s in shape]
        dt = min(hs) / 2
        u0 = g.standard_normal(shape)
        for prec in (M.PREC_F64, M.PREC_F32_F64UPDATE):
            d = M.make_desc(shape_xyz, P=3, quad_points=3, beta=0.6, pde=M.PDE_HEAT, dt=dt, prec=prec)
            ctx = M.molt_create(d)
            try:
                u = to_dev(u0, torch.float64)
                M.molt_step(ctx, u, None, nsteps=2, t=[0.0])
                got = u.cpu().numpy()
            finally:
                M.molt_destroy(ctx)
            want = u0
            for _ in range(2):
                want = schemes.heat_step(want, hs, dt, 1.0, 0.6, None, 3, 3)
            assert_grid_parity(got, want, tol_for(prec), what=str(prec))
    elif case.startswith("wave"):
        shape = (64,) if case == "wave1d" else (40, 56)
        shape_xyz = tuple(reversed(shape))
        per = case == "wave2d_periodic"
        bc = M.BC_PERIODIC if per else M.BC_DIRICHLET
        hs = [1.0 / (s if per else s - 1) for s in shape]
        dt = 2 * min(hs)
        u0 = g.standard_normal(shape)
        if not per:
            workloads.zero_boundary(u0)
        for prec in (M.PREC_F64, M.PREC_F32_F64UPDATE):
            d = M.make_desc(shape_xyz, bc=[bc] * len(shape), P=2, quad_points=6, beta=0.8, pde=M.PDE_WAVE, c=1.0,
                            dt=dt, prec=prec)
            ctx = M.molt_create(d)
            try:
                u = to_dev(u0, torch.float64)
                up = torch.empty_like(u)
                M.molt_step(ctx, u, up, nsteps=3, t=[0.0])
                got = u.cpu().numpy()
            finally:
                M.molt_destroy(ctx)
            bcs = ["periodic" if per else "dirichlet"] * len(shape)
            prev, cur = None, u0
            for k in range(3):
                nxt = schemes.wave_step(cur, prev, hs, dt, 1.0, 0.8, bcs, 6, 2, from_rest=(k == 0))
                prev, cur = cur, nxt
            assert_grid_parity(got, cur, tol_for(prec), what=str(prec))
    else:
        n = 256
        h = 2 * np.pi / n
        x = np.arange(n) * h
        u0 = -np.cos(x) + 1e-3 * g.standard_normal(n)
        for prec in (M.PREC_F64, M.PREC_F32):
            d = M.make_desc((n,), lo=[0.0], hi=[2 * np.pi], P=1, quad_points=5, weights=M.W_WENOZ, beta=1.0,
                            pde=M.PDE_HJ, cfl=1.5, dt=0.0, prec=prec)
            ctx = M.molt_create(d)
            try:
                u = to_dev(u0, state_dtype(prec))
                t = M.molt_step(ctx, u, None, nsteps=3, t=[0.0])
                got = u.double().cpu().numpy()
            finally:
                M.molt_destroy(ctx)
            uu = u0.astype(np.float32).astype(np.float64) if prec == M.PREC_F32 else u0
            speeds = schemes.hj_initial_speeds(uu, [h], 1.5, 1.0, 5, "wenoz")
            for _ in range(3):
                uu, _, speeds = schemes.hj_step(uu, [h], speeds, 1.5, 1.0, 5, "wenoz")
            assert_grid_parity(got, uu, tol_for(prec), what=str(prec))


def test_hj_3d_is_rejected():
    need_gpu()
    d = M.make_desc((16, 16, 16), P=1, quad_points=5, weights=M.W_WENOZ, pde=M.PDE_HJ, cfl=1.5, prec=M.PREC_F32)
    with pytest.raises(M.MoltError) as e:
        M.molt_create(d)
    assert e.value.status == M.MOLT_EUNSUPPORTED


@pytest.mark.parametrize("prec", [M.PREC_F64, M.PREC_F32_F64UPDATE, M.PREC_F32])
@pytest.mark.parametrize("shape_xyz", [(96, 80), (24, 20, 16)])
def test_heat_axis_streams_match_serial_axes(prec, shape_xyz):
    """Small heat problems sweep their axes on two streams at once
    (MOLT_OPT_AXIS_STREAMS, default on): in 2-D the same values as the axes
    one after another, bit for bit (S_x + S_y either way); in 3-D the sums
    add as S_x + (S_y + S_z) instead of (S_x + S_y) + S_z, so the two differ
    by rounding only; both match the oracle's SSP-RK3 step."""
    need_gpu()
    import torch
    nd = len(shape_xyz)
    hs = [1.0 / n for n in shape_xyz]
    dt = 0.5 * min(hs)
    shape_np = tuple(reversed(shape_xyz))
    u0 = np.cos(2 * np.pi * np.arange(shape_np[-1]) / shape_np[-1]) + 0.1 * workloads.rng(21).standard_normal(shape_np)
    if prec == M.PREC_F32:
        u0 = u0.astype(np.float32).astype(np.float64)
    d = M.make_desc(shape_xyz, P=3, quad_points=3, beta=0.6, pde=M.PDE_HEAT, diffusivity=1.0, dt=dt, prec=prec)
    out = {}
    for mode in (1, 0):
        ctx = M.molt_create(d)
        try:
            M.molt_set_option(ctx, M.OPT_AXIS_STREAMS, mode)
            u = to_dev(u0, state_dtype(prec))
            M.molt_step(ctx, u, None, nsteps=3, t=[0.0])
            out[mode] = u.double().cpu().numpy()
        finally:
            M.molt_destroy(ctx)
    if nd == 2:
        assert np.array_equal(out[0], out[1])
    else:
        assert_grid_parity(out[1], out[0], 1e-14 if prec == M.PREC_F64 else 1e-6, what="streams vs serial")
    want = u0
    for _ in range(3):
        want = schemes.heat_step(want, hs[::-1], dt, 1.0, 0.6, None, 3, 3)
    assert_grid_parity(out[1], want, tol_for(prec), what="%dD" % nd)


@pytest.mark.parametrize("prec", [M.PREC_F64, M.PREC_F32_F64UPDATE])
def test_heat_graph_replay_matches_direct_launches(prec):
    """On a stream that can be captured, small heat problems replay one
    captured step per step after a first direct one (and re-capture when the
    state array changes); on the legacy default stream every step launches
    directly.  Same values bit for bit, and the oracle's steps."""
    need_gpu()
    import torch
    n = 128
    h = 1.0 / n
    dt = h / 2
    u0 = workloads.heat_modes(n)
    d = M.make_desc((n, n), P=3, quad_points=3, beta=0.6, pde=M.PDE_HEAT, diffusivity=1.0, dt=dt, prec=prec)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = M.molt_create(d, stream)
        try:
            a = to_dev(u0, torch.float64)
            t = M.molt_step(ctx, a, None, nsteps=4, t=[0.0])
            b = a.clone()                                   # a new state array: captured again
            t = M.molt_step(ctx, b, None, nsteps=3, t=t)
            stream.synchronize()
            got = b.cpu().numpy()
        finally:
            M.molt_destroy(ctx)
    ctx = M.molt_create(d)
    try:
        c = to_dev(u0, torch.float64)
        M.molt_step(ctx, c, None, nsteps=7, t=[0.0])
        direct = c.cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    assert np.array_equal(got, direct)
    want = u0
    for _ in range(7):
        want = schemes.heat_step(want, [h, h], dt, 1.0, 0.6, None, 3, 3)
    assert_grid_parity(got, want, tol_for(prec))
    assert abs(t[0] - 7 * dt) < 1e-14
