"""Pins of the time integrators on non-uniform axes (the oracle's ``grids``):
uniform nodes reproduce the uniform schemes; on stretched grids the heat
equation decays its modes at the exact rate e^{-k^2 t} (periodic and
Dirichlet lines) and the Hamilton-Jacobi step converges at first order to the
characteristic solution."""
import math

import numpy as np

from oracle import schemes


def _stretch(xi, L, amp):
    return xi + amp * (L / (2 * np.pi)) * np.sin(2 * np.pi * xi / L)


def test_uniform_nodes_reproduce_the_uniform_heat_and_wave_steps():
    ny, nx, L = 12, 16, 2.0
    u = np.random.default_rng(31).standard_normal((ny, nx))
    hx, hy = L / nx, L / ny
    gx = (L * np.arange(nx) / nx, L)
    # y: a Dirichlet axis of ny nodes on [0, L]
    yd = np.linspace(0.0, L, ny)
    hyd = L / (ny - 1)
    bc = ["dirichlet", "periodic"]
    for grids in ((None, gx), ((yd, None), gx), ((yd, None), None)):
        got = schemes.heat_step(u, [hyd, hx], 0.01, bc=bc, npts=6, grids=grids)
        want = schemes.heat_step(u, [hyd, hx], 0.01, bc=bc, npts=6)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
        got = schemes.wave_step(u, 0.5 * u, [hyd, hx], 0.02, bc=bc, grids=grids)
        want = schemes.wave_step(u, 0.5 * u, [hyd, hx], 0.02, bc=bc)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
    del hy


def test_uniform_nodes_reproduce_the_uniform_hj_step():
    n, L = 24, 2 * np.pi
    h = L / n
    x = h * np.arange(n)
    u = -np.cos(x)[None, :] + 0.5 * np.sin(x)[:, None]
    grids = ((x, L), (x, L))
    sp = schemes.hj_initial_speeds(u, [h, h], grids=grids)
    np.testing.assert_allclose(sp, schemes.hj_initial_speeds(u, [h, h]), rtol=1e-13)
    got, dt, _ = schemes.hj_step(u, [h, h], sp, grids=grids)
    want, dt2, _ = schemes.hj_step(u, [h, h], sp)
    assert dt == dt2
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def _heat_mode_error(n, dt, dirichlet):
    """1-D heat on a stretched grid, u0 = sin 2x on [0, 2 pi) (periodic) or
    sin x on [0, pi] (Dirichlet), to T = 0.25: max error against the decayed
    mode."""
    T = 0.25
    if dirichlet:
        L, k = np.pi, 1
        x = _stretch(np.linspace(0.0, L, n + 1), L, 0.25)
        grids, bc = ((x, None),), ["dirichlet"]
    else:
        L, k = 2 * np.pi, 2
        x = _stretch(L * np.arange(n) / n, L, 0.3)
        grids, bc = ((x, L),), ["periodic"]
    u = np.sin(k * x)
    steps = int(round(T / dt))
    for _ in range(steps):
        u = schemes.heat_step(u, [1.0], dt, beta=0.6, bc=bc, npts=6, P=3, grids=grids)
    return np.abs(u - math.exp(-k * k * steps * dt) * np.sin(k * x)).max()


def test_heat_on_stretched_grids_decays_modes_at_the_exact_rate():
    for dirichlet in (False, True):
        errs = [_heat_mode_error(96, dt, dirichlet) for dt in (0.05, 0.025, 0.0125)]
        rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
        assert errs[-1] < 1e-3, (dirichlet, errs)
        assert all(r > 1.5 for r in rates), (dirichlet, errs, rates)


def test_hj_on_stretched_grids_converges_first_order():
    """u_t + |u_x|^2/2 = 0 in 1-D, u0 = -cos x: the characteristic solution
    (smooth while t < 1) on grids x = xi + 0.2 sin xi, dxs = the smallest cell."""
    def exact(x, t):
        x0 = x.copy()
        for _ in range(60):
            x0 = x0 - (x0 + t * np.sin(x0) - x) / (1 + t * np.cos(x0))
        return -np.cos(x0) + 0.5 * t * np.sin(x0) ** 2

    L, T = 2 * np.pi, 0.4
    errs = []
    for n in (32, 64, 128):
        x = _stretch(L * np.arange(n) / n, L, 0.2)
        hmin = np.diff(np.r_[x, x[0] + L]).min()
        grids = ((x, L),)
        u = -np.cos(x)
        speeds = schemes.hj_initial_speeds(u, [hmin], grids=grids)
        t = 0.0
        while True:
            dt = schemes.hj_dt(speeds, [hmin], 1.5)
            if t + dt > T:
                break
            u, dt_used, speeds = schemes.hj_step(u, [hmin], speeds, grids=grids)
            t += dt_used
        errs.append(np.abs(u - exact(x, t)).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(0.7 < r < 1.8 for r in rates), (errs, rates)


def test_uniform_nodes_reproduce_the_uniform_advection_diffusion_step():
    ny, nx, L = 10, 14, 2.0
    u = 1.0 + 0.3 * np.random.default_rng(37).standard_normal((ny, nx))
    hx, hy = L / nx, L / ny
    grids = ((L * np.arange(ny) / ny, L), (L * np.arange(nx) / nx, L))
    for kind, kappa, rk3 in (("burgers", 0.05, True), ("linear", 0.0, False)):
        got = schemes.advdiff_step(u, [hy, hx], 0.05, kind, [0.5, -1.0], 2.0, kappa=kappa, beta=0.6, npts=6,
                                   P=3 if rk3 else 1, rk3=rk3, grids=grids)
        want = schemes.advdiff_step(u, [hy, hx], 0.05, kind, [0.5, -1.0], 2.0, kappa=kappa, beta=0.6, npts=6,
                                    P=3 if rk3 else 1, rk3=rk3)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_advection_diffusion_on_a_stretched_grid_converges_at_third_order():
    """u_t + u_x = kappa u_xx on a stretched periodic grid, u0 = sin x, SSP-RK3
    with P = 3, dt = h/2, to T = 0.5: the exact solution is
    e^{-kappa t} sin(x - t); halving h cuts the error about 8 times (third
    order in time, Sec. 2.5: an s-stage method with s-term sums)."""
    L, kappa, T = 2 * np.pi, 0.1, 0.5
    errs = []
    for n in (24, 48):
        x = _stretch(L * np.arange(n) / n, L, 0.3)
        dt = 0.5 * L / n
        steps = int(round(T / dt))
        u = np.sin(x)
        for _ in range(steps):
            u = schemes.advdiff_step(u, [L / n], dt, "linear", [1.0], 1.0, kappa=kappa, beta=0.6, npts=6, P=3,
                                     rk3=True, grids=((x, L),))
        errs.append(np.abs(u - math.exp(-kappa * steps * dt) * np.sin(x - steps * dt)).max())
    assert errs[1] < 1e-3
    assert errs[0] / errs[1] > 6.5, errs


def test_uniform_nodes_reproduce_the_uniform_hj_rk3_step():
    n, L = 20, 2 * np.pi
    h = L / n
    x = h * np.arange(n)
    u = -np.cos(x)[None, :] + 0.5 * np.sin(x)[:, None]
    grids = ((x, L), (x, L))
    sp = schemes.hj_initial_speeds_P(u, [h, h], P=2, grids=grids)
    np.testing.assert_allclose(sp, schemes.hj_initial_speeds_P(u, [h, h], P=2), rtol=1e-13)
    got, dt, _ = schemes.hj_step_rk3(u, [h, h], sp, P=2, grids=grids)
    want, dt2, _ = schemes.hj_step_rk3(u, [h, h], sp, P=2)
    assert dt == dt2
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
