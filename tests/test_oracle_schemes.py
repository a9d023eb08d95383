"""Pins of the oracle's time integrators: closed-form discrete solutions built
from the (brute-force-pinned) Fourier symbol, non-growth, and the exact
characteristic solution of the Hamilton-Jacobi problem."""
import math

import numpy as np
import pytest

from oracle import schemes, stability, sweep
from paper_2007_03041_gb300 import workloads


def _rk3_poly(z):
    return 1 + z + z * z / 2 + z ** 3 / 6


@pytest.mark.parametrize("npts,P,beta", [(3, 3, 0.6), (6, 3, 0.6), (3, 1, 0.6)])
def test_heat_rk3_matches_closed_form_discrete_solution(npts, P, beta):
    # each periodic Fourier mode is an eigenvector of every operator: u^n =
    # R(z)^n u^0 with z = -beta^2 (S_P(theta_x) + S_P(theta_y)), R the RK3
    # polynomial (SSP-RK3 is third-order, so its linear amplification is R).
    N = 32
    h = 1.0 / N
    dt = h / 2
    alpha = beta / math.sqrt(dt)
    nu = alpha * h
    j = np.arange(N)
    modes = [((3, 1), 0.7), ((5, 9), -1.3), ((15, 2), 0.4)]
    u0 = np.zeros((N, N))
    want = np.zeros((N, N))
    nsteps = 7
    for (kx, ky), a in modes:
        tx, ty = 2 * np.pi * kx / N, 2 * np.pi * ky / N
        m = a * np.cos(tx * j[None, :] + ty * j[:, None])
        u0 += m
        z = -beta ** 2 * (stability.partial_sum_symbol(tx, nu, "0", npts, P).real
                          + stability.partial_sum_symbol(ty, nu, "0", npts, P).real)
        want += _rk3_poly(z) ** nsteps * m
    u = u0
    for _ in range(nsteps):
        u = schemes.heat_step(u, [h, h], dt, 1.0, beta, None, npts, P)
    np.testing.assert_allclose(u, want, atol=1e-13)


def test_wave_leapfrog_matches_closed_form_dirichlet_sine_modes():
    # Dirichlet sine modes are odd about both ends, hence modes of the doubled
    # periodic line at theta = pi k / N; started from rest, the mode amplitude
    # is cos(n phi) with cos phi = 1 - beta^2 Q / 2, Q = sum_d S_2(theta_d).
    n = 13
    N = n - 1
    h = 1.0 / N
    dt = 2 * h
    beta = 0.8
    alpha = beta / dt
    nu = alpha * h
    j = np.arange(n)
    kz, ky, kx = 2, 5, 9
    th = [math.pi * k / N for k in (kz, ky, kx)]
    u0 = (np.sin(th[0] * j)[:, None, None] * np.sin(th[1] * j)[None, :, None]
          * np.sin(th[2] * j)[None, None, :])
    Qs = sum(stability.partial_sum_symbol(t, nu, "0", 6, 2).real for t in th)
    phi = math.acos(1 - beta ** 2 * Qs / 2)
    bc = ["dirichlet"] * 3
    prev = u0
    u = schemes.wave_step(u0, None, [h] * 3, dt, 1.0, beta, bc, 6, 2, from_rest=True)
    for step in range(1, 6):
        np.testing.assert_allclose(u, math.cos(step * phi) * u0, atol=2e-14)
        u, prev = schemes.wave_step(u, prev, [h] * 3, dt, 1.0, beta, bc, 6, 2), u


@pytest.mark.parametrize("dt_over_h", [0.5, 2.0, 20.0])
def test_heat_norm_non_increasing_below_beta_max(dt_over_h):
    N = 24
    h = 1.0 / N
    dt = dt_over_h * h
    bmax = stability.beta_max(lambda b: b / math.sqrt(dt) * h, 2, 3, 3, "rk3")
    beta = 0.6 if bmax > 0.6 else 0.95 * bmax
    u = workloads.random_lines((N, N), seed=4)
    norms = [np.linalg.norm(u)]
    for _ in range(200):
        u = schemes.heat_step(u, [h, h], dt, 1.0, beta, None, 3, 3)
        norms.append(np.linalg.norm(u))
    assert all(norms[i + 1] <= norms[i] * (1 + 1e-13) for i in range(len(norms) - 1))


def test_heat_grows_above_beta_max():
    # the same check has teeth: beta well above the bound blows up
    N = 24
    h = 1.0 / N
    dt = h / 2
    u = workloads.random_lines((N, N), seed=4)
    n0 = np.linalg.norm(u)
    for _ in range(60):
        u = schemes.heat_step(u, [h, h], dt, 1.0, 1.0, None, 3, 3)
    assert np.linalg.norm(u) > 10 * n0


def test_wave_from_rest_never_exceeds_initial_norm():
    # with real phi every mode amplitude is |cos(n phi)| <= 1 (Parseval)
    n = 12
    h = 1.0 / n
    dt = 2 * h
    u0 = workloads.random_lines((n, n, n), seed=9)
    n0 = np.linalg.norm(u0)
    prev = u0
    u = schemes.wave_step(u0, None, [h] * 3, dt, 1.0, 0.8, None, 6, 2, from_rest=True)
    for _ in range(300):
        assert np.linalg.norm(u) <= n0 * (1 + 1e-12)
        u, prev = schemes.wave_step(u, prev, [h] * 3, dt, 1.0, 0.8, None, 6, 2), u


def test_beta_max_readings():
    # cfg heat 256^2: dt = h/2, P=3: the chosen beta = 0.6 is below the bound;
    # wave 512^3 Dirichlet: nu = beta/2, P=2: beta = 0.8 below the bound;
    # the paper's beta = 1 is above both bounds for these couplings.
    h = 1 / 256
    dt = h / 2
    bh = stability.beta_max(lambda b: b / math.sqrt(dt) * h, 2, 3, 3, "rk3")
    bw = stability.beta_max(lambda b: b / 2.0, 3, 6, 2, "leapfrog")
    assert 0.6 < bh < 1.0 and 0.8 < bw < 1.0
    assert abs(stability.rk3_real_limit() + 2.5127453266) < 1e-9


# ---------------------------------------------------------------- HJ
def _exact_separable_hj(x, t):
    """u_t + u_x^2/2 = 0, u(x,0) = -cos x: characteristics x = x0 + t sin x0,
    u = -cos x0 + t sin^2 x0 / 2 (smooth while t < 1)."""
    x0 = x.copy()
    for _ in range(60):
        x0 = x0 - (x0 + t * np.sin(x0) - x) / (1 + t * np.cos(x0))
    return -np.cos(x0) + 0.5 * t * np.sin(x0) ** 2


def _run_hj(N, T):
    h = 2 * np.pi / N
    x = np.arange(N) * h
    u = -np.cos(x)[None, :] - np.cos(x)[:, None]
    speeds = schemes.hj_initial_speeds(u, [h, h])
    t = 0.0
    while t < T - 1e-14:
        dt = schemes.hj_dt(speeds, [h, h], 1.5)
        if t + dt > T:
            break
        u, dt_used, speeds = schemes.hj_step(u, [h, h], speeds)
        t += dt_used
    return u, x, t


def test_hj_converges_to_characteristic_solution_first_order():
    errs = []
    for N in (32, 64, 128):
        u, x, t = _run_hj(N, 0.4)
        ex = _exact_separable_hj(x, t)
        exact2 = ex[None, :] + ex[:, None]
        errs.append(np.abs(u - exact2).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(0.7 < r < 1.6 for r in rates), (errs, rates)


def test_hj_separable_data_stays_separable_and_constants_stay_put():
    N = 32
    h = 2 * np.pi / N
    g = np.random.default_rng(1)
    f = g.standard_normal(N) * 0.1
    u = np.tile(f, (N, 1))       # depends on x only
    speeds = schemes.hj_initial_speeds(u, [h, h])
    for _ in range(3):
        u, _, speeds = schemes.hj_step(u, [h, h], speeds)
    assert np.abs(u - u[0:1, :]).max() < 1e-15
    c = np.full((N, N), 0.25)
    sp = schemes.hj_initial_speeds(c, [h, h])
    c2, dt, _ = schemes.hj_step(c, [h, h], sp)
    assert np.abs(c2 - 0.25).max() < 1e-15 and dt == 10 * h


def test_lax_friedrichs_hamiltonian_consistency():
    # equal one-sided derivatives give the exact Hamiltonian; r >= |H'|
    p = np.array([0.3, -1.2]), np.array([0.3, -1.2])
    q = np.array([2.0, 0.0]), np.array([2.0, 0.0])
    Hh, sp = schemes.hj_hamiltonian([p, q])
    np.testing.assert_allclose(Hh, 0.5 * (p[0] ** 2 + q[0] ** 2))
    assert sp == [1.2, 2.0]
