"""Pins of the oracle's forms for the test problems of Sec. 5.1 (first order
in time, P = 1, 6-point linear quadrature): the local Lax-Friedrichs
Hamiltonian for general H, forward-Euler advection and diffusion against
their closed-form discrete solutions (Fourier symbols, an independent route
from the recurrences), the manufactured Hamilton-Jacobi problem's first-order
convergence, and the L-infinity errors the paper prints for 5277^2 grids."""
import math
import os
import pathlib

import numpy as np
import pytest

from oracle import schemes, stability
from paper_2007_03041_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.txt")


def _paper_numbers():
    out = {}
    for line in pathlib.Path(GOLDEN).read_text().splitlines():
        line = line.split("#")[0].split()
        if len(line) == 2:
            out[line[0]] = float(line[1])
    return out


KINDS = [(schemes.H_HALF_SQ, None, 0.0), (schemes.H_LINEAR, (1.0, -0.5), 0.0),
         (schemes.H_AFFINE_SQ, (1.0, 1.0), 1.0), (schemes.H_AFFINE_SQ, (-0.7, 0.3), -0.4)]


@pytest.mark.parametrize("kind,a,h0", KINDS)
def test_llf_consistent_and_r_bounds_the_slope_on_the_box(kind, a, h0):
    g = np.random.default_rng(3)
    # consistency: equal one-sided derivatives give H itself
    p = [g.standard_normal(50), g.standard_normal(50)]
    Hh, _ = schemes.hj_hamiltonian([(p[0], p[0]), (p[1], p[1])], kind, a, h0)
    np.testing.assert_allclose(Hh, schemes.hamiltonian(kind, p, a, h0), rtol=1e-14, atol=1e-14)
    # r_d >= |dH/dp_d| everywhere on the box of one-sided derivatives (what
    # makes H^ monotone with r frozen), with equality somewhere on it
    ders = [(g.standard_normal(200), g.standard_normal(200)) for _ in range(2)]
    r = schemes.llf_r(ders, kind, a, h0)
    best = [np.zeros(200), np.zeros(200)]
    for _ in range(64):
        w = [g.uniform(0, 1, 200) for _ in range(2)]
        pt = [dm + wd * (dp - dm) for (dm, dp), wd in zip(ders, w)]
        gr = schemes.hamiltonian_grad(kind, pt, a, h0)
        for d in range(2):
            assert np.all(np.abs(gr[d]) <= r[d] * (1 + 1e-14) + 1e-15)
            best[d] = np.maximum(best[d], np.abs(gr[d]))
    for corner in ((0, 0), (0, 1), (1, 0), (1, 1)):
        gr = schemes.hamiltonian_grad(kind, [ders[d][corner[d]] for d in range(2)], a, h0)
        for d in range(2):
            best[d] = np.maximum(best[d], np.abs(gr[d]))
    for d in range(2):
        np.testing.assert_allclose(best[d], r[d], rtol=1e-14, atol=1e-15)


def test_llf_special_cases():
    g = np.random.default_rng(4)
    ders = [(g.standard_normal(100), g.standard_normal(100)) for _ in range(2)]
    # linear advection: the upwind value of each axis
    a = (1.0, -0.5)
    Hh, sp = schemes.hj_hamiltonian(ders, schemes.H_LINEAR, a)
    np.testing.assert_allclose(Hh, 1.0 * ders[0][0] - 0.5 * ders[1][1], rtol=1e-14, atol=1e-15)
    assert sp == [1.0, 0.5]
    # (h0 + a.p)^2/2 with a = (1, 0), h0 = 0 is p_x^2/2: the x part of |p|^2/2
    Ha, spa = schemes.hj_hamiltonian(ders, schemes.H_AFFINE_SQ, (1.0, 0.0), 0.0)
    Hx, spx = schemes.hj_hamiltonian(ders[:1], schemes.H_HALF_SQ)
    np.testing.assert_allclose(Ha, Hx, rtol=1e-14, atol=1e-15)
    assert spa[0] == spx[0] and spa[1] == 0.0


def _advection_closed_form(n, steps, a, beta=1.0, npts=6):
    """Example 1 by Fourier modes: each mode of u0 is multiplied per step by
    G = 1 - dt (sum_d a_d * symbol of the upwind one-sided derivative)."""
    h = 2 * math.pi / n
    dt = h / max(abs(x) for x in a)        # CFL 1
    alpha = beta / h                       # beta / (CFL h)
    nu = alpha * h
    modes = {(0, 0): 0.25, (1, 0): -0.125, (-1, 0): -0.125, (0, 1): -0.125, (0, -1): -0.125,
             (1, 1): 1 / 16, (1, -1): 1 / 16, (-1, 1): 1 / 16, (-1, -1): 1 / 16}
    x, y = workloads.paper_grid(n)
    out = np.zeros((n, n), dtype=complex)
    for (kx, ky), am in modes.items():
        H = 0.0
        for ad, k in zip(a, (kx, ky)):
            if ad > 0:
                H = H + ad * alpha * (1 - stability.symbol(k * h, nu, "R", npts))
            else:
                H = H + ad * (-alpha) * (1 - stability.symbol(k * h, nu, "L", npts))
        G = 1 - dt * H
        out += am * G ** steps * np.exp(1j * (kx * x + ky * y))
    return out.real


@pytest.mark.parametrize("a", [(1.0, 1.0), (-1.0, 0.5)])
def test_advection_example_matches_closed_form(a):
    """a = (a_x, a_y)."""
    n, steps = 32, 12
    h = 2 * math.pi / n
    u = workloads.advection_initial(n)
    # the oracle's axes are numpy's ([y][x]): velocities (a_y, a_x)
    kw = dict(cfl=1.0, npts=6, weights="linear", hamiltonian=schemes.H_LINEAR, a=a[::-1])
    sp = schemes.hj_initial_speeds(u, [h, h], **kw)
    for _ in range(steps):
        u, dt, sp = schemes.hj_step(u, [h, h], sp, **kw)
    assert abs(dt - h / max(abs(x) for x in a)) < 1e-15
    want = _advection_closed_form(n, steps, a)
    assert np.abs(u - want).max() < 1e-13


def _diffusion_closed_form_amplitude(n, steps, beta=1.0, npts=6):
    h = 2 * math.pi / n
    dt = h
    nu = beta / math.sqrt(dt) * h
    G = 1 - beta ** 2 * stability.partial_sum_symbol(h, nu, "0", npts, 1).real
    return G ** steps


def test_diffusion_example_matches_closed_form():
    n, steps = 32, 10
    h = 2 * math.pi / n
    u = workloads.diffusion_initial(n)
    for _ in range(steps):
        u = schemes.heat_euler_step(u, [h, h], h, beta=1.0, npts=6, P=1)
    want = _diffusion_closed_form_amplitude(n, steps) * workloads.diffusion_initial(n)
    assert np.abs(u - want).max() < 1e-13


def _run_manufactured(n, T):
    h = 2 * math.pi / n
    F = workloads.manufactured_hj_source(n)
    kw = dict(cfl=1.0, npts=6, weights="linear", hamiltonian=schemes.H_AFFINE_SQ, a=(1.0, 1.0), h0=1.0)
    u = np.zeros((n, n))
    sp = schemes.hj_initial_speeds(u, [h, h], **kw)
    t = 0.0
    while t < T:
        u, dt, sp = schemes.hj_step(u, [h, h], sp, source=F, t=t, **kw)
        t += dt
    return u, t


def test_manufactured_hj_converges_first_order():
    errs = []
    # the runs end at the first step past T = 0.5 and are compared with the
    # exact solution at that time
    for n in (64, 128, 256):
        u, t = _run_manufactured(n, 0.5)
        errs.append(np.abs(u - workloads.manufactured_hj_solution(n, t)).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(0.85 < r < 1.3 for r in rates), (errs, rates)


def test_closed_form_errors_at_5277_near_printed_values():
    """The paper's 5277^2 L-infinity errors (Sec. 5.1 figure caption) against
    the closed-form discrete solutions of the same schemes: the same order of
    magnitude (the paper does not state its grid and final-step conventions,
    so only a soft bound holds)."""
    ref = _paper_numbers()
    n = 5277
    h = 2 * math.pi / n
    # Example 1 to T = 2 pi: n steps of dt = h
    adv = np.abs(_advection_closed_form(n, n, (1.0, 1.0)) - workloads.advection_initial(n)).max()
    # Example 2 to T = 1: the nearest whole number of steps of dt = h
    steps = round(1.0 / h)
    amp = _diffusion_closed_form_amplitude(n, steps)
    dif = abs(amp - math.exp(-steps * h)) * 2.0
    for got, key in ((adv, "linf_5277_advection"), (dif, "linf_5277_diffusion")):
        assert ref[key] / 1.5 < got < ref[key] * 1.5, (key, got, ref[key])


def test_hj_rk3_linear_advection_matches_closed_form():
    """SSP-RK3 with three-term one-sided sums (Sec. 2.5) for H = a.grad u:
    each mode is multiplied per step by R(z), R the RK3 polynomial and
    z = -dt sum_d a_d * (symbol of the upwind three-term sum)."""
    n, steps = 32, 5
    h = 2 * math.pi / n
    a = (1.0, -0.5)                      # (a_x, a_y)
    beta, cfl = 0.3, 1.0
    u = workloads.advection_initial(n)
    kw = dict(cfl=cfl, beta=beta, npts=6, weights="linear", P=3, hamiltonian=schemes.H_LINEAR, a=a[::-1])
    sp = schemes.hj_initial_speeds_P(u, [h, h], **kw)
    for _ in range(steps):
        u, dt, sp = schemes.hj_step_rk3(u, [h, h], sp, **kw)
    alpha = beta / (cfl * h)
    nu = alpha * h
    modes = {(0, 0): 0.25, (1, 0): -0.125, (-1, 0): -0.125, (0, 1): -0.125, (0, -1): -0.125,
             (1, 1): 1 / 16, (1, -1): 1 / 16, (-1, 1): 1 / 16, (-1, -1): 1 / 16}
    x, y = workloads.paper_grid(n)
    want = np.zeros((n, n), dtype=complex)
    for (kx, ky), am in modes.items():
        H = 0.0
        for ad, k in zip(a, (kx, ky)):
            if ad > 0:
                H = H + ad * alpha * stability.partial_sum_symbol(k * h, nu, "R", 6, 3)
            else:
                H = H + ad * (-alpha) * stability.partial_sum_symbol(k * h, nu, "L", 6, 3)
        z = -dt * H
        G = 1 + z + z * z / 2 + z ** 3 / 6
        want += am * G ** steps * np.exp(1j * (kx * x + ky * y))
    assert abs(dt - h) < 1e-15
    assert np.abs(u - want.real).max() < 1e-13


def test_hj_rk3_manufactured_source_is_third_order_in_time_per_step():
    """With the manufactured source, the step error of SSP-RK3 with P = 3 is
    smaller than forward Euler's at the same dt (one step from the exact
    solution at t = 0.2, on a fine grid)."""
    n = 128
    h = 2 * math.pi / n
    F = workloads.manufactured_hj_source(n)
    t0 = 0.2
    u0 = workloads.manufactured_hj_solution(n, t0)
    kw = dict(cfl=1.0, npts=6, weights="linear", hamiltonian=schemes.H_AFFINE_SQ, a=(1.0, 1.0), h0=1.0)
    sp = schemes.hj_initial_speeds_P(u0, [h, h], P=3, **kw)
    u_rk, dt, _ = schemes.hj_step_rk3(u0, [h, h], sp, t=t0, P=3, source=F, **kw)
    u_fe, dt_fe, _ = schemes.hj_step(u0, [h, h], sp, source=F, t=t0, **kw)
    assert abs(dt - dt_fe) < 1e-15
    e_rk = np.abs(u_rk - workloads.manufactured_hj_solution(n, t0 + dt)).max()
    e_fe = np.abs(u_fe - workloads.manufactured_hj_solution(n, t0 + dt)).max()
    assert e_rk < 0.2 * e_fe, (e_rk, e_fe)
