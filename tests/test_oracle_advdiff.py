"""Pins of the oracle's flux-split advection-diffusion step (Sec. 2.5): the
linear flux against the closed-form discrete solution from the Fourier
symbols (forward Euler with P = 1 and SSP-RK3 with P = 3), exact mass
conservation for Burgers' flux on periodic lines, and first-order
convergence to the exact inviscid Burgers solution before the shock."""
import math

import numpy as np
import pytest

from oracle import schemes, stability


def _grid(n):
    return 2 * np.pi * np.arange(n) / n


@pytest.mark.parametrize("rk3,P", [(False, 1), (True, 3), (True, 1)])
def test_linear_flux_matches_closed_form(rk3, P):
    n, steps = 32, 6
    h = 2 * np.pi / n
    a = (0.7, -0.4)            # (a_x, a_y)
    # beta = 0.3: every mode has |G| <= 1 for the three schemes (RK3 with P = 3
    # already amplifies the highest modes at beta = 0.4 here)
    c, kappa, beta, dt = 1.0, 0.05, 0.3, 0.6 * h
    x = _grid(n)
    modes = {(1, 0): 0.8, (2, -1): -0.5, (0, 3): 0.3, (-3, 2): 0.2}
    u = sum(am * np.cos(kx * x[None, :] + ky * x[:, None]) for (kx, ky), am in modes.items())
    for _ in range(steps):
        # oracle axes follow the array ([y][x]): velocities (a_y, a_x)
        u = schemes.advdiff_step(u, [h, h], dt, schemes.FLUX_LINEAR, a[::-1], c, kappa, beta, 6, P, rk3)
    nu_a = beta / (c * dt) * h
    nu_d = beta / math.sqrt(kappa * dt) * h
    want = np.zeros((n, n))
    for (kx, ky), am in modes.items():
        for sgn in (1, -1):              # cos = (e^{i t} + e^{-i t})/2
            z = 0.0
            for ad, k in zip(a, (kx, ky)):
                th = sgn * k * h
                SR = stability.partial_sum_symbol(th, nu_a, "R", 6, P)
                SL = stability.partial_sum_symbol(th, nu_a, "L", 6, P)
                z = z - (beta / c) * (0.5 * (ad + c) * SR - 0.5 * (ad - c) * SL)
                z = z - beta ** 2 * stability.partial_sum_symbol(th, nu_d, "0", 6, P)
            G = 1 + z + z * z / 2 + z ** 3 / 6 if rk3 else 1 + z
            want = want + (0.5 * am * G ** steps * np.exp(1j * sgn * (kx * x[None, :] + ky * x[:, None]))).real
    assert np.abs(u - want).max() < 1e-13


def test_burgers_conserves_mass():
    n = 48
    h = 2 * np.pi / n
    x = _grid(n)
    u = 0.3 + np.sin(x)[None, :] * np.cos(2 * x)[:, None] + 0.2 * np.cos(3 * x)[:, None]
    m0 = u.sum()
    c = 1.6
    for _ in range(5):
        u = schemes.advdiff_step(u, [h, h], 0.5 * h / c, schemes.FLUX_BURGERS, None, c, 0.02, 0.9, 6, 1)
    assert abs(u.sum() - m0) < 1e-12 * np.abs(u).sum()


def _burgers_exact(x, t):
    """u = sin(x - u t), by fixed-point iteration (contracting for t < 1)."""
    u = np.sin(x)
    for _ in range(200):
        u = np.sin(x - u * t)
    return u


def test_inviscid_burgers_converges_first_order():
    T, errs = 0.5, []
    for n in (64, 128, 256):
        h = 2 * np.pi / n
        x = _grid(n)
        u = np.sin(x)
        dt = 0.5 * h
        steps = int(round(T / dt))
        for _ in range(steps):
            u = schemes.advdiff_step(u, [h], dt, schemes.FLUX_BURGERS, None, 1.0, 0.0, 1.0, 6, 1)
        errs.append(np.abs(u - _burgers_exact(x, steps * dt)).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(0.85 < r < 1.3 for r in rates), (errs, rates)
