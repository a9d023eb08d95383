"""Pins of oracle/dense.py: the dense-matrix evaluation of the linear schemes
against the line-by-line oracle, and the periodic axis matrix against the
exact discrete symbol (an independent closed form: a circulant matrix's
eigenvalues are its symbol on the grid's Fourier modes)."""
import numpy as np
import pytest

from oracle import dense, schemes, sweep, stability


@pytest.mark.parametrize("bc", ["periodic", "dirichlet"])
@pytest.mark.parametrize("op,npts,P", [("0", 6, 2), ("R", 5, 1), ("L", 3, 3)])
def test_axis_matrix_applies_partial_sum(bc, op, npts, P):
    n = 37
    g = np.random.default_rng(1)
    V = g.standard_normal((5, n))
    dx = 1.0 / (n if bc == "periodic" else n - 1)
    M = dense.axis_matrix(n, 0.3 / dx, dx, op, bc, npts, P)
    want = sweep.partial_sum_lines(V, 0.3 / dx, dx, op, bc, npts, P)
    assert np.abs(V @ M.T - want).max() < 1e-13


@pytest.mark.parametrize("op", ["0", "R", "L"])
def test_periodic_axis_matrix_eigenvalues_are_the_symbol(op):
    n, nu, npts, P = 48, 0.4, 6, 2
    M = dense.axis_matrix(n, nu * n, 1.0 / n, op, "periodic", npts, P)
    theta = 2 * np.pi * np.arange(n) / n
    want = stability.partial_sum_symbol(theta, nu, op, npts, P)
    # Fourier modes diagonalise the circulant matrix: M e_k = s(theta_k) e_k
    j = np.arange(n)
    for k in range(n):
        mode = np.exp(1j * j * theta[k])
        assert np.abs(M @ mode - want[k] * mode).max() < 1e-13


@pytest.mark.parametrize("bc", ["periodic", "dirichlet"])
def test_dense_wave_steps_match_schemes(bc):
    shape = (14, 17, 20)
    h = [1.0 / (m if bc == "periodic" else m - 1) for m in shape]
    dt = 2 * min(h)
    g = np.random.default_rng(2)
    u0 = g.standard_normal(shape)
    bcs = [bc] * 3
    mats = dense.wave_matrices(shape, h, dt, 1.0, 0.8, bcs, 6, 2)
    a_prev, a = None, u0
    b_prev, b = None, u0
    for k in range(4):
        a, a_prev = schemes.wave_step(a, a_prev, h, dt, 1.0, 0.8, bcs, 6, 2, from_rest=(k == 0)), a
        b, b_prev = dense.wave_step(b, b_prev, mats, 0.8, from_rest=(k == 0)), b
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()
    assert np.abs(a_prev - b_prev).max() < 1e-12 * np.abs(a_prev).max()


def test_dense_heat_steps_match_schemes():
    shape = (24, 18)
    h = [1.0 / m for m in shape]
    dt = 0.5 * min(h)
    g = np.random.default_rng(3)
    u0 = g.standard_normal(shape)
    mats = dense.heat_matrices(shape, h, dt, 1.0, 0.6, None, 3, 3)
    a = b = u0
    for _ in range(3):
        a = schemes.heat_step(a, h, dt, 1.0, 0.6, None, 3, 3)
        b = dense.heat_step(b, mats, 0.6)
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()
