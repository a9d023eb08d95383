"""Pins of the non-uniform periodic oracle: on a uniform grid it is the
uniform oracle; constants lie in the kernel of D (the weights of each point
sum to 1 - q_i); the O(n^2) image sum of the kernel integral of the
piecewise interpolant on a tiny stretched grid; and convergence of
L_0^{-1}[sin kx] to the exact alpha^2/(alpha^2+k^2) sin kx at the order of
the rule on smoothly stretched grids."""
import math

import numpy as np
import pytest
from numpy.polynomial import polynomial as npoly

from oracle import nonuniform, sweep
from oracle.quadrature import STENCIL, lagrange_basis


def _stretched(n, L=2 * np.pi, amp=0.3):
    """x = xi + amp sin(xi) on a uniform xi-grid (monotone for amp < 1)."""
    xi = L * np.arange(n) / n
    return xi + amp * np.sin(xi)


@pytest.mark.parametrize("npts", [3, 5, 6])
@pytest.mark.parametrize("op", ["R", "L", "0"])
def test_uniform_grid_reproduces_the_uniform_oracle(npts, op):
    n, L, alpha = 40, 2.0, 7.0
    x = L * np.arange(n) / n
    v = np.random.default_rng(2).standard_normal(n)
    got = nonuniform.partial_sum(v, x, L, alpha, op, npts, 2)
    want = sweep.partial_sum(v[None, :], 1, alpha, L / n, op, "periodic", npts, 2)[0]
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


@pytest.mark.parametrize("npts", [3, 6])
def test_weights_sum_to_one_minus_q_and_constants_are_in_the_kernel(npts):
    n, L, alpha = 30, 2 * np.pi, 3.0
    x = _stretched(n)
    cR, cL, q = nonuniform.weights(x, L, alpha, npts)
    np.testing.assert_allclose(cR.sum(axis=1), 1 - q, rtol=1e-13)
    qL = np.roll(q, -1)                # the cell right of x_i
    np.testing.assert_allclose(cL.sum(axis=1), 1 - qL, rtol=1e-13)
    for op in "RL0":
        S = nonuniform.partial_sum(np.full(n, 0.7), x, L, alpha, op, npts, 2)
        assert np.abs(S).max() < 1e-13


def test_image_sum_brute_force_on_a_tiny_stretched_grid():
    """L_R^{-1}[v](x_i) = sum over all earlier cells (every period) of
    alpha int e^{-alpha (x_i - s)} p_j(s) ds, p_j the cell's interpolant --
    summed cell by cell with 40 periods of images."""
    n, L, alpha, npts = 9, 2 * np.pi, 1.3, 6
    x = _stretched(n, amp=0.5)
    v = np.cos(x) + 0.3 * np.sin(2 * x)
    offs = STENCIL[npts]
    gx, gw = np.polynomial.legendre.leggauss(40)

    def node(j):
        k, r = divmod(j, n)
        return x[r] + k * L

    want = np.zeros(n)
    for i in range(n):
        tot = 0.0
        for j in range(i - 40 * n, i + 1):       # cells [x_{j-1}, x_j] left of x_i
            a, b = node(j - 1), node(j)
            s = 0.5 * (b - a) * gx + 0.5 * (b + a)
            nodes = [node(j + l) - node(j) for l in offs]
            vals = [v[(j + l) % n] for l in offs]
            p = sum(vals[m] * npoly.polyval(s - node(j), lagrange_basis(nodes, m)) for m in range(len(offs)))
            tot += np.sum(0.5 * (b - a) * gw * alpha * np.exp(-alpha * (node(i) - s)) * p)
        want[i] = tot
    got = nonuniform.inverse(v, x, L, alpha, "R", npts)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_converges_to_the_continuous_operator_on_stretched_grids():
    L, alpha, k = 2 * np.pi, 4.0, 3
    errs = []
    for n in (64, 128, 256):
        x = _stretched(n)
        got = nonuniform.inverse(np.sin(k * x), x, L, alpha, "0", 6)
        errs.append(np.abs(got - alpha ** 2 / (alpha ** 2 + k ** 2) * np.sin(k * x)).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(r > 5.0 for r in rates), (errs, rates)
