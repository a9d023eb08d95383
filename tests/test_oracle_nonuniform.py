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


# ---------------------------------------------------------------- WENO-Z
# Point-local linear weights and smoothness indicators (Sec. 2.4: on a
# non-uniform mesh the linear weights are local to each point).

def _jagged(n, L=2 * np.pi, seed=5, spread=0.6):
    """Nodes with independent random cell widths (no smooth mapping)."""
    w = 1.0 + spread * np.random.default_rng(seed).uniform(-1, 1, n)
    x = np.concatenate([[0.0], np.cumsum(w)[:-1]])
    return x * (L / w.sum())


@pytest.mark.parametrize("npts", [5, 6])
def test_weno_tables_on_a_uniform_grid_are_the_uniform_constants(npts):
    """d_r and the smoothness matrices of every point reduce to the uniform
    ones (those are pinned to the closed forms of App. C)."""
    from oracle import quadrature
    n, L, alpha = 24, 3.0, 5.0
    x = L * np.arange(n) / n
    t = nonuniform.weno_tables(x, L, alpha, npts)
    rule = quadrature.QuadratureRule(alpha * L / n, npts)
    for side in "RL":
        np.testing.assert_allclose(t[side]["d"], np.broadcast_to(rule.d, (n, 3)), rtol=0, atol=1e-12)
        for r in range(3):
            np.testing.assert_allclose(t[side]["sub"][:, r], np.broadcast_to(rule.sub_c[r], (n, len(rule.sub_c[r]))),
                                       rtol=0, atol=1e-14)
            np.testing.assert_allclose(t[side]["M"][:, r], np.broadcast_to(rule.beta_M[r], t[side]["M"][:, r].shape),
                                       rtol=0, atol=1e-10)


@pytest.mark.parametrize("op", ["R", "L", "0"])
def test_weno_on_a_uniform_grid_reproduces_the_uniform_oracle(op):
    n, L, alpha = 40, 2.0, 7.0
    x = L * np.arange(n) / n
    xs = x * 2 * np.pi / L
    v = np.sign(np.sin(xs)) + 0.2 * np.cos(3 * xs)       # jumps: the nonlinear weights matter
    got = nonuniform.partial_sum(v, x, L, alpha, op, 5, 2, weights_kind="wenoz")
    want = sweep.partial_sum(v[None, :], 1, alpha, L / n, op, "periodic", 5, 2, weights="wenoz")[0]
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("npts", [5, 6])
def test_weno_linear_weights_are_partitions_of_unity_and_substencils_sum_to_one_minus_q(npts):
    n, L, alpha = 20, 2 * np.pi, 2.5
    x = _jagged(n)
    t = nonuniform.weno_tables(x, L, alpha, npts)
    _, _, q = nonuniform.weights(x, L, alpha, npts)
    for side, qs in (("R", q), ("L", np.roll(q, -1))):
        np.testing.assert_allclose(t[side]["d"].sum(axis=1), 1.0, rtol=0, atol=1e-13)
        for r in range(3):
            np.testing.assert_allclose(t[side]["sub"][:, r].sum(axis=1), 1 - qs, rtol=1e-13)
    for op in "RL0":
        S = nonuniform.partial_sum(np.full(n, -1.3), x, L, alpha, op, npts, 2, weights_kind="wenoz")
        assert np.abs(S).max() < 1e-13


@pytest.mark.parametrize("npts", [5, 6])
def test_weno_reproduces_the_exact_integral_of_substencil_degree_data(npts):
    """On data of the substencils' degree every p_r is the data itself, so
    beta_0 = beta_1 = beta_2, tau = 0, omega = d, and J is the exact kernel
    integral of the polynomial (adaptive quadrature here)."""
    from scipy.integrate import quad
    n, L, alpha = 24, 2 * np.pi, 1.7
    x = _jagged(n, seed=8)
    deg = 2 if npts == 5 else 3
    coef = [0.3, -1.1, 0.45, 0.2][:deg + 1]
    poly = lambda s: npoly.polyval(s, coef)
    v = poly(x)
    t = nonuniform.weno_tables(x, L, alpha, npts)
    JR, JL = nonuniform.local_integrals(v, x, L, alpha, npts, "wenoz", t)
    offs = STENCIL[npts]
    for i in range(-min(offs), n - max(offs)):           # stencils that do not wrap
        vals = np.array([v[i + l] for l in offs])
        om = nonuniform.weno_weights_at(vals, t["R"]["d"][i], t["R"]["M"][i])
        np.testing.assert_allclose(om, t["R"]["d"][i], rtol=0, atol=1e-9)
        want = quad(lambda s: alpha * math.exp(-alpha * (x[i] - s)) * poly(s), x[i - 1], x[i], epsabs=1e-15)[0]
        assert abs(JR[i] - want) < 1e-13
    for i in range(max(offs), n + min(offs)):            # J_L reads v_{i-l}
        want = quad(lambda s: alpha * math.exp(-alpha * (s - x[i])) * poly(s), x[i], x[i + 1], epsabs=1e-15)[0]
        assert abs(JL[i] - want) < 1e-13


def test_weno_smoothness_indicator_of_a_quadratic_has_its_closed_form():
    """p(s) = s^2 on the cell [a, b] of width dx: p' = 2s, p'' = 2, so
    beta = dx int_a^b 4 s^2 ds + dx^3 int_a^b 4 ds = 4 dx (b^3 - a^3)/3 + 4 dx^4."""
    n, L, alpha = 16, 2 * np.pi, 3.0
    x = _jagged(n, seed=11)
    t = nonuniform.weno_tables(x, L, alpha, 5)
    v = x ** 2
    for i in range(3, n - 3):
        for side, sign, (a, b) in (("R", 1, (x[i - 1], x[i])), ("L", -1, (x[i], x[i + 1]))):
            vals = np.array([v[i + sign * l] for l in STENCIL[5]])
            dx = b - a
            want = 4 * dx * (b ** 3 - a ** 3) / 3 + 4 * dx ** 4
            for r in range(3):
                got = vals[r:r + 3] @ t[side]["M"][i, r] @ vals[r:r + 3]
                assert abs(got - want) < 1e-12 * max(1.0, want)


def test_weno_is_invariant_under_scaling_and_mirroring():
    """x -> lam x with alpha -> alpha/lam leaves every nu and beta unchanged;
    mirroring the line (x -> L - x, order reversed) swaps J_R and J_L."""
    n, L, alpha = 18, 2 * np.pi, 2.2
    x = _jagged(n, seed=13)
    v = np.where(x < 2.0, 1.0, -0.5) + 0.1 * np.sin(x)
    JR, JL = nonuniform.local_integrals(v, x, L, alpha, 5, "wenoz")
    lam = 3.7
    JR2, JL2 = nonuniform.local_integrals(v, lam * x, lam * L, alpha / lam, 5, "wenoz")
    np.testing.assert_allclose(JR2, JR, rtol=0, atol=1e-12)
    np.testing.assert_allclose(JL2, JL, rtol=0, atol=1e-12)
    # mirrored nodes y_j = L - x_{n-1-j} (shifted to start at 0), data reversed
    y = L - x[::-1]
    y = y - y[0]
    JRm, JLm = nonuniform.local_integrals(v[::-1].copy(), y, L, alpha, 5, "wenoz")
    np.testing.assert_allclose(JRm[::-1], JL, rtol=0, atol=1e-12)
    np.testing.assert_allclose(JLm[::-1], JR, rtol=0, atol=1e-12)


def test_weno_drops_the_substencil_across_a_jump():
    """A jump between x_{i-3} and x_{i-2} lies only in S_0 of J_R(x_i): the
    constant substencils have beta = 0, so omega_0 = O(eps) and J_R is the
    constant's integral (1 - q_i) c to that accuracy."""
    n, L, alpha = 30, 2 * np.pi, 2.0
    x = _jagged(n, seed=17)
    c = 0.8
    i = 12
    v = np.full(n, c)
    v[:i - 2] = -1.0
    v[i + 3:] = c                                        # the stencil of i sees one jump
    t = nonuniform.weno_tables(x, L, alpha, 5)
    vals = np.array([v[i + l] for l in STENCIL[5]])
    om = nonuniform.weno_weights_at(vals, t["R"]["d"][i], t["R"]["M"][i])
    assert om[0] < 1e-5, om
    JR, _ = nonuniform.local_integrals(v, x, L, alpha, 5, "wenoz", t)
    _, _, q = nonuniform.weights(x, L, alpha, 5)
    assert abs(JR[i] - (1 - q[i]) * c) < 1e-5


def test_weno_converges_on_stretched_grids():
    """Smooth data: omega -> d, and L_0^{-1}[sin kx] reaches the continuous
    alpha^2/(alpha^2 + k^2) sin kx at high order on a smoothly stretched grid."""
    L, alpha, k = 2 * np.pi, 4.0, 3
    errs = []
    for n in (64, 128, 256):
        x = _stretched(n)
        got = nonuniform.inverse(np.sin(k * x), x, L, alpha, "0", 5, weights_kind="wenoz",
                                 weno=nonuniform.weno_tables(x, L, alpha, 5))
        errs.append(np.abs(got - alpha ** 2 / (alpha ** 2 + k ** 2) * np.sin(k * x)).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(r > 3.5 for r in rates), (errs, rates)


# ---------------------------------------------------------------- Dirichlet
# Non-uniform Dirichlet lines (Sec. 2.3): nodes x_0 = a .. x_N = b, mirrored
# ghost nodes with odd-reflected data, boundary constants from the boundary
# values.

def _dirichlet_nodes(N, a=0.0, b=np.pi, amp=0.25):
    t = np.linspace(0.0, 1.0, N + 1)
    return a + (b - a) * (t + amp * np.sin(2 * np.pi * t) / (2 * np.pi))


@pytest.mark.parametrize("npts,kind", [(3, "linear"), (6, "linear"), (5, "linear"), (5, "wenoz")])
@pytest.mark.parametrize("op", ["R", "L", "0"])
def test_dirichlet_on_a_uniform_grid_reproduces_the_uniform_oracle(npts, kind, op):
    N, a, b, alpha = 30, 0.5, 2.0, 9.0
    x = np.linspace(a, b, N + 1)
    v = np.random.default_rng(21).standard_normal(N + 1)
    got = nonuniform.partial_sum(v, x, None, alpha, op, npts, 2, kind)
    want = sweep.partial_sum(v[None, :], 1, alpha, (b - a) / N, op, "dirichlet", npts, 2, weights=kind)[0]
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("npts,kind", [(6, "linear"), (5, "wenoz")])
def test_dirichlet_is_the_doubled_periodic_line_with_odd_data(npts, kind):
    """Homogeneous data: the Dirichlet line equals the periodic line of
    period 2(b - a) through the nodes mirrored about b, with the data odd
    about a and b (images + uniqueness of the 2x2 solve), for L_0 and S_P."""
    N, alpha = 17, 4.0
    x = _dirichlet_nodes(N)
    a, b = x[0], x[-1]
    v = np.random.default_rng(22).standard_normal(N + 1)
    v[0] = v[-1] = 0.0
    xd = np.concatenate([x, 2 * b - x[-2:0:-1]])
    vd = np.concatenate([v, -v[-2:0:-1]])
    got = nonuniform.partial_sum(v, x, None, alpha, "0", npts, 3, kind)
    want = nonuniform.partial_sum(vd, xd, 2 * (b - a), alpha, "0", npts, 3, kind)[:N + 1]
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("op", ["R", "L", "0"])
def test_dirichlet_keeps_constants_in_the_kernel_of_D_and_meets_the_boundary_values(op):
    N, alpha = 20, 3.0
    x = _dirichlet_nodes(N, amp=0.4)
    S = nonuniform.partial_sum(np.full(N + 1, 0.9), x, None, alpha, op, 6, 2)
    assert np.abs(S).max() < 1e-13
    v = np.random.default_rng(23).standard_normal(N + 1)
    Li = nonuniform.inverse(v, x, None, alpha, op, 6)
    if op in "R0":
        assert abs(Li[0] - v[0]) < 1e-13                 # L^{-1}[v](a) = v(a)
    if op in "L0":
        assert abs(Li[-1] - v[-1]) < 1e-13               # L^{-1}[v](b) = v(b)


def test_dirichlet_right_inverse_is_the_cell_by_cell_integral_plus_the_inflow_term():
    """L_R^{-1}[v](x_i) = sum over the cells left of x_i of alpha int
    e^{-alpha (x_i - s)} p_j(s) ds (p_j the interpolant of the cell's stencil,
    with mirrored ghosts) + v(a) e^{-alpha (x_i - a)} -- no recurrence."""
    N, alpha, npts = 9, 2.3, 6
    x = _dirichlet_nodes(N, amp=0.5)
    v = np.cos(x) + 0.4 * x
    offs = STENCIL[npts]
    gx, gw = np.polynomial.legendre.leggauss(40)

    def node(j):
        if j < 0:
            return 2 * x[0] - x[-j]
        if j > N:
            return 2 * x[N] - x[2 * N - j]
        return x[j]

    def val(j):
        if j < 0:
            return 2 * v[0] - v[-j]
        if j > N:
            return 2 * v[N] - v[2 * N - j]
        return v[j]

    want = np.zeros(N + 1)
    for i in range(N + 1):
        tot = v[0] * math.exp(-alpha * (x[i] - x[0]))
        for j in range(1, i + 1):
            a, b = node(j - 1), node(j)
            s = 0.5 * (b - a) * gx + 0.5 * (b + a)
            nodes = [node(j + l) - node(j) for l in offs]
            p = sum(val(j + l) * npoly.polyval(s - node(j), lagrange_basis(nodes, m)) for m, l in enumerate(offs))
            tot += np.sum(0.5 * (b - a) * gw * alpha * np.exp(-alpha * (x[i] - s)) * p)
        want[i] = tot
    got = nonuniform.inverse(v, x, None, alpha, "R", npts)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_dirichlet_converges_to_the_continuous_operator_on_stretched_grids():
    """sin kx on [0, pi] is odd about both ends, so the homogeneous Dirichlet
    L_0^{-1}[sin kx] is alpha^2/(alpha^2 + k^2) sin kx."""
    alpha, k = 4.0, 3
    errs = []
    for N in (64, 128, 256):
        x = _dirichlet_nodes(N)
        got = nonuniform.inverse(np.sin(k * x), x, None, alpha, "0", 6)
        errs.append(np.abs(got - alpha ** 2 / (alpha ** 2 + k ** 2) * np.sin(k * x)).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(r > 5.0 for r in rates), (errs, rates)
