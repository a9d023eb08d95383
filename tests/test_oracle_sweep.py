"""Pins of the oracle's fast summation (recurrences + boundary constants +
partial sums) against brute force, closed-form symbols and invariants."""
import math

import numpy as np
import pytest
from numpy.polynomial import polynomial as npoly
from scipy import integrate

from oracle import sweep, stability
from oracle import quadrature as Q


# ---------------------------------------------------------------- brute force
def _local_interp(vext_fn, i, offsets):
    """Polynomial in the local variable t = s - i (grid units) interpolating v
    at the nodes i + l, l in offsets -- the interpolant J_R(x_i) uses on the
    cell [x_{i-1}, x_i] (or, with mirrored offsets, J_L on [x_i, x_{i+1}])."""
    nodes = np.array(offsets, dtype=float)
    vals = np.array([vext_fn(i + int(l)) for l in offsets])
    return npoly.polyfit(nodes, vals, len(nodes) - 1)


def _cell_integral(alpha, dx, p, t0, t1, dist0, direction):
    """alpha dx int_{t0}^{t1} e^{-alpha dx (dist0 + direction*t)} p(t) dt."""
    f = lambda t: alpha * dx * math.exp(-alpha * dx * (dist0 + direction * t)) * npoly.polyval(t, p)
    return integrate.quad(f, t0, t1, epsabs=1e-17, epsrel=1e-14)[0]


def brute_inverse_periodic(v, alpha, dx, op, npts):
    """O(N^2) L^{-1}[v](x_i): the exponential kernel integrated exactly (scipy
    adaptive quadrature) against the piecewise stencil interpolant of the
    periodic data, summing periodic images until they vanish."""
    N = len(v)
    offs = Q.STENCIL[npts]
    mirrored = tuple(-l for l in offs)

    def vf(k):
        return v[k % N]

    polysR = [_local_interp(vf, k, offs) for k in range(N)]      # cell [x_{k-1}, x_k]
    polysL = [_local_interp(vf, k, mirrored) for k in range(N)]  # cell [x_k, x_{k+1}]
    nimg = int(40.0 / (alpha * dx * N)) + 2
    out = np.zeros(N)
    for i in range(N):
        tot_R = 0.0
        tot_L = 0.0
        for m in range(0, nimg * N):
            # R: cell [x_{k-1}, x_k], k = i - m; s = x_k + t dx, t in [-1, 0];
            # distance x_i - s = (m - t) dx
            tot_R += _cell_integral(alpha, dx, polysR[(i - m) % N], -1.0, 0.0, m, -1.0)
            # L: cell [x_k, x_{k+1}], k = i + m; s = x_k + t dx, t in [0, 1];
            # distance s - x_i = (m + t) dx; the mirrored interpolant is in t
            tot_L += _cell_integral(alpha, dx, polysL[(i + m) % N], 0.0, 1.0, m, 1.0)
        out[i] = {"R": tot_R, "L": tot_L, "0": 0.5 * (tot_R + tot_L)}[op]
    return out


@pytest.mark.parametrize("npts", [3, 5, 6])
@pytest.mark.parametrize("op", ["L", "R", "0"])
def test_periodic_recurrence_matches_brute_force(npts, op):
    g = np.random.default_rng(11)
    N = 12
    v = g.standard_normal(N)
    dx = 1.0 / N
    alpha = 2.3 / dx * 0.4   # nu = 0.92
    got = sweep.inverse_operator(v[None, :], alpha, dx, op, "periodic", npts)[0]
    want = brute_inverse_periodic(v, alpha, dx, op, npts)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


def brute_inverse_dirichlet_L0(v, alpha, dx, npts):
    """O(N^2) Dirichlet L_0^{-1}: (alpha/2) int_a^b e^{-alpha|x-s|} p(s) ds by
    adaptive quadrature of the piecewise interpolant (ghosts by odd reflection
    about the boundary values), plus A e^{-alpha(x-a)} + B e^{-alpha(b-x)}
    with A, B from L^{-1}[v](a) = v(a), L^{-1}[v](b) = v(b) (numpy solve)."""
    n = len(v)
    N = n - 1
    offs = Q.STENCIL[npts]
    mirrored = tuple(-l for l in offs)

    def vf(k):
        if k < 0:
            return 2 * v[0] - v[-k]
        if k > N:
            return 2 * v[N] - v[2 * N - k]
        return v[k]

    I0 = np.zeros(n)
    for i in range(n):
        tot = 0.0
        for k in range(1, i + 1):          # cells [x_{k-1}, x_k] left of x_i
            tot += 0.5 * _cell_integral(alpha, dx, _local_interp(vf, k, offs), -1.0, 0.0, i - k, -1.0)
        for k in range(i, N):              # cells [x_k, x_{k+1}] right of x_i
            tot += 0.5 * _cell_integral(alpha, dx, _local_interp(vf, k, mirrored), 0.0, 1.0, k - i, 1.0)
        I0[i] = tot
    mu = math.exp(-alpha * dx * N)
    A, B = np.linalg.solve(np.array([[1.0, mu], [mu, 1.0]]), np.array([v[0] - I0[0], v[N] - I0[N]]))
    x = np.arange(n)
    return I0 + A * np.exp(-alpha * dx * x) + B * np.exp(-alpha * dx * (N - x))


@pytest.mark.parametrize("npts", [3, 5, 6])
def test_dirichlet_L0_matches_brute_force(npts):
    g = np.random.default_rng(5)
    n = 11
    v = g.standard_normal(n)
    dx = 0.1
    alpha = 3.0   # nu = 0.3: A, B reach across the whole line
    got = sweep.inverse_operator(v[None, :], alpha, dx, "0", "dirichlet", npts)[0]
    want = brute_inverse_dirichlet_L0(v, alpha, dx, npts)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)
    assert abs(got[0] - v[0]) < 1e-13 and abs(got[-1] - v[-1]) < 1e-13


# ------------------------------------------------------------- closed forms
@pytest.mark.parametrize("npts", [3, 5, 6])
@pytest.mark.parametrize("op", ["L", "R", "0"])
def test_periodic_fourier_symbol(npts, op):
    N = 48
    dx = 2 * np.pi / N
    alpha = 0.37 / dx
    j = np.arange(N)
    for k in (1, 7, 23):
        th = 2 * np.pi * k / N
        lam = stability.symbol(th, alpha * dx, op, npts)
        for phase in (0.0, 0.3):
            v = np.cos(th * j + phase)
            got = sweep.inverse_operator(v[None, :], alpha, dx, op, "periodic", npts)[0]
            want = (lam * np.exp(1j * (th * j + phase))).real
            np.testing.assert_allclose(got, want, atol=2e-15 * N)


def test_symbol_converges_to_continuous_symbol():
    # L_0^{-1} on e^{ikx} -> alpha^2/(alpha^2+k^2) as dx -> 0 at fixed alpha, at
    # the order of the quadrature (6 points: O(dx^6)).
    alpha, k = 5.0, 3.0
    errs = []
    for N in (32, 64, 128):
        dx = 2 * np.pi / N
        lam = stability.symbol(k * dx, alpha * dx, "0", 6).real
        errs.append(abs(lam - alpha ** 2 / (alpha ** 2 + k ** 2)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(5.5 < r < 6.6 for r in rates), rates
    # and the one-sided operators -> alpha/(alpha +- i k)
    dx = 2 * np.pi / 256
    lamR = stability.symbol(k * dx, alpha * dx, "R", 6)
    assert abs(lamR - alpha / (alpha + 1j * k)) < 1e-9


def test_dirichlet_equals_doubled_periodic_with_odd_data():
    g = np.random.default_rng(3)
    n = 17
    N = n - 1
    v = g.standard_normal(n)
    v[0] = v[-1] = 0.0
    dx = 1.0 / N
    for alpha, npts, P in ((6.0, 6, 2), (20.0, 3, 3), (2.0, 5, 1)):
        got = sweep.partial_sum_lines(v[None, :], alpha, dx, "0", "dirichlet", npts, P)[0]
        # odd extension to period 2N: w_j = v_j (0..N), w_{2N-j} = -v_j
        w = np.concatenate([v[:N], -v[N:0:-1]])
        per = sweep.partial_sum_lines(w[None, :], alpha, dx, "0", "periodic", npts, P)[0]
        np.testing.assert_allclose(got, per[:n], atol=1e-14)


# ------------------------------------------------------------- invariants
@pytest.mark.parametrize("npts", [3, 5, 6])
@pytest.mark.parametrize("op", ["L", "R", "0"])
def test_constants_are_in_the_kernel_of_D(npts, op):
    v = np.full((2, 20), 1.7)
    S = sweep.partial_sum_lines(v, 9.0, 0.05, op, "periodic", npts, 3)
    assert np.abs(S).max() < 1e-14


@pytest.mark.parametrize("npts", [3, 5, 6])
def test_local_integrals_exact_on_polynomials(npts):
    # J_R(x_i) = alpha int_{x_{i-1}}^{x_i} e^{-alpha(x_i-s)} v(s) ds exactly for
    # polynomials of degree < npts (interior nodes, no ghosts involved).
    n, dx, alpha = 30, 0.07, 4.0
    coef = np.random.default_rng(1).standard_normal(npts)
    x = np.arange(n) * dx
    v = npoly.polyval(x, coef)[None, :]
    rule = Q.QuadratureRule(alpha * dx, npts)
    vext = sweep.extend(v, "dirichlet")
    centres = np.arange(5, n - 5)
    JR = sweep.local_integrals(vext, centres, rule, "R")[0]
    JL = sweep.local_integrals(vext, centres, rule, "L")[0]
    for m, i in enumerate(centres):
        fR = lambda s: alpha * math.exp(-alpha * (x[i] - s)) * npoly.polyval(s, coef)
        fL = lambda s: alpha * math.exp(-alpha * (s - x[i])) * npoly.polyval(s, coef)
        assert abs(JR[m] - integrate.quad(fR, x[i] - dx, x[i], epsabs=1e-16)[0]) < 1e-13
        assert abs(JL[m] - integrate.quad(fL, x[i], x[i] + dx, epsabs=1e-16)[0]) < 1e-13


def test_wenoz_reduces_to_linear_on_quadratics():
    n, dx, alpha = 40, 0.1, 6.0
    x = np.arange(n) * dx
    v = (0.3 - 1.2 * x + 0.7 * x * x)[None, :]
    rule = Q.QuadratureRule(alpha * dx, 5)
    vext = sweep.extend(v, "dirichlet")
    c = np.arange(4, n - 4)
    for side in "RL":
        lin = sweep.local_integrals(vext, c, rule, side, "linear")
        wz = sweep.local_integrals(vext, c, rule, side, "wenoz")
        np.testing.assert_allclose(wz, lin, atol=1e-13)


def test_wenoz_suppresses_substencil_across_a_jump():
    # a step between x_0 and x_1 (relative to centre i): only the substencil
    # {-3,-2,-1} of J_R(x_i) stays on one side of it... use jump inside S_2 only
    rule = Q.QuadratureRule(0.5, 5)
    W = np.array([[0.0, 0.0, 0.0, 0.0, 1.0]])      # v_{i-3..i+1}, jump between i and i+1
    om = sweep._weno_weights(rule, W)[0]
    assert om[2] < 1e-3 and abs(om.sum() - 1) < 1e-15
    W = np.array([[0.1, 0.2, 0.3, 0.4, 0.5]])      # linear data: weights = d
    np.testing.assert_allclose(sweep._weno_weights(rule, W)[0], rule.d, atol=1e-15)


def test_truncation_theorem_slope():
    # d_xx = -alpha^2 (S_P + O(alpha^{-(2P+2)})) on sin(kx) (Sec. 2.2): the
    # error of -alpha^2 S_P against -k^2 decays like alpha^{-2P}.
    k = 2.0
    for P in (1, 2, 3):
        errs = []
        alphas = (40.0, 80.0)
        for alpha in alphas:
            N = 4096
            dx = 2 * np.pi / N
            s = stability.partial_sum_symbol(k * dx, alpha * dx, "0", 6, P).real
            errs.append(abs(-alpha ** 2 * s + k ** 2))
        slope = math.log(errs[0] / errs[1]) / math.log(alphas[1] / alphas[0])
        assert abs(slope - 2 * P) < 0.05, (P, slope)


def test_partial_sum_along_axes_of_nd_array():
    g = np.random.default_rng(2)
    u = g.standard_normal((6, 7, 8))
    S = sweep.partial_sum(u, 1, 3.0, 0.1, "0", "periodic", 6, 2)
    for z in range(6):
        for x in range(8):
            line = sweep.partial_sum_lines(u[z, :, x][None, :], 3.0, 0.1, "0", "periodic", 6, 2)[0]
            np.testing.assert_allclose(S[z, :, x], line, atol=1e-15)


@pytest.mark.parametrize("npts", [3, 5, 6])
@pytest.mark.parametrize("op", ["L", "R", "0"])
def test_tiny_periodic_lines_follow_the_symbol(npts, op):
    """Lines shorter than the stencil (n = 1..5, the stencil wraps onto the
    same points): every discrete mode still gets the symbol's factor, since
    the recurrences with the periodic closure sum all images exactly."""
    for n in range(1, 6):
        dx = 2 * np.pi / n
        alpha = 0.8 / dx
        j = np.arange(n)
        for k in range(n):
            th = 2 * np.pi * k / n
            lam = stability.symbol(th, alpha * dx, op, npts)
            v = np.cos(th * j + 0.4)
            got = sweep.inverse_operator(v[None, :], alpha, dx, op, "periodic", npts)[0]
            want = (lam * np.exp(1j * (th * j + 0.4))).real
            np.testing.assert_allclose(got, want, atol=1e-14, err_msg=f"n={n} k={k}")


@pytest.mark.parametrize("npts", [3, 5, 6])
def test_short_dirichlet_lines_meet_the_boundary_values(npts):
    """Dirichlet lines of 2-6 nodes (ghosts reflected about the ends, clamped
    where the line is shorter than the stencil): L_0^{-1}[v] takes the
    boundary values at both ends, L_R^{-1}[v](a) = v(a), L_L^{-1}[v](b) = v(b),
    and constants lie in the kernel of D."""
    rng = np.random.default_rng(44)
    for n in range(2, 7):
        dx = 1.0 / (n - 1)
        alpha = 0.9 / dx
        v = rng.standard_normal((1, n))
        L0 = sweep.inverse_operator(v, alpha, dx, "0", "dirichlet", npts)[0]
        LR = sweep.inverse_operator(v, alpha, dx, "R", "dirichlet", npts)[0]
        LL = sweep.inverse_operator(v, alpha, dx, "L", "dirichlet", npts)[0]
        assert abs(L0[0] - v[0, 0]) < 1e-14 and abs(L0[-1] - v[0, -1]) < 1e-14, n
        assert abs(LR[0] - v[0, 0]) < 1e-14 and abs(LL[-1] - v[0, -1]) < 1e-14, n
        for op in "LR0":
            S = sweep.partial_sum_lines(np.full((1, n), 0.6), alpha, dx, op, "dirichlet", npts, 2)
            assert np.abs(S).max() < 1e-14, (n, op)
