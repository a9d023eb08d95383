"""Oracle: time integrators that consume the successive-convolution partial sums.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__``.

* Heat (Sec. 2.1 diffusion, Sec. 2.5 RK coupling): u_t = kappa Lap u with
  d_xx ~ -alpha^2 S_P per axis (Eq. "representation of second derivative in
  D"), alpha = beta/sqrt(kappa dt) (Sec. 2.1), so dt*F(u) = -beta^2 sum_d S_{P,d}[u].
  Integrator (reading: the paper couples an s-stage RK method with an s-term
  partial sum, Sec. 2.5; we take the 3-stage SSP Runge-Kutta method in
  Shu-Osher form with P = 3).
* Wave (Sec. 2.1 wave equation): central differencing in time with
  d_xx ~ -alpha^2 S_P, alpha = beta/(c dt):
      u^{n+1} = 2u^n - u^{n-1} - beta^2 sum_d S_{P,d}[u^n].
  Reading: a start from rest (u_t = 0) takes the second-order Taylor step
  u^1 = u^0 - beta^2/2 sum_d S_{P,d}[u^0].
* Hamilton-Jacobi (Sec. 2.5, numerical Hamiltonian; Sec. 4.4 adaptive rule;
  Algorithm 1): u^{n+1} = u^n - dt^n H^(u_x^-, u_x^+, u_y^-, u_y^+) with
  d_x^- u = alpha D_R[u], d_x^+ u = -alpha D_L[u] (P = 1, Eq.
  "representations used in paper"), the monotone (Lax-Friedrichs) numerical
  Hamiltonian H^ = H(mean) + sum_d r_d (v_d^- - v_d^+)/2 and
  dt^n = CFL * min_d(dx_d / c_d) from the wave speeds of the previous step
  ("lagged", Algorithm 1).  Readings: H = |grad u|^2/2 so r_d =
  max(|v_d^-|, |v_d^+|) pointwise (local LF); c_d = max over the grid of r_d;
  alpha = beta/(CFL dx) (= beta/(c_max dt) whenever the CFL rule sets dt, so
  nu = beta/CFL stays fixed); dt is capped at 10 dx when c -> 0; at the first
  step the speeds of u^0 serve as the lagged speeds.
* The test problems of Sec. 5.1 (first order in time, P = 1): forward Euler
  for the heat equation (Example 2), u^{n+1} = u^n - beta^2 sum_d S_{1,d}[u^n];
  the Hamilton-Jacobi step with other Hamiltonians, H = u_x + u_y (Example 1,
  linear advection) and H = (1 + u_x + u_y)^2/2 (Example 3), and a source
  F(x, t) on the right-hand side (Example 3's manufactured solution):
  u^{n+1} = u^n - dt^n (H^ - F(., t_n)).  The local Lax-Friedrichs r_d is the
  largest |dH/dp_d| over the box of one-sided derivatives prod_d
  [min(v_d^-, v_d^+), max(v_d^-, v_d^+)]; for these Hamiltonians |dH/dp_d| is
  the absolute value of an affine function, so the largest value sits at a
  corner of the box, and the oracle evaluates every corner.
* Non-uniform axes (Sec. 2.4): ``grids[ax] = (x, L)`` gives the nodes of that
  array axis (period L, or L None for a Dirichlet line) and its partial sums
  use the point-local weights; alpha does not depend on the spacing for the
  heat and wave equations, and for Hamilton-Jacobi ``dxs[ax]`` is the
  smallest cell width of the axis (dt = CFL min_d dx_d / c_d and
  alpha = beta/(CFL min dx) as on uniform grids).
"""
import itertools

import numpy as np

from . import nonuniform
from .sweep import partial_sum, BC_PERIODIC

# 3-stage SSP RK in Shu-Osher form: u_s = a0 u^n + a1 (u_{s-1} + dt F(u_{s-1}))
SSPRK3 = ((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0))


def axis_sum(u, ax, alpha, dx, op, bc, npts, P, weights="linear", weight_fn=None, grids=None):
    """S_P along array axis ``ax``: uniform spacing dx, or the nodes of a
    non-uniform axis (grids[ax] = (x, L))."""
    g = grids[ax] if grids is not None else None
    if g is None:
        return partial_sum(u, ax, alpha, dx, op, bc, npts, P, weights, weight_fn)
    if weight_fn is not None:
        raise ValueError("learned weights run on uniform axes")
    return nonuniform.partial_sum_axis(u, ax, g[0], g[1], alpha, op, npts, P, weights)


def heat_rhs_dt(u, dxs, dt, kappa, beta, bc, npts, P, grids=None):
    """dt * F(u) = -kappa alpha^2 dt sum_d S_{P,d}[u] = -beta^2 sum_d S_{P,d}[u]."""
    alpha = beta / np.sqrt(kappa * dt)
    acc = np.zeros_like(u)
    for ax in range(u.ndim):
        acc += axis_sum(u, ax, alpha, dxs[ax], "0", bc[ax], npts, P, grids=grids)
    return -kappa * alpha * alpha * dt * acc


def heat_step(u, dxs, dt, kappa=1.0, beta=0.6, bc=None, npts=3, P=3, grids=None):
    """One SSP-RK3 step of the heat equation."""
    bc = bc or [BC_PERIODIC] * u.ndim
    un = np.asarray(u, dtype=np.float64)
    us = un
    for a0, a1 in SSPRK3:
        us = a0 * un + a1 * (us + heat_rhs_dt(us, dxs, dt, kappa, beta, bc, npts, P, grids))
    return us


def wave_step(u, u_prev, dxs, dt, c=1.0, beta=0.8, bc=None, npts=6, P=2, from_rest=False, grids=None):
    """One step of the wave equation; returns u^{n+1}."""
    bc = bc or [BC_PERIODIC] * u.ndim
    alpha = beta / (c * dt)
    S = np.zeros_like(u, dtype=np.float64)
    for ax in range(u.ndim):
        S += axis_sum(u, ax, alpha, dxs[ax], "0", bc[ax], npts, P, grids=grids)
    # c^2 dt^2 d_xx ~ -c^2 dt^2 alpha^2 S = -beta^2 S
    if from_rest:
        return u - 0.5 * beta * beta * S
    return 2.0 * u - u_prev - beta * beta * S


def hj_derivatives(u, alpha, dxs, npts=5, weights="wenoz", weight_fn=None, P=1, grids=None):
    """(v_d^-, v_d^+) for every axis d: v^- = alpha sum_{p<=P} D_R^p[u],
    v^+ = -alpha sum_{p<=P} D_L^p[u] (Sec. 2.5; P = 1 for forward Euler)."""
    out = []
    for ax in range(u.ndim):
        dm = alpha * axis_sum(u, ax, alpha, dxs[ax], "R", BC_PERIODIC, npts, P, weights, weight_fn, grids)
        dp = -alpha * axis_sum(u, ax, alpha, dxs[ax], "L", BC_PERIODIC, npts, P, weights, weight_fn, grids)
        out.append((dm, dp))
    return out


H_HALF_SQ, H_LINEAR, H_AFFINE_SQ = "half_sq", "linear", "affine_sq"


def hamiltonian(kind, p, a=None, h0=0.0):
    """H(p) for the gradient components p[d]: |p|^2/2, a.p, or (h0 + a.p)^2/2
    (d and a[d] follow the array axes, as everywhere in the oracle)."""
    if kind == H_HALF_SQ:
        return 0.5 * sum(pd * pd for pd in p)
    s = sum(a[d] * pd for d, pd in enumerate(p))
    if kind == H_LINEAR:
        return s
    return 0.5 * (h0 + s) ** 2


def hamiltonian_grad(kind, p, a=None, h0=0.0):
    """[dH/dp_d] for the same Hamiltonians."""
    if kind == H_HALF_SQ:
        return list(p)
    if kind == H_LINEAR:
        return [a[d] + 0.0 * p[d] for d in range(len(p))]
    s = h0 + sum(a[d] * pd for d, pd in enumerate(p))
    return [a[d] * s for d in range(len(p))]


def llf_r(ders, kind=H_HALF_SQ, a=None, h0=0.0):
    """r_d = max over the corners of the box prod_d I(v_d^-, v_d^+) of |dH/dp_d|."""
    nd = len(ders)
    r = [np.zeros_like(np.asarray(ders[0][0], dtype=np.float64)) for _ in range(nd)]
    for corner in itertools.product((0, 1), repeat=nd):
        p = [ders[d][corner[d]] for d in range(nd)]
        g = hamiltonian_grad(kind, p, a, h0)
        for d in range(nd):
            r[d] = np.maximum(r[d], np.abs(g[d]))
    return r


def hj_hamiltonian(ders, kind=H_HALF_SQ, a=None, h0=0.0):
    """Local Lax-Friedrichs numerical Hamiltonian (Sec. 2.5)
        H^ = H(means) - sum_d r_d (v_d^+ - v_d^-)/2,
    r_d from ``llf_r``, and the per-axis wave speeds c_d = max_grid r_d
    (Sec. 4.4)."""
    means = [0.5 * (dm + dp) for dm, dp in ders]
    Hh = hamiltonian(kind, means, a, h0)
    r = llf_r(ders, kind, a, h0)
    speeds = []
    for d, (dm, dp) in enumerate(ders):
        Hh = Hh - r[d] * 0.5 * (dp - dm)
        speeds.append(float(r[d].max()))
    return Hh, speeds


def source_at(coefs, t):
    """F(x, t) = sum_k t^k F_k(x)."""
    return sum((t ** k) * F for k, F in enumerate(coefs))


def hj_dt(speeds, dxs, cfl):
    """dt = CFL * min_d dx_d / c_d (Eq. "adaptive time rule"), capped at 10 dx."""
    cands = [cfl * dx / c for dx, c in zip(dxs, speeds) if c > 0.0]
    cap = 10.0 * min(dxs)
    return min(cands + [cap])


def hj_initial_speeds(u, dxs, cfl=1.5, beta=1.0, npts=5, weights="wenoz", weight_fn=None,
                      hamiltonian=H_HALF_SQ, a=None, h0=0.0, grids=None):
    alpha = beta / (cfl * min(dxs))
    _, speeds = hj_hamiltonian(hj_derivatives(u, alpha, dxs, npts, weights, weight_fn, 1, grids), hamiltonian, a,
                               h0)
    return speeds


def hj_step(u, dxs, lagged_speeds, cfl=1.5, beta=1.0, npts=5, weights="wenoz", weight_fn=None,
            hamiltonian=H_HALF_SQ, a=None, h0=0.0, source=None, t=0.0, grids=None):
    """One forward-Euler step u^{n+1} = u^n - dt^n (H^ - F(., t)); returns
    (u^{n+1}, dt^n, speeds of u^n) -- the speeds become the lagged speeds of
    the next step (Algorithm 1).  source: the coefficients F_k of F."""
    alpha = beta / (cfl * min(dxs))
    dt = hj_dt(lagged_speeds, dxs, cfl)
    Hh, speeds = hj_hamiltonian(hj_derivatives(u, alpha, dxs, npts, weights, weight_fn, 1, grids), hamiltonian, a,
                                h0)
    if source is not None:
        Hh = Hh - source_at(source, t)
    return u - dt * Hh, dt, speeds


def heat_euler_step(u, dxs, dt, kappa=1.0, beta=1.0, bc=None, npts=6, P=1, grids=None):
    """One forward-Euler step of the heat equation (Sec. 5.1, Example 2)."""
    bc = bc or [BC_PERIODIC] * u.ndim
    un = np.asarray(u, dtype=np.float64)
    return un + heat_rhs_dt(un, dxs, dt, kappa, beta, bc, npts, P, grids)


# ---------------------------------------------------------------- advection-diffusion
# Sec. 2.5: u_t + sum_d d_d g(u) = kappa Lap u, the flux split by global
# Lax-Friedrichs, g = g^+ + g^-, g^{+-} = (g(u) +- c u)/2 with c >= max |g'(u)|
# (reading: the paper's r = max g1' taken as a bound c given with the
# problem, so the operators' alpha stays fixed), the upwind derivatives
# d^- g^+ = alpha sum_p D_R^p[g^+] and d^+ g^- = -alpha sum_p D_L^p[g^-]
# (Sec. 2.2), alpha = beta/(c dt), and the diffusion -kappa alpha_nu^2
# sum_p D_0^p[u] with alpha_nu = beta/sqrt(kappa dt).  Hence
#   dt F(u) = -(beta/c) sum_d (S_R[g_d^+] - S_L[g_d^-]) - beta^2 sum_d S_0[u].
FLUX_LINEAR, FLUX_BURGERS = "linear", "burgers"


def flux(kind, u, a=1.0):
    """g(u): a u (linear) or u^2/2 (Burgers)."""
    return a * u if kind == FLUX_LINEAR else 0.5 * u * u


def advdiff_rhs_dt(u, dxs, dt, kind, a, c, kappa, beta, npts, P, bc=None, weights="linear", grids=None):
    """dt * F(u); a[d] per array axis (linear flux), c the splitting bound;
    weights: the local-quadrature weights of every sweep (linear or WENO-Z);
    grids: non-uniform axes as for the heat and wave steps."""
    bc = bc or [BC_PERIODIC] * u.ndim
    alpha = beta / (c * dt)
    out = np.zeros_like(u)
    for ax in range(u.ndim):
        g = flux(kind, u, a[ax] if kind == FLUX_LINEAR else 1.0)
        gp = 0.5 * (g + c * u)
        gm = 0.5 * (g - c * u)
        dminus = alpha * axis_sum(gp, ax, alpha, dxs[ax], "R", bc[ax], npts, P, weights, grids=grids)
        dplus = -alpha * axis_sum(gm, ax, alpha, dxs[ax], "L", bc[ax], npts, P, weights, grids=grids)
        out = out - dt * (dminus + dplus)
    if kappa > 0:
        an = beta / np.sqrt(kappa * dt)
        for ax in range(u.ndim):
            out = out - kappa * dt * an * an * axis_sum(u, ax, an, dxs[ax], "0", bc[ax], npts, P, weights,
                                                        grids=grids)
    return out


def advdiff_step(u, dxs, dt, kind, a, c, kappa=0.0, beta=1.0, npts=6, P=1, rk3=False, weights="linear",
                 grids=None):
    """One step: forward Euler, or the 3-stage SSP Runge-Kutta method (Shu-Osher form)."""
    un = np.asarray(u, dtype=np.float64)
    if not rk3:
        return un + advdiff_rhs_dt(un, dxs, dt, kind, a, c, kappa, beta, npts, P, None, weights, grids)
    us = un
    for a0, a1 in SSPRK3:
        us = a0 * un + a1 * (us + advdiff_rhs_dt(us, dxs, dt, kind, a, c, kappa, beta, npts, P, None, weights,
                                                 grids))
    return us


def hj_step_rk3(u, dxs, lagged_speeds, t=0.0, cfl=1.5, beta=1.0, npts=5, weights="wenoz", P=3,
                hamiltonian=H_HALF_SQ, a=None, h0=0.0, source=None, grids=None):
    """One step of the 3-stage SSP Runge-Kutta method on u_t = -H^ + F with
    P-term one-sided sums (Sec. 2.5: an s-stage method with s-term sums):
        u1 = u + dt L(u, t), u2 = 3/4 u + 1/4 (u1 + dt L(u1, t + dt)),
        u^{n+1} = 1/3 u + 2/3 (u2 + dt L(u2, t + dt/2)),  L = -(H^ - F).
    dt from the lagged speeds (Algorithm 1) for the whole step; returns
    (u^{n+1}, dt, speeds of u^n)."""
    alpha = beta / (cfl * min(dxs))
    dt = hj_dt(lagged_speeds, dxs, cfl)
    stage_t = (t, t + dt, t + 0.5 * dt)
    un = np.asarray(u, dtype=np.float64)
    us, speeds0 = un, None
    for (a0, a1), ts in zip(SSPRK3, stage_t):
        Hh, sp = hj_hamiltonian(hj_derivatives(us, alpha, dxs, npts, weights, None, P, grids), hamiltonian, a, h0)
        if speeds0 is None:
            speeds0 = sp
        if source is not None:
            Hh = Hh - source_at(source, ts)
        us = a0 * un + a1 * (us - dt * Hh)
    return us, dt, speeds0


def hj_initial_speeds_P(u, dxs, cfl=1.5, beta=1.0, npts=5, weights="wenoz", P=3, hamiltonian=H_HALF_SQ, a=None,
                        h0=0.0, grids=None):
    """Speeds of u^0 with P-term one-sided sums (the first step's lagged speeds)."""
    alpha = beta / (cfl * min(dxs))
    _, speeds = hj_hamiltonian(hj_derivatives(u, alpha, dxs, npts, weights, None, P, grids), hamiltonian, a, h0)
    return speeds
