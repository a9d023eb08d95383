"""Oracle: exact discrete Fourier symbols of the periodic operators.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__``.

For a periodic uniform line and the mode v_j = e^{i j theta}, the local
integrals (Sec. 2.4) and the recurrences with the periodic constants
(Sec. 2.3) give exactly

    L_R^{-1} v = lambda_R v,  lambda_R = Jhat_R / (1 - q e^{-i theta}),
    Jhat_R(theta) = sum_l c_l e^{i l theta},
    L_L^{-1} v = lambda_L v,  lambda_L = Jhat_L / (1 - q e^{+i theta}),
    Jhat_L(theta) = sum_l c_l e^{-i l theta},
    L_0^{-1} = (L_L^{-1} + L_R^{-1})/2,

(the periodic sum over images, q = e^{-nu}).  D has symbol 1 - lambda and the
partial sum S_P has symbol sum_{p=1}^P (1 - lambda)^p.  The bound on beta
follows from requiring the scheme's amplification to stay in the stability
region of the integrator for every resolved mode (Sec. 2.5 states
unconditional stability for linear problems with RK up to order 3 for the
paper's choice of alpha; with the additive multi-dimensional coupling used
here the bound on beta below is what keeps that property).
"""
import numpy as np

from .quadrature import local_weights, STENCIL


def symbol(theta, nu, op, npts):
    c = local_weights(nu, STENCIL[npts])
    offs = np.array(STENCIL[npts], dtype=np.float64)
    q = np.exp(-nu)
    th = np.asarray(theta, dtype=np.float64)[..., None]
    JR = np.sum(c * np.exp(1j * offs * th), axis=-1)
    JL = np.sum(c * np.exp(-1j * offs * th), axis=-1)
    t = np.asarray(theta, dtype=np.float64)
    lamR = JR / (1.0 - q * np.exp(-1j * t))
    lamL = JL / (1.0 - q * np.exp(1j * t))
    if op == "R":
        return lamR
    if op == "L":
        return lamL
    return 0.5 * (lamL + lamR)


def partial_sum_symbol(theta, nu, op, npts, P):
    d = 1.0 - symbol(theta, nu, op, npts)
    return sum(d ** p for p in range(1, P + 1))


def rk3_real_limit():
    """Left end of the real interval of the 3-stage, third-order RK stability
    region: the real root of 1 + z + z^2/2 + z^3/6 = -1."""
    roots = np.roots([1.0 / 6.0, 0.5, 1.0, 2.0])
    return float(min(r.real for r in roots if abs(r.imag) < 1e-12))


def beta_max(nu_of_beta, ndim, npts, P, integrator, ntheta=4097, iters=60):
    """Largest beta with  beta^2 * ndim * max_theta S_P(theta) <= limit,
    limit = |rk3_real_limit()| (heat, SSP-RK3) or 4 (wave, leapfrog); nu
    depends on beta through ``nu_of_beta``.  Found by bisection."""
    limit = abs(rk3_real_limit()) if integrator == "rk3" else 4.0
    th = np.linspace(0.0, np.pi, ntheta)

    def ok(beta):
        s = partial_sum_symbol(th, nu_of_beta(beta), "0", npts, P).real
        return s.min() >= -1e-14 and beta * beta * ndim * s.max() <= limit

    lo, hi = 1e-3, 4.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if ok(mid):
            lo = mid
        else:
            hi = mid
    return lo
