"""Oracle: weights of the local integrals J_R, J_L (Sec. 2.4, App. C).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__``.

With nu = alpha*dx and the substitution s = x_i + t*dx, t in [-1, 0], the
right-moving local integral of Eq. (JR),

    J_R(x_i) = alpha * int_{x_{i-1}}^{x_i} exp(-alpha (x_i - s)) p(s) ds,

becomes nu * int_{-1}^{0} exp(nu t) p(x_i + t dx) dt.  Writing the interpolant
p through the stencil nodes x_{i+l} (l in the offset set) in the Lagrange
basis gives J_R(x_i) = sum_l c_l v_{i+l} with

    c_l(nu) = nu * int_{-1}^{0} exp(nu t) ell_l(t) dt           (Eq. 2.4.1/2)

This module evaluates that integral directly by Gauss-Legendre quadrature of
the Lagrange basis polynomial times the exponential -- never through the
closed forms of App. C, so small nu costs no accuracy.  J_L uses the same
weights on the mirrored stencil (App. C, "mirror-symmetry").

Stencils (offsets l relative to x_i for J_R on the cell [x_{i-1}, x_i]):
  * 6 points {-3..2} with cubic substencils {-3..0},{-2..1},{-1..2}: Sec. 2.4.
  * 5 points {-3..1} with quadratic substencils {-3..-1},{-2..0},{-1..1}, and
  * 3 points {-1,0,1}: not printed in the paper; built by the same
    construction (reading: the upwind-biased 5-point set, and the centred
    3-point set whose discrete D_0 symbol stays inside [0, 1]).
"""
import numpy as np
from numpy.polynomial import polynomial as npoly

STENCIL = {
    6: (-3, -2, -1, 0, 1, 2),
    5: (-3, -2, -1, 0, 1),
    3: (-1, 0, 1),
}
SUBSTENCILS = {
    6: ((-3, -2, -1, 0), (-2, -1, 0, 1), (-1, 0, 1, 2)),
    5: ((-3, -2, -1), (-2, -1, 0), (-1, 0, 1)),
}
# WENO-Z constant (Sec. 2.4, commented WENO-Z step): eps = 1e-6.
WENOZ_EPS = 1e-6

_GL_X, _GL_W = np.polynomial.legendre.leggauss(48)
# map [-1, 1] -> [-1, 0]
_T = 0.5 * (_GL_X - 1.0)
_WT = 0.5 * _GL_W


def lagrange_basis(nodes, j):
    """Monomial coefficients (ascending) of the Lagrange basis polynomial
    ell_j on ``nodes`` (ell_j(nodes[m]) = delta_jm)."""
    roots = [n for m, n in enumerate(nodes) if m != j]
    c = npoly.polyfromroots(roots)
    return c / npoly.polyval(nodes[j], c)


def local_weights(nu, offsets):
    """c_l(nu) = nu * int_{-1}^0 e^{nu t} ell_l(t) dt for each offset l
    (Eq. for J_R^{(r)} / J_R on the large stencil, Sec. 2.4)."""
    nodes = [float(o) for o in offsets]
    e = np.exp(nu * _T)
    return np.array([nu * np.sum(_WT * e * npoly.polyval(_T, lagrange_basis(nodes, j)))
                     for j in range(len(nodes))])


def linear_weights(nu, npts):
    """Linear weights d_r with sum_r d_r J^{(r)} = J on the large stencil
    (Eq. "WENO linear weights", Sec. 2.4).

    Solved as the (consistent, overdetermined) linear system that matches the
    weight of every large-stencil node; the residual is asserted to vanish.
    Reading: App. C prints d_0 with a garbled numerator; this definition is
    the one Sec. 2.4 states, and it reproduces the printed d_2 exactly.
    """
    big = local_weights(nu, STENCIL[npts])
    subs = SUBSTENCILS[npts]
    m = len(subs[0])
    M = np.zeros((len(big), len(subs)))
    for r, s in enumerate(subs):
        M[r:r + m, r] = local_weights(nu, s)
    d, *_ = np.linalg.lstsq(M, big, rcond=None)
    resid = np.abs(M @ d - big).max()
    assert resid < 1e-13 * max(1.0, np.abs(big).max()), resid
    return d


def smoothness_matrix(offsets, orders):
    """Symmetric matrix M with beta(v) = v^T M v, where

        beta = sum_{l in orders} int_{x_{i-1}}^{x_i} dx^{2l-1} (d^l p / dx^l)^2 dx
             = sum_{l in orders} int_{-1}^{0} (d^l p / dt^l)^2 dt

    for the interpolant p through ``offsets`` (smoothness indicator of the
    commented WENO step, Sec. 2.4).  Reading: orders (2, 3) for the cubic
    substencils -- this reproduces the closed forms printed (commented) in
    App. C -- and orders (1, 2) for quadratic substencils (Jiang-Shu form).
    Integrals of polynomials are exact under the 48-point rule.
    """
    nodes = [float(o) for o in offsets]
    n = len(nodes)
    M = np.zeros((n, n))
    for l in orders:
        ders = [npoly.polyval(_T, npoly.polyder(lagrange_basis(nodes, j), l)) for j in range(n)]
        for a in range(n):
            for b in range(n):
                M[a, b] += np.sum(_WT * ders[a] * ders[b])
    return M


def smoothness_orders(npts):
    return (2, 3) if npts == 6 else (1, 2)


class QuadratureRule:
    """All per-(nu, stencil) constants the oracle needs for one axis."""

    def __init__(self, nu, npts):
        if npts not in STENCIL:
            raise ValueError("quadrature points must be 3, 5 or 6")
        self.nu = float(nu)
        self.npts = npts
        self.offsets = STENCIL[npts]
        self.c = local_weights(nu, self.offsets)
        if npts in SUBSTENCILS:
            self.sub_offsets = SUBSTENCILS[npts]
            self.sub_c = [local_weights(nu, s) for s in self.sub_offsets]
            self.d = linear_weights(nu, npts)
            orders = smoothness_orders(npts)
            self.beta_M = [smoothness_matrix(s, orders) for s in self.sub_offsets]
        else:
            self.sub_offsets = None
