"""Oracle: the fast summation on non-uniform periodic lines.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__``.

The paper builds its quadrature for uniform grids and notes (Sec. 2.4) that
on a non-uniform mesh the weights become local to each point and are
computed for it.  This module writes that case out from the definitions:

* nodes x_0 < ... < x_{n-1} of one period [a, a + L); x_{j+n} = x_j + L;
* J_R(x_i) = alpha int_{x_{i-1}}^{x_i} e^{-alpha (x_i - s)} p_i(s) ds with p_i
  the interpolant through the nodes x_{i+l}, l in the J_R stencil (Sec. 2.4),
  so J_R(x_i) = sum_l c_{i,l} v_{i+l},
  c_{i,l} = alpha int_{x_{i-1}}^{x_i} e^{-alpha (x_i - s)} ell_{i,l}(s) ds;
* J_L(x_i) = alpha int_{x_i}^{x_{i+1}} e^{-alpha (s - x_i)} p~_i(s) ds on the
  mirrored stencil x_{i-l};
* recurrences with the cell decays q_i = e^{-alpha (x_i - x_{i-1})}:
  I_R(x_i) = q_i I_R(x_{i-1}) + J_R(x_i), I_L(x_i) = q_{i+1} I_L(x_{i+1}) + J_L(x_i);
* periodicity (Sec. 2.3): the images of every period add the constants that
  make I_R and I_L periodic; one period's partial sums I^0 close with
  mu = prod_i q_i = e^{-alpha L}: I_R(x_{-1}) = I_R^0(x_{n-1}) / (1 - mu);
* L_R^{-1} = I_R, L_L^{-1} = I_L, L_0^{-1} = (I_L + I_R)/2, D = I - L^{-1},
  S_P = sum_{p<=P} D^p (Sec. 2.1-2.2).

The integrals are evaluated by Gauss-Legendre quadrature of the Lagrange
basis times the exponential (48 points per cell).
"""
import numpy as np
from numpy.polynomial import polynomial as npoly

from .quadrature import STENCIL, lagrange_basis

_GL_X, _GL_W = np.polynomial.legendre.leggauss(48)


def _node(x, L, j):
    n = len(x)
    k, r = divmod(j, n)
    return x[r] + k * L


def weights(x, L, alpha, npts):
    """(cR, cL, q): per point i the J_R weights on nodes x_{i+l}, the J_L
    weights on nodes x_{i-l} (l in the J_R stencil), and q_i."""
    n = len(x)
    offs = STENCIL[npts]
    cR = np.zeros((n, len(offs)))
    cL = np.zeros((n, len(offs)))
    q = np.zeros(n)
    for i in range(n):
        xi = x[i]
        a, b = _node(x, L, i - 1), xi
        q[i] = np.exp(-alpha * (b - a))
        s = 0.5 * (b - a) * _GL_X + 0.5 * (b + a)
        w = 0.5 * (b - a) * _GL_W * alpha * np.exp(-alpha * (xi - s))
        nodes = [_node(x, L, i + l) - xi for l in offs]
        for m in range(len(offs)):
            cR[i, m] = np.sum(w * npoly.polyval(s - xi, lagrange_basis(nodes, m)))
        a, b = xi, _node(x, L, i + 1)
        s = 0.5 * (b - a) * _GL_X + 0.5 * (b + a)
        w = 0.5 * (b - a) * _GL_W * alpha * np.exp(-alpha * (s - xi))
        nodes = [_node(x, L, i - l) - xi for l in offs]
        for m in range(len(offs)):
            cL[i, m] = np.sum(w * npoly.polyval(s - xi, lagrange_basis(nodes, m)))
    return cR, cL, q


def inverse(v, x, L, alpha, op, npts, tables=None):
    """L_op^{-1}[v] on one periodic non-uniform line (op in R, L, 0)."""
    n = len(x)
    cR, cL, q = tables if tables is not None else weights(x, L, alpha, npts)
    offs = STENCIL[npts]
    JR = np.array([sum(cR[i, m] * v[(i + l) % n] for m, l in enumerate(offs)) for i in range(n)])
    JL = np.array([sum(cL[i, m] * v[(i - l) % n] for m, l in enumerate(offs)) for i in range(n)])
    mu = np.prod(q)
    IR = np.zeros(n)
    acc = 0.0
    for i in range(n):
        acc = q[i] * acc + JR[i]
        IR[i] = acc
    xR = IR[-1] / (1.0 - mu)               # I_R at x_{-1}, the previous period's last node
    acc = xR
    for i in range(n):
        acc = q[i] * acc + JR[i]
        IR[i] = acc
    IL = np.zeros(n)
    acc = 0.0
    for i in range(n - 1, -1, -1):
        acc = q[(i + 1) % n] * acc + JL[i]
        IL[i] = acc
    xL = IL[0] / (1.0 - mu)                # I_L at x_n, the next period's first node
    acc = xL
    for i in range(n - 1, -1, -1):
        acc = q[(i + 1) % n] * acc + JL[i]
        IL[i] = acc
    if op == "R":
        return IR
    if op == "L":
        return IL
    return 0.5 * (IL + IR)


def partial_sum(v, x, L, alpha, op, npts, P):
    """S_P = sum_{p<=P} D^p[v] on one periodic non-uniform line."""
    tables = weights(x, L, alpha, npts)
    S = np.zeros(len(x))
    w = np.asarray(v, dtype=np.float64)
    for _ in range(P):
        w = w - inverse(w, x, L, alpha, op, npts, tables)
        S = S + w
    return S
