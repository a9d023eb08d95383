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

WENO-Z on non-uniform lines (Sec. 2.4: the linear weights become local to
each point): per point i and direction, the substencil rules c^{(r)} on the
substencils S_r of the J_R stencil (mirrored for J_L), the linear weights d_r
with sum_r d_r c^{(r)} = c (the large-stencil rule at that point), and the
smoothness indicators of the commented WENO step,

    beta_r = sum_l dx_i^{2l-1} int_cell (d^l p_r / ds^l)^2 ds,

with dx_i the width of the integration cell (x_i - x_{i-1} for J_R,
x_{i+1} - x_i for J_L) -- on a uniform grid this is the uniform indicator.
The WENO-Z map (eps = 1e-6) then weights the J^{(r)} as on uniform grids.

Dirichlet lines (Sec. 2.3; pass L = None): the nodes x_0 = a < ... < x_N = b
include both boundary nodes (N >= 3).  Stencils reach ghost nodes mirrored
about the ends, x_{-j} = 2a - x_j and x_{N+j} = 2b - x_{N-j}, holding the odd
reflection of the data about the boundary values, v_{-j} = 2 v_0 - v_j and
v_{N+j} = 2 v_N - v_{N-j} (the readings of the uniform oracle with the
actual node positions).  The recurrences start from I_R(x_0) = 0 and
I_L(x_N) = 0, and the boundary constants are fixed by the boundary values:
A = v(a) for L_R, B = v(b) for L_L, and for L_0 the 2x2 system
[[1, mu], [mu, 1]] (A, B) = (v_0 - I_0(a), v_N - I_0(b)), mu = e^{-alpha (b - a)}.
"""
import numpy as np
from numpy.polynomial import polynomial as npoly

from .quadrature import STENCIL, SUBSTENCILS, WENOZ_EPS, lagrange_basis, smoothness_orders

_GL_X, _GL_W = np.polynomial.legendre.leggauss(48)


def _node(x, L, j):
    """x_j for any j: periodic images (period L), or for a Dirichlet line
    (L None) the ghost nodes mirrored about the ends."""
    n = len(x)
    if L is None:
        N = n - 1
        if j < 0:
            return 2.0 * x[0] - x[-j]
        if j > N:
            return 2.0 * x[N] - x[2 * N - j]
        return x[j]
    k, r = divmod(j, n)
    return x[r] + k * L


def _value(v, L, j):
    """v_j for any j: periodic wrap, or (L None) odd reflection about the
    boundary values."""
    n = len(v)
    if L is None:
        N = n - 1
        if j < 0:
            return 2.0 * v[0] - v[-j]
        if j > N:
            return 2.0 * v[N] - v[2 * N - j]
        return v[j]
    return v[j % n]


def _cell(x, L, i, side):
    """(a, b, sign): the integration cell of J_R (side R: [x_{i-1}, x_i],
    nodes x_{i+l}) or J_L (side L: [x_i, x_{i+1}], nodes x_{i-l})."""
    if side == "R":
        return _node(x, L, i - 1), x[i], 1
    return x[i], _node(x, L, i + 1), -1


def _cell_rule(x, L, alpha, i, side, offs):
    """alpha int_cell e^{-alpha |s - x_i|} ell_m(s) ds for the Lagrange basis
    on the nodes of ``offs`` (Eqs. "JR", "JL" with p the interpolant)."""
    a, b, sign = _cell(x, L, i, side)
    xi = x[i]
    s = 0.5 * (b - a) * _GL_X + 0.5 * (b + a)
    w = 0.5 * (b - a) * _GL_W * alpha * np.exp(-alpha * np.abs(s - xi))
    nodes = [_node(x, L, i + sign * l) - xi for l in offs]
    return np.array([np.sum(w * npoly.polyval(s - xi, lagrange_basis(nodes, m))) for m in range(len(offs))])


def weights(x, L, alpha, npts):
    """(cR, cL, q): per point i the J_R weights on nodes x_{i+l}, the J_L
    weights on nodes x_{i-l} (l in the J_R stencil), and q_i."""
    n = len(x)
    offs = STENCIL[npts]
    cR = np.zeros((n, len(offs)))
    cL = np.zeros((n, len(offs)))
    q = np.zeros(n)
    for i in range(n):
        q[i] = np.exp(-alpha * (x[i] - _node(x, L, i - 1)))
        cR[i] = _cell_rule(x, L, alpha, i, "R", offs)
        cL[i] = _cell_rule(x, L, alpha, i, "L", offs)
    return cR, cL, q


def _smoothness_matrix(x, L, i, side, offs, orders):
    """M with beta = v^T M v: sum_l dx^{2l-1} int_cell ell_a^{(l)} ell_b^{(l)} ds
    over the cell of x_i on the given side, in physical coordinates."""
    a, b, sign = _cell(x, L, i, side)
    xi = x[i]
    dx = b - a
    s = 0.5 * (b - a) * _GL_X + 0.5 * (b + a) - xi
    w = 0.5 * (b - a) * _GL_W
    nodes = [_node(x, L, i + sign * l) - xi for l in offs]
    m = len(offs)
    M = np.zeros((m, m))
    for l in orders:
        ders = [npoly.polyval(s, npoly.polyder(lagrange_basis(nodes, j), l)) for j in range(m)]
        for p in range(m):
            for r in range(m):
                M[p, r] += dx ** (2 * l - 1) * np.sum(w * ders[p] * ders[r])
    return M


def weno_tables(x, L, alpha, npts):
    """Per side ('R', 'L') a dict of the point-local WENO constants:
    sub (n, 3, m) substencil rules, d (n, 3) linear weights, M (n, 3, m, m)
    smoothness matrices (npts 5: quadratic substencils; 6: cubic)."""
    n = len(x)
    subs = SUBSTENCILS[npts]
    offs = STENCIL[npts]
    m = len(subs[0])
    orders = smoothness_orders(npts)
    out = {}
    for side in "RL":
        sub = np.zeros((n, 3, m))
        d = np.zeros((n, 3))
        Ms = np.zeros((n, 3, m, m))
        for i in range(n):
            big = _cell_rule(x, L, alpha, i, side, offs)
            A = np.zeros((len(offs), 3))
            for r, so in enumerate(subs):
                sub[i, r] = _cell_rule(x, L, alpha, i, side, so)
                A[r:r + m, r] = sub[i, r]
                Ms[i, r] = _smoothness_matrix(x, L, i, side, so, orders)
            # sum_r d_r c^{(r)} = c on every node of the large stencil
            # (consistent: the system is exact on data of the substencil degree)
            d[i], *_ = np.linalg.lstsq(A, big, rcond=None)
            resid = np.abs(A @ d[i] - big).max()
            assert resid < 1e-12 * max(1.0, np.abs(big).max()), resid
        out[side] = {"sub": sub, "d": d, "M": Ms}
    return out


def weno_weights_at(vals, d, Ms):
    """WENO-Z nonlinear weights (commented WENO-Z step of Sec. 2.4) of one
    point from its stencil values ``vals`` (large-stencil order)."""
    m = Ms.shape[-1]
    beta = np.array([vals[r:r + m] @ Ms[r] @ vals[r:r + m] for r in range(3)])
    tau = abs(beta[0] - beta[2])
    wt = d * (1.0 + tau / (WENOZ_EPS + beta))
    return wt / wt.sum()


def local_integrals(v, x, L, alpha, npts, weights_kind="linear", tables=None):
    """(J_R, J_L) at every point: the large-stencil rule (linear) or the
    WENO-Z combination of the substencil rules (wenoz)."""
    n = len(x)
    offs = STENCIL[npts]
    if weights_kind == "linear":
        cR, cL, _ = tables if tables is not None else weights(x, L, alpha, npts)
        JR = np.array([sum(cR[i, m] * _value(v, L, i + l) for m, l in enumerate(offs)) for i in range(n)])
        JL = np.array([sum(cL[i, m] * _value(v, L, i - l) for m, l in enumerate(offs)) for i in range(n)])
        return JR, JL
    if weights_kind != "wenoz":
        raise ValueError(weights_kind)
    wt = tables if tables is not None else weno_tables(x, L, alpha, npts)
    m = wt["R"]["sub"].shape[-1]
    J = {}
    for side, sign in (("R", 1), ("L", -1)):
        t = wt[side]
        out = np.zeros(n)
        for i in range(n):
            vals = np.array([_value(v, L, i + sign * l) for l in offs])
            om = weno_weights_at(vals, t["d"][i], t["M"][i])
            out[i] = sum(om[r] * (t["sub"][i, r] @ vals[r:r + m]) for r in range(3))
        J[side] = out
    return J["R"], J["L"]


def inverse(v, x, L, alpha, op, npts, tables=None, weights_kind="linear", weno=None):
    """L_op^{-1}[v] on one non-uniform line (op in R, L, 0): periodic with
    period L, or Dirichlet (L None)."""
    n = len(x)
    if L is None and n < 4:
        raise ValueError("a Dirichlet line needs at least 4 nodes")
    cR, cL, q = tables if tables is not None else weights(x, L, alpha, npts)
    JR, JL = local_integrals(v, x, L, alpha, npts, weights_kind,
                             (cR, cL, q) if weights_kind == "linear" else weno)
    if L is None:
        return _inverse_dirichlet(np.asarray(v, dtype=np.float64), np.asarray(x, dtype=np.float64), alpha, op,
                                  JR, JL, q)
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


def _inverse_dirichlet(v, x, alpha, op, JR, JL, q):
    """Recurrences from I_R(x_0) = 0 and I_L(x_N) = 0, then the boundary
    constants from the boundary values (Sec. 2.3, the 2x2 algebra of Sec. 3.3)."""
    N = len(x) - 1
    IR = np.zeros(N + 1)
    for i in range(1, N + 1):
        IR[i] = q[i] * IR[i - 1] + JR[i]
    IL = np.zeros(N + 1)
    for i in range(N - 1, -1, -1):
        IL[i] = q[i + 1] * IL[i + 1] + JL[i]
    ea = np.exp(-alpha * (x - x[0]))      # e^{-alpha (x_i - a)}
    eb = np.exp(-alpha * (x[N] - x))      # e^{-alpha (b - x_i)}
    mu = np.exp(-alpha * (x[N] - x[0]))
    if op == "R":
        return IR + v[0] * ea
    if op == "L":
        return IL + v[N] * eb
    I0 = 0.5 * (IL + IR)
    r0, r1 = v[0] - I0[0], v[N] - I0[N]
    A = (r0 - mu * r1) / (1.0 - mu * mu)
    B = (r1 - mu * r0) / (1.0 - mu * mu)
    return I0 + A * ea + B * eb


def partial_sum(v, x, L, alpha, op, npts, P, weights_kind="linear", tables=None, weno=None):
    """S_P = sum_{p<=P} D^p[v] on one non-uniform line, periodic or (L None)
    Dirichlet (``tables``, ``weno``: the line's weights() / weno_tables(),
    built when not given)."""
    if tables is None:
        tables = weights(x, L, alpha, npts)
    if weights_kind == "wenoz" and weno is None:
        weno = weno_tables(x, L, alpha, npts)
    S = np.zeros(len(x))
    w = np.asarray(v, dtype=np.float64)
    for _ in range(P):
        w = w - inverse(w, x, L, alpha, op, npts, tables, weights_kind, weno)
        S = S + w
    return S


def partial_sum_axis(u, ax, x, L, alpha, op, npts, P, weights_kind="linear"):
    """S_P along axis ``ax`` of an n-D array whose lines along that axis have
    the nodes x (period L, or L None for Dirichlet lines); every line is
    independent (dimensional splitting, Sec. 2.2)."""
    tables = weights(x, L, alpha, npts)
    weno = weno_tables(x, L, alpha, npts) if weights_kind == "wenoz" else None
    um = np.moveaxis(np.asarray(u, dtype=np.float64), ax, -1)
    out = np.empty_like(um)
    for idx in np.ndindex(um.shape[:-1]):
        out[idx] = partial_sum(um[idx], x, L, alpha, op, npts, P, weights_kind, tables, weno)
    return np.moveaxis(out, -1, ax)
