"""Oracle: fast summation of L^{-1} and the successive-convolution partial sums.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__``.

Follows Sec. 2.1-2.4 of the paper in its notation:

* operators (Eqs. "left/right-moving inverse op", "second derivative inverse
  op", Sec. 2.1):
      L_R^{-1}[v](x) = I_R[v](x) + A e^{-alpha (x-a)}
      L_L^{-1}[v](x) = I_L[v](x) + B e^{-alpha (b-x)}
      L_0^{-1}[v](x) = I_0[v](x) + A e^{-alpha (x-a)} + B e^{-alpha (b-x)},
      I_0 = (I_L + I_R)/2 (split of Sec. 3.3, Eq. "DD partial xx local inverse op")
* D_* = I - L_*^{-1} (Eq. "D operators"), D^k = D(D^{k-1}) (Eq. "successive
  relation"), partial sums S_P = sum_{p=1}^P D^p (Eqs. for d_x^+, d_x^-, d_xx).
* grid x_i = a + i dx, i = 0..N (Sec. 2.4), recurrences
      I_R(x_i) = e^{-alpha dx} I_R(x_{i-1}) + J_R(x_i),  I_R(x_0) = 0
      I_L(x_i) = e^{-alpha dx} I_L(x_{i+1}) + J_L(x_i),  I_L(x_N) = 0
* periodic boundary constants (Eqs. "constants A and B for partial x / xx",
  Sec. 2.3): A = I_*(b)/(1-mu), B = I_*(a)/(1-mu), mu = e^{-alpha (b-a)}.

Readings (the paper is silent or garbled here):
* Periodic lines store the N unique points x_0..x_{N-1}; x_N is x_0 again and
  dx = (b-a)/N, so mu = e^{-nu N}.
* Dirichlet lines store all N+1 nodes x_0..x_N, dx = (b-a)/N.  A and B are
  fixed by enforcing the boundary values directly (Sec. 2.3): for L_0,
  L_0^{-1}[v](a) = v(a) and L_0^{-1}[v](b) = v(b), i.e. the 2x2 system
  [[1, mu], [mu, 1]] (A, B) = (v_0 - I_0(a), v_N - I_0(b)) -- the algebra of
  the 2x2 block solve of Sec. 3.3; for L_R, A = v(a) (App. A, Dirichlet
  inflow); for L_L, B = v(b).  Stencil ghosts are the odd reflection about
  the boundary value, v_{-j} = 2 v_0 - v_j and v_{N+j} = 2 v_N - v_{N-j}
  (for homogeneous data, v_{-j} = -v_j).
"""
import numpy as np

from .quadrature import QuadratureRule, WENOZ_EPS

BC_PERIODIC = "periodic"
BC_DIRICHLET = "dirichlet"
OPS = ("L", "R", "0")
GHOST = 3


def extend(V, bc):
    """Ghost extension of lines V (L, n) by GHOST cells per side; index
    k + GHOST of the result holds v_k for k in -GHOST .. n-1+GHOST."""
    L, n = V.shape
    g = GHOST
    if bc == BC_PERIODIC:
        idx = np.arange(-g, n + g) % n
        return V[:, idx]
    if bc == BC_DIRICHLET:
        out = np.empty((L, n + 2 * g))
        out[:, g:g + n] = V
        for j in range(1, g + 1):
            out[:, g - j] = 2.0 * V[:, 0] - V[:, min(j, n - 1)]
            out[:, g + n - 1 + j] = 2.0 * V[:, n - 1] - V[:, max(n - 1 - j, 0)]
        return out
    raise ValueError(bc)


def _weno_weights(rule, W):
    """WENO-Z nonlinear weights (commented WENO-Z step of Sec. 2.4):
    w~_r = d_r (1 + tau/(eps + beta_r)), tau = |beta_0 - beta_2|, normalised.
    W: (..., npts) stencil values in stencil order; returns (..., 3)."""
    m = len(rule.sub_offsets[0])
    betas = []
    for r in range(3):
        w = W[..., r:r + m]
        betas.append(np.einsum("...a,ab,...b->...", w, rule.beta_M[r], w))
    tau = np.abs(betas[0] - betas[2])
    wt = np.stack([rule.d[r] * (1.0 + tau / (WENOZ_EPS + betas[r])) for r in range(3)], axis=-1)
    return wt / wt.sum(axis=-1, keepdims=True)


def _stencil_values(Vext, centres, offsets, sign):
    """Array (L, len(centres), npts) of v_{i + sign*l} for l in offsets."""
    g = GHOST
    cols = [Vext[:, centres + sign * l + g] for l in offsets]
    return np.stack(cols, axis=-1)


def local_integrals(Vext, centres, rule, side, weights="linear", weight_fn=None):
    """J_R (side 'R') or J_L (side 'L') at grid indices ``centres``.

    J_R(x_i) = sum_l c_l v_{i+l};  J_L(x_i) = sum_l c_l v_{i-l} (App. C,
    mirror symmetry).  weights:
      'linear'  -- the large-stencil rule (equivalently sum_r d_r J^{(r)}),
      'wenoz'   -- sum_r w_r J^{(r)} with WENO-Z weights from the smoothness
                   indicators of the (mirrored) substencil values,
      'learned' -- sum_r w_r J^{(r)} with w = weight_fn(stencil values).
    """
    sign = 1 if side == "R" else -1
    if weights == "linear":
        Wv = _stencil_values(Vext, centres, rule.offsets, sign)
        return Wv @ rule.c
    Wv = _stencil_values(Vext, centres, rule.offsets, sign)
    m = len(rule.sub_offsets[0])
    Jr = np.stack([Wv[..., r:r + m] @ rule.sub_c[r] for r in range(3)], axis=-1)
    if weights == "wenoz":
        om = _weno_weights(rule, Wv)
    elif weights == "learned":
        om = weight_fn(Wv)
    else:
        raise ValueError(weights)
    return np.sum(om * Jr, axis=-1)


def inverse_operator(V, alpha, dx, op, bc, npts, weights="linear", weight_fn=None, rule=None):
    """L_op^{-1}[v] on every line of V (L, n), following Sec. 2.1-2.4."""
    V = np.asarray(V, dtype=np.float64)
    L, n = V.shape
    nu = alpha * dx
    if rule is None:
        rule = QuadratureRule(nu, npts)
    q = np.exp(-nu)                      # e^{-alpha dx}
    N = n if bc == BC_PERIODIC else n - 1   # number of intervals, x_0..x_N
    mu = np.exp(-alpha * N * dx)         # e^{-alpha (b-a)}
    Vext = extend(V, bc)
    idx = np.arange(N + 1)               # paper's node index 0..N
    stor = idx % n                       # storage index (x_N == x_0 if periodic)

    # I_R: I_R(x_0) = 0; I_R(x_i) = q I_R(x_{i-1}) + J_R(x_i), i = 1..N
    JR = local_integrals(Vext, stor[1:], rule, "R", weights, weight_fn) if N > 0 else np.zeros((L, 0))
    IR = np.zeros((L, N + 1))
    for i in range(1, N + 1):
        IR[:, i] = q * IR[:, i - 1] + JR[:, i - 1]
    # I_L: I_L(x_N) = 0; I_L(x_i) = q I_L(x_{i+1}) + J_L(x_i), i = N-1..0
    JL = local_integrals(Vext, stor[:N], rule, "L", weights, weight_fn)
    IL = np.zeros((L, N + 1))
    for i in range(N - 1, -1, -1):
        IL[:, i] = q * IL[:, i + 1] + JL[:, i]

    ea = np.exp(-alpha * dx * idx)        # e^{-alpha (x_i - a)}
    eb = np.exp(-alpha * dx * (N - idx))  # e^{-alpha (b - x_i)}
    if op == "R":
        A = IR[:, N] / (1.0 - mu) if bc == BC_PERIODIC else V[:, 0]
        Linv = IR + A[:, None] * ea
    elif op == "L":
        B = IL[:, 0] / (1.0 - mu) if bc == BC_PERIODIC else V[:, n - 1]
        Linv = IL + B[:, None] * eb
    elif op == "0":
        I0 = 0.5 * (IL + IR)
        if bc == BC_PERIODIC:
            A = I0[:, N] / (1.0 - mu)
            B = I0[:, 0] / (1.0 - mu)
        else:
            r0 = V[:, 0] - I0[:, 0]
            r1 = V[:, n - 1] - I0[:, N]
            # (A, B) = (1 - mu^2)^{-1} [[1, -mu], [-mu, 1]] (r0, r1)  (Sec. 3.3)
            A = (r0 - mu * r1) / (1.0 - mu * mu)
            B = (r1 - mu * r0) / (1.0 - mu * mu)
        Linv = I0 + A[:, None] * ea + B[:, None] * eb
    else:
        raise ValueError(op)
    return Linv[:, :n]


def partial_sum_lines(V, alpha, dx, op, bc, npts, P, weights="linear", weight_fn=None):
    """S_P = sum_{p=1}^P D^p[v], D = I - L^{-1} (Eqs. "D operators",
    "successive relation for D")."""
    rule = QuadratureRule(alpha * dx, npts)
    v = np.asarray(V, dtype=np.float64)
    S = np.zeros_like(v)
    for _ in range(P):
        v = v - inverse_operator(v, alpha, dx, op, bc, npts, weights, weight_fn, rule)
        S = S + v
    return S


def _to_lines(u, axis):
    ua = np.moveaxis(np.asarray(u, dtype=np.float64), axis, -1)
    return ua.reshape(-1, ua.shape[-1]), ua.shape


def _from_lines(Vl, shape, axis):
    return np.moveaxis(Vl.reshape(shape), -1, axis)


def partial_sum(u, axis, alpha, dx, op, bc, npts, P, weights="linear", weight_fn=None):
    """S_P along ``axis`` of an n-D array (dimensional splitting: each line
    along the axis is independent, Sec. 2.2)."""
    Vl, shape = _to_lines(u, axis)
    return _from_lines(partial_sum_lines(Vl, alpha, dx, op, bc, npts, P, weights, weight_fn), shape, axis)


def D_op(u, axis, alpha, dx, op, bc, npts, weights="linear", weight_fn=None):
    """D_op[u] = u - L_op^{-1}[u] along ``axis``."""
    return partial_sum(u, axis, alpha, dx, op, bc, npts, 1, weights, weight_fn)
