"""Oracle: the WENO-weight network of the learned weight path, in FP64.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__``.

The paper has no learned component; this follows the network the learned
path specifies: 5 stencil values -> 32 -> 32 -> 3, GELU after both hidden
layers, softmax output = the three nonlinear weights w_r of the WENO
combination J = sum_r w_r J^{(r)} (Sec. 2.4, commented WENO step).

Conventions (shared by the CUDA kernels, restated here independently):
* input normalisation: x_j = (v_j - v_c) / (max_j |v_j - v_c| + 1e-30), v_c the
  middle of the 5 values (reading: normalised by the local spread, so the
  input is shift- and scale-free like the WENO weights themselves);
* GELU in its tanh form, z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)));
* weights and biases are BF16; the kernels round the inputs and the hidden
  activations to BF16 before each matrix product and accumulate in FP32
  (``emulate_bf16=True`` reproduces those roundings, in FP64 otherwise);
* loss = mean over stencils of sum_r (p_r - w_r)^2 against WENO-Z targets;
* fallback: where max_r |p_r - wZ_r| > 1e-2 (or is not finite) the WENO-Z
  weights are used.

Parameter vector (FP32 master order): W1 (32x5), b1 (32), W2 (32x32),
b2 (32), W3 (3x32), b3 (3).
"""
import math

import numpy as np

SHAPES = (("W1", (32, 5)), ("b1", (32,)), ("W2", (32, 32)), ("b2", (32,)), ("W3", (3, 32)), ("b3", (3,)))
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)
FALLBACK_TOL = 1e-2


def bf16_round(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = (b + 0x7FFF + lsb) >> 16 << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(theta):
    out, k = {}, 0
    for name, shape in SHAPES:
        m = int(np.prod(shape))
        out[name] = np.asarray(theta[k:k + m], dtype=np.float64).reshape(shape)
        k += m
    return out


def pack(params):
    return np.concatenate([np.asarray(params[n], dtype=np.float64).ravel() for n, _ in SHAPES])


def init_params(seed=50):
    """He-style random initial parameters (seeded)."""
    g = np.random.Generator(np.random.PCG64(seed))
    p = {}
    p["W1"] = g.standard_normal((32, 5)) * math.sqrt(2.0 / 5)
    p["b1"] = np.zeros(32)
    p["W2"] = g.standard_normal((32, 32)) * math.sqrt(2.0 / 32)
    p["b2"] = np.zeros(32)
    p["W3"] = g.standard_normal((3, 32)) * math.sqrt(1.0 / 32)
    p["b3"] = np.zeros(3)
    return pack(p)


def normalise(V):
    """(n, 5) stencil values -> (n, 5) network inputs."""
    V = np.asarray(V, dtype=np.float64)
    d = V - V[:, 2:3]
    return d / (np.abs(d).max(axis=1, keepdims=True) + 1e-30)


GELU_C = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(GELU_C * (z + GELU_A * z ** 3)))


def gelu_grad(z):
    t = np.tanh(GELU_C * (z + GELU_A * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_C * (1.0 + 3.0 * GELU_A * z * z)


def forward(theta, X, emulate_bf16=True):
    """Network outputs p (n, 3) and the cached intermediates."""
    P = unpack(theta)
    r = bf16_round if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    W1, b1, W2, b2, W3, b3 = (r(P[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3"))
    x = r(X)
    z1 = x @ W1.T + b1
    a1 = r(gelu(z1))
    z2 = a1 @ W2.T + b2
    a2 = r(gelu(z2))
    z3 = a2 @ W3.T + b3
    z3s = z3 - z3.max(axis=1, keepdims=True)
    e = np.exp(z3s)
    p = e / e.sum(axis=1, keepdims=True)
    return p, dict(x=x, z1=z1, a1=a1, z2=z2, a2=a2, p=p, W2=W2, W3=W3)


def loss(theta, X, Yt, emulate_bf16=True):
    p, _ = forward(theta, X, emulate_bf16)
    return float(np.mean(np.sum((p - Yt) ** 2, axis=1)))


def loss_and_grad(theta, X, Yt, emulate_bf16=True):
    """Mean-squared loss and its gradient with respect to the FP32 master
    parameters (backpropagation by hand: softmax, GELU and the three affine
    layers; the BF16 roundings are treated as identity in the backward pass)."""
    p, c = forward(theta, X, emulate_bf16)
    n = X.shape[0]
    L = float(np.mean(np.sum((p - Yt) ** 2, axis=1)))
    g = 2.0 * (p - Yt) / n                                  # dL/dp
    dz3 = p * (g - np.sum(g * p, axis=1, keepdims=True))   # softmax Jacobian
    dW3 = dz3.T @ c["a2"]
    db3 = dz3.sum(axis=0)
    dz2 = (dz3 @ c["W3"]) * gelu_grad(c["z2"])
    dW2 = dz2.T @ c["a1"]
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ c["W2"]) * gelu_grad(c["z1"])
    dW1 = dz1.T @ c["x"]
    db1 = dz1.sum(axis=0)
    return L, pack(dict(W1=dW1, b1=db1, W2=dW2, b2=db2, W3=dW3, b3=db3))


def learned_weight_fn(theta, rule, emulate_bf16=True):
    """weight_fn for oracle.sweep.local_integrals(weights='learned'): network
    weights with the WENO-Z fallback."""
    from .sweep import _weno_weights

    def fn(Wv):
        shp = Wv.shape[:-1]
        V = Wv.reshape(-1, 5)
        p, _ = forward(theta, normalise(V), emulate_bf16)
        wz = _weno_weights(rule, V)
        bad = ~(np.abs(p - wz).max(axis=1) <= FALLBACK_TOL)   # non-finite outputs fall back too
        p[bad] = wz[bad]
        return p.reshape(shp + (3,))
    return fn


def adam_step(theta, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, 2015, Algorithm 1) in FP64: the first and
    second moment estimates, their bias corrections by 1 - beta^step, and the
    step lr * mhat / (sqrt(vhat) + eps).  Returns (theta, m, v)."""
    g = np.asarray(grad, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return np.asarray(theta, dtype=np.float64) - lr * mhat / (np.sqrt(vhat) + eps), m, v


def blob_values(theta):
    """The BF16 network blob as float64 values in its storage order: W1 (32x16,
    inputs 5.. zero), W2 (32x32), W3 (8x32, rows 3.. zero), b1, b2, b3 (8)."""
    P = unpack(theta)
    W1 = np.zeros((32, 16)); W1[:, :5] = P["W1"]
    W3 = np.zeros((8, 32)); W3[:3] = P["W3"]
    b3 = np.zeros(8); b3[:3] = P["b3"]
    flat = np.concatenate([W1.ravel(), P["W2"].ravel(), W3.ravel(), P["b1"], P["b2"], b3])
    return bf16_round(flat)


def stencils(u, pos, axis, side):
    """5-value stencils of the periodic 2-D array u (ny, nx) at flat indices
    pos along axis 0 (x) or 1 (y): offsets -3..1 (side 0, J_R orientation) or
    +3..-1 (side 1, mirrored for J_L)."""
    u = np.asarray(u)
    ny, nx = u.shape
    yi, xi = np.divmod(np.asarray(pos, dtype=np.int64), nx)
    offs = np.arange(-3, 2) if side == 0 else np.arange(3, -2, -1)
    if axis == 0:
        return u[yi[:, None], (xi[:, None] + offs[None, :]) % nx]
    return u[(yi[:, None] + offs[None, :]) % ny, xi[:, None]]
