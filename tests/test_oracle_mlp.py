"""Pins of the oracle's WENO-weight network (learned weight path): the hand
backpropagation against central finite differences, softmax/normalisation
invariants, BF16 rounding, and the WENO-Z fallback."""
import numpy as np
import pytest

from oracle import mlp, sweep
from oracle.quadrature import QuadratureRule


def test_bf16_rounding_known_values():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.140625, 1e-3])
    r = mlp.bf16_round(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                      # tie -> even mantissa
    assert r[2] == 1.0 + 2 * 2 ** -7        # tie -> even (upwards)
    assert r[3] == -2.5 and r[4] == 3.140625
    assert abs(r[5] - 1e-3) < 1e-3 * 2 ** -8


def test_gradient_matches_finite_differences():
    g = np.random.default_rng(3)
    theta = mlp.init_params(5)
    X = mlp.normalise(g.standard_normal((40, 5)))
    Y = g.dirichlet(np.ones(3), size=40)
    L, grad = mlp.loss_and_grad(theta, X, Y, emulate_bf16=False)
    eps = 1e-6
    for k in g.choice(mlp.NPARAMS, size=60, replace=False):
        tp = theta.copy(); tp[k] += eps
        tm = theta.copy(); tm[k] -= eps
        fd = (mlp.loss(tp, X, Y, False) - mlp.loss(tm, X, Y, False)) / (2 * eps)
        assert abs(fd - grad[k]) < 1e-6 * max(1.0, abs(fd)) + 1e-9, (k, fd, grad[k])


def test_softmax_outputs_and_input_invariance():
    g = np.random.default_rng(4)
    theta = mlp.init_params(7)
    V = g.standard_normal((30, 5))
    p, _ = mlp.forward(theta, mlp.normalise(V))
    assert np.all(p > 0) and np.allclose(p.sum(axis=1), 1.0, atol=1e-14)
    # inputs are shift and positive-scale invariant
    np.testing.assert_allclose(mlp.normalise(3.0 * V + 7.0), mlp.normalise(V), atol=1e-14)
    assert np.allclose(np.abs(mlp.normalise(V)).max(axis=1), 1.0)


def test_gelu_gradient():
    z = np.linspace(-4, 4, 41)
    fd = (mlp.gelu(z + 1e-6) - mlp.gelu(z - 1e-6)) / 2e-6
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, atol=1e-8)


def test_fallback_reproduces_wenoz_when_every_stencil_trips():
    # a network that outputs (1, 0, 0) for every stencil is far from WENO-Z
    # on smooth data, so every stencil falls back: learned J == WENO-Z J
    theta = np.zeros(mlp.NPARAMS)
    P = mlp.unpack(theta)
    P["b3"] = np.array([50.0, 0.0, 0.0])
    theta = mlp.pack(P)
    n, dx, alpha = 64, 2 * np.pi / 64, 1.0 / (1.5 * 2 * np.pi / 64)
    x = np.arange(n) * dx
    v = (np.sin(x) + 0.3 * np.cos(3 * x))[None, :]
    rule = QuadratureRule(alpha * dx, 5)
    fn = mlp.learned_weight_fn(theta, rule, emulate_bf16=False)
    vext = sweep.extend(v, "periodic")
    c = np.arange(n)
    for side in "RL":
        a = sweep.local_integrals(vext, c, rule, side, "learned", fn)
        b = sweep.local_integrals(vext, c, rule, side, "wenoz")
        np.testing.assert_allclose(a, b, atol=1e-15)


def test_fallback_catches_non_finite_outputs():
    # a NaN weight makes every output NaN; the fallback must still give WENO-Z
    theta = np.zeros(mlp.NPARAMS)
    P = mlp.unpack(theta)
    P["b3"] = np.array([np.nan, 0.0, 0.0])
    theta = mlp.pack(P)
    rule = QuadratureRule(2.0 / 3.0, 5)
    V = np.random.default_rng(8).standard_normal((20, 5))
    w = mlp.learned_weight_fn(theta, rule, emulate_bf16=False)(V)
    np.testing.assert_allclose(w, sweep._weno_weights(rule, V), atol=0)


def test_network_with_constant_logits_returns_their_softmax():
    # zero weights: the outputs are softmax(b3) for any input (closed form)
    theta = np.zeros(mlp.NPARAMS)
    P = mlp.unpack(theta)
    d = np.array([0.1, 0.6, 0.3])
    P["b3"] = np.log(d)
    p, _ = mlp.forward(mlp.pack(P), mlp.normalise(np.random.default_rng(2).standard_normal((9, 5))), False)
    np.testing.assert_allclose(p, np.tile(d, (9, 1)), atol=1e-15)


def test_adam_first_step_is_a_signed_step_of_size_lr():
    # step 1 from zero moments: mhat = g, vhat = g^2, so the update is
    # lr * g / (|g| + eps) -- lr times the sign of g up to eps
    g = np.array([3.0, -0.5, 1e-3, -2e2])
    th, m, v = mlp.adam_step(np.zeros(4), np.zeros(4), np.zeros(4), g, 1, 0.01, eps=1e-12)
    np.testing.assert_allclose(th, -0.01 * np.sign(g), rtol=1e-8)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)
    # a constant gradient keeps mhat = g and vhat = g^2 at every step
    th2, m2, v2 = mlp.adam_step(th, m, v, g, 2, 0.01, eps=1e-12)
    np.testing.assert_allclose(th2, -0.02 * np.sign(g), rtol=1e-8)


def test_blob_layout_and_stencil_gather():
    theta = np.arange(mlp.NPARAMS, dtype=np.float64) / 64.0
    b = mlp.blob_values(theta)
    assert b.size == 3728 // 2
    assert b[16 * 3 + 4] == mlp.bf16_round(theta[3 * 5 + 4]) and b[16 * 3 + 5] == 0.0   # W1[3][4], pad
    assert b[512 + 32 * 7 + 9] == mlp.bf16_round(theta[192 + 7 * 32 + 9])               # W2[7][9]
    assert b[1536 + 32 * 2 + 31] == mlp.bf16_round(theta[1248 + 2 * 32 + 31])           # W3[2][31]
    assert np.all(b[1536 + 96:1536 + 256] == 0.0)
    assert b[1856 + 2] == mlp.bf16_round(theta[1346]) and np.all(b[1859:] == 0.0)       # b3
    # gather: u[y, x] = 100 y + x, so a stencil is an arithmetic sequence
    ny, nx = 7, 9
    u = 100.0 * np.arange(ny)[:, None] + np.arange(nx)[None, :]
    pos = np.array([0, 8, 3 * nx + 4, ny * nx - 1])
    sx = mlp.stencils(u, pos, 0, 0)
    np.testing.assert_array_equal(sx[2], 300.0 + np.arange(1, 6))
    np.testing.assert_array_equal(sx[0], [6.0, 7.0, 8.0, 0.0, 1.0])        # periodic wrap in x
    sy = mlp.stencils(u, pos, 1, 1)
    np.testing.assert_array_equal(sy[2], 4.0 + 100.0 * np.array([6, 5, 4, 3, 2]))
    np.testing.assert_array_equal(sy[3], 8.0 + 100.0 * np.array([2, 1, 0, 6, 5]))   # wrap in y
