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
