"""The process-pool form of the oracle's partial sums and Hamilton-Jacobi step
(tests/oracle_parallel.py) against the oracle itself."""
import numpy as np

from oracle import schemes, sweep
from oracle.parallel import LinePool


def test_pool_matches_the_oracle():
    n = 48
    h = 2 * np.pi / n
    x = np.arange(n) * h
    g = np.random.default_rng(5)
    u = -np.cos(x)[None, :] - np.cos(x)[:, None] + 0.01 * g.standard_normal((n, n))
    with LinePool(3) as pool:
        for ax in (0, 1):
            for op in ("R", "L", "0"):
                a = pool.partial_sum(u, ax, 20.0, h, op, "periodic", 5, 2, "wenoz")
                b = sweep.partial_sum(u, ax, 20.0, h, op, "periodic", 5, 2, "wenoz")
                assert np.abs(a - b).max() <= 1e-14 * np.abs(b).max()
        sp = schemes.hj_initial_speeds(u, [h, h])
        assert np.allclose(pool.hj_initial_speeds(u, [h, h]), sp, rtol=1e-14, atol=0)
        a, b = u, u
        la = lb = sp
        for _ in range(3):
            a, dta, la = pool.hj_step(a, [h, h], la)
            b, dtb, lb = schemes.hj_step(b, [h, h], lb)
            assert abs(dta - dtb) <= 1e-15 * dtb
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


def test_pool_with_learned_weights_matches_the_oracle():
    """Learned weights: the workers rebuild the weight function from the
    network's parameters, so the pooled step equals schemes.hj_step with the
    oracle's learned weight function."""
    from oracle import mlp
    from oracle.quadrature import QuadratureRule
    from paper_2007_03041_gb300 import workloads
    n = 40
    h = 2 * np.pi / n
    x = np.arange(n) * h
    u = -np.cos(x)[None, :] - np.abs(np.sin(x))[:, None]
    theta = workloads.mlp_initial_params().astype(np.float64)
    cfl, beta = 1.5, 1.0
    fn = mlp.learned_weight_fn(theta, QuadratureRule(beta / cfl, 5), emulate_bf16=True)
    with LinePool(2) as pool:
        sp = schemes.hj_initial_speeds(u, [h, h], cfl, beta, 5, "learned", fn)
        assert np.allclose(pool.hj_initial_speeds(u, [h, h], cfl, beta, 5, "learned", theta), sp, rtol=1e-14, atol=0)
        a, dta, _ = pool.hj_step(u, [h, h], sp, cfl, beta, 5, "learned", theta)
        b, dtb, _ = schemes.hj_step(u, [h, h], sp, cfl, beta, 5, "learned", fn)
    assert dta == dtb
    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()
