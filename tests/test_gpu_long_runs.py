"""Parity over the stated lengths of the runs, against the FP64 oracle:

* 3-D wave (Dirichlet, P = 2, 6-point rule, FP32 sweeps with FP64 boundary
  solve and leapfrog update, dt = 2h): all 50 steps, compared in full, on a
  128^3 grid (the oracle's axis sums as dense matrices, oracle/dense.py), with
  the line-per-lane sweeps and with the scan sweeps;
* the 64 batched heat problems (sides 128..2048, P = 3, FP32 sweeps + FP64
  update, SSP-RK3): all 200 steps against the closed-form discrete solution
  at sampled points;
* 2-D Hamilton-Jacobi (WENO-Z, FP32, CFL 1.5, lagged adaptive dt): all 500
  steps on a 256^2 grid (the oracle's partial sums on blocks of lines in a
  process pool), well past the formation of the kinks;
* the same with learned WENO weights (the network, trained by the oracle's
  own Adam on stencils of the oracle's states, with the WENO-Z fallback):
  50 steps on a 512^2 grid against the oracle's BF16-emulated forward.

The wave and heat states are held to the FP32 path's stated tolerance:
relative L2 1e-5, plus the largest pointwise error over the largest value
(2e-5) and the first and last 4 points of every line.  The Hamilton-Jacobi
state is held to it before the kinks form; after that, to a bound measured
with the oracle itself (see the test)."""
import math

import numpy as np
import pytest

from oracle import dense, mlp, stability, sweep
from oracle.quadrature import QuadratureRule
from paper_2007_03041_gb300 import molt as M
from paper_2007_03041_gb300 import workloads
from tests.gpu_util import need_gpu, to_dev, assert_parity, rel_l2, max_rel, TOL_F32, MAX_F32, assert_grid_parity

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.mark.parametrize("lanes", [1, 0])
def test_wave_50_steps_in_full(lanes):
    need_gpu()
    import torch
    n, nsteps = 128, 50
    h = 1.0 / (n - 1)
    dt = 2 * h
    u0 = workloads.wave_bumps(n)
    d = M.make_desc((n, n, n), bc=[M.BC_DIRICHLET] * 3, P=2, quad_points=6, beta=0.8, pde=M.PDE_WAVE,
                    c=1.0, dt=dt, prec=M.PREC_F32_F64UPDATE)
    ctx = M.molt_create(d)
    try:
        M.molt_set_option(ctx, M.OPT_LANES, lanes)
        u = to_dev(u0, torch.float64)
        up = torch.zeros_like(u)
        t = M.molt_step(ctx, u, up, nsteps=1, t=[0.0])
        t = M.molt_step(ctx, u, up, nsteps=nsteps - 1, t=t)
        got, gotp = u.cpu().numpy(), up.cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    assert abs(t[0] - nsteps * dt) < 1e-12
    mats = dense.wave_matrices(u0.shape, [h] * 3, dt, 1.0, 0.8, ["dirichlet"] * 3, 6, 2)
    prev, cur = None, u0
    for k in range(nsteps):
        prev, cur = cur, dense.wave_step(cur, prev, mats, 0.8, from_rest=(k == 0))
    for ax in range(3):
        assert_parity(got, cur, TOL_F32, MAX_F32, line_axis=ax, what="u^50 (lanes=%d)" % lanes)
    assert_parity(gotp, prev, TOL_F32, MAX_F32, what="u^49 (lanes=%d)" % lanes)


def _rk3(z):
    return 1.0 + z + z * z / 2.0 + z ** 3 / 6.0


def _modal_heat(n, seed, nsteps, iy, ix, beta=0.6, npts=3, P=3):
    """Closed-form discrete solution of the periodic heat step (dt = h/2): every
    Fourier mode of u0 is multiplied by the RK3 polynomial of its exact
    discrete symbol once per step."""
    k, a = workloads.heat_mode_params(seed)
    h = 1.0 / n
    nu = beta / math.sqrt(h / 2) * h
    out = np.zeros(len(ix))
    for (kx, ky), am in zip(k, a):
        tx, ty = 2 * np.pi * kx / n, 2 * np.pi * ky / n
        z = -beta ** 2 * (stability.partial_sum_symbol(tx, nu, "0", npts, P).real
                          + stability.partial_sum_symbol(ty, nu, "0", npts, P).real)
        out += am * _rk3(z) ** nsteps * np.cos(tx * ix + ty * iy)
    return out


def test_batched_64_problems_200_steps_closed_form():
    """After 200 steps the modes of the small problems have decayed by many
    orders of magnitude, so the bound is on the error relative to the initial
    amplitude (and relative to the final values where those are not tiny)."""
    need_gpu()
    import torch
    nsteps = 200
    sides = workloads.batched_sides()
    descs = [M.make_desc((n, n), P=3, quad_points=3, beta=0.6, pde=M.PDE_HEAT, dt=0.5 / n,
                         prec=M.PREC_F32_F64UPDATE) for n in sides]
    u0s = workloads.batched_heat(sides=sides)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = M.molt_create(descs, stream=s)
        try:
            us = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in u0s]
            M.molt_step(ctx, us, None, nsteps=nsteps, t=[0.0] * len(us))
            s.synchronize()
            got = [x.cpu().numpy() for x in us]
        finally:
            M.molt_destroy(ctx)
    g = workloads.rng(77)
    for i, (n, a0, gi) in enumerate(zip(sides, u0s, got)):
        iy = g.integers(0, n, 512)
        ix = g.integers(0, n, 512)
        iy[:2], ix[:2] = [0, n - 1], [n - 1, 0]
        want = _modal_heat(n, 3000 + i, nsteps, iy, ix)
        err = np.abs(gi[iy, ix] - want).max()
        assert err <= TOL_F32 * np.abs(a0).max(), (i, n, err)
        if np.abs(want).max() > 1e-3 * np.abs(a0).max():
            assert_grid_parity(gi[iy, ix], want, TOL_F32, what=str((i, n)), ends=False)


def test_hj_wenoz_500_steps():
    """The FP32-state form over the stated 500 steps.  Near the kinks (t ~ 1,
    past step 40 on this grid) the problem amplifies perturbations of FP32
    size by about 10^4: the oracle itself, run with its state rounded to FP32
    after every step, departs from the pure FP64 oracle by 2.6e-3 at step 100
    and 4.4e-5 at step 500.  So at each checkpoint (step 20, before the kinks,
    and step 500) the GPU result is held to the stated tolerance or to twice
    the distance of the oracle's own FP32-state run from the FP64 oracle,
    whichever is larger (relative L2 and largest pointwise error)."""
    need_gpu()
    import torch
    from oracle.parallel import LinePool
    n, early, nsteps = 256, 20, 500
    h = 2 * np.pi / n
    u0 = workloads.hj_initial(n)
    d = M.make_desc((n, n), lo=[0, 0], hi=[2 * np.pi] * 2, P=1, quad_points=5, weights=M.W_WENOZ, beta=1.0,
                    pde=M.PDE_HJ, cfl=1.5, dt=0.0, prec=M.PREC_F32)
    ctx = M.molt_create(d)
    try:
        u = to_dev(u0, torch.float32)
        t = M.molt_step(ctx, u, None, nsteps=early, t=[0.0])
        got_early = u.double().cpu().numpy()
        t = M.molt_step(ctx, u, None, nsteps=nsteps - early, t=t)
        got = u.double().cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    start = u0.astype(np.float32).astype(np.float64)
    a, b = start, start          # FP64 oracle; oracle with FP32 state storage
    ta = tb = 0.0
    checks = {}
    with LinePool() as pool:
        sa = sb = pool.hj_initial_speeds(start, [h, h])
        for k in range(1, nsteps + 1):
            a, dta, sa = pool.hj_step(a, [h, h], sa)
            b, dtb, sb = pool.hj_step(b, [h, h], sb)
            b = b.astype(np.float32).astype(np.float64)
            ta += dta
            tb += dtb
            if k in (early, nsteps):
                checks[k] = (a, max(TOL_F32, 2 * rel_l2(b, a)), max(MAX_F32, 2 * max_rel(b, a)))
    for k, got_k in ((early, got_early), (nsteps, got)):
        want, tl2, tmax = checks[k]
        for ax in range(2):
            assert_parity(got_k, want, tl2, tmax, line_axis=ax, what="HJ u^%d" % k)
    assert checks[early][1] == TOL_F32      # before the kinks FP32 storage alone stays below the stated bound
    # the time is the sum of the lagged steps dt = cfl h / c_max: held like the
    # state, to 1e-3 or twice the FP32-state oracle's own departure
    assert abs(t[0] - ta) < max(1e-3 * ta, 2 * abs(tb - ta))


NU_HJ = 1.0 / 1.5   # nu = alpha h = beta / CFL of the Hamilton-Jacobi runs


def _oracle_trained_theta(states, seed=workloads.SEED_MLP, steps=300, batch=2048, lr=3e-3):
    """A network trained entirely by the oracle: stencils of the given states
    (both axes and sides, seeded positions), WENO-Z targets, minibatch Adam in
    FP64 on the BF16-emulated loss.  Returns the FP32 master parameters."""
    rule = QuadratureRule(NU_HJ, 5)
    X = []
    for k, u in enumerate(states):
        ny, nx = u.shape
        for axis in (0, 1):
            for side in (0, 1):
                pos = workloads.mlp_positions(batch * steps // (4 * len(states)) + 1, nx, ny,
                                              seed + 4 * k + 2 * axis + side)
                X.append(mlp.stencils(u, pos, axis, side))
    X = np.concatenate(X)
    X = X[workloads.rng(seed).permutation(len(X))]
    Y = sweep._weno_weights(rule, X)
    theta = workloads.mlp_initial_params(seed).astype(np.float64)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    for s in range(1, steps + 1):
        r0 = ((s - 1) * batch) % (len(X) - batch)
        _, g = mlp.loss_and_grad(theta, mlp.normalise(X[r0:r0 + batch]), Y[r0:r0 + batch], emulate_bf16=True)
        theta, m, v = mlp.adam_step(theta, m, v, g, s, lr)
    return theta.astype(np.float32)


def test_hj_learned_50_steps():
    """The learned-weight form (BF16 network + WENO-Z fallback, FP32) over 50
    steps at 512^2.  Held as the WENO-Z run is: to the stated tolerance, or to
    twice the distance of the oracle's own FP32-state run from the FP64
    oracle where that is larger -- here a fallback decision taken on the other
    side of the 1e-2 threshold is one more FP32-size perturbation -- at step
    20 and at step 50.  The network falls back on part of the stencils only."""
    need_gpu()
    import torch
    from oracle.parallel import LinePool
    n, early, nsteps = 512, 20, 50
    h = 2 * np.pi / n
    u0 = workloads.hj_initial(n)
    start = u0.astype(np.float32).astype(np.float64)
    with LinePool() as pool:
        # training states: u^0 and the oracle's WENO-Z state after 40 steps
        sp = pool.hj_initial_speeds(start, [h, h])
        w = start
        for _ in range(40):
            w, _, sp = pool.hj_step(w, [h, h], sp)
        theta32 = _oracle_trained_theta([start, w])
        theta = theta32.astype(np.float64)
        d = M.make_desc((n, n), lo=[0, 0], hi=[2 * np.pi] * 2, P=1, quad_points=5, weights=M.W_LEARNED,
                        beta=1.0, pde=M.PDE_HJ, cfl=1.5, dt=0.0, prec=M.PREC_F32)
        ctx = M.molt_create(d)
        try:
            th = torch.tensor(theta32, device="cuda")
            blob = torch.empty(M.MLP_BLOB_BYTES, dtype=torch.uint8, device="cuda")
            M.molt_mlp_pack(th, blob)
            M.molt_set_mlp(ctx, blob)
            u = to_dev(u0, torch.float32)
            t = M.molt_step(ctx, u, None, nsteps=early, t=[0.0])
            got_early = u.double().cpu().numpy()
            t = M.molt_step(ctx, u, None, nsteps=nsteps - early, t=t)
            got = u.double().cpu().numpy()
            evaluated, fallbacks = M.molt_mlp_stats(ctx)
        finally:
            M.molt_destroy(ctx)
        a, b = start, start
        ta = tb = 0.0
        checks = {}
        sa = sb = pool.hj_initial_speeds(start, [h, h], 1.5, 1.0, 5, "learned", theta)
        for k in range(1, nsteps + 1):
            a, dta, sa = pool.hj_step(a, [h, h], sa, 1.5, 1.0, 5, "learned", theta)
            b, dtb, sb = pool.hj_step(b, [h, h], sb, 1.5, 1.0, 5, "learned", theta)
            b = b.astype(np.float32).astype(np.float64)
            ta += dta
            tb += dtb
            if k in (early, nsteps):
                checks[k] = (a, max(TOL_F32, 2 * rel_l2(b, a)), max(MAX_F32, 2 * max_rel(b, a)))
    for k, got_k in ((early, got_early), (nsteps, got)):
        want, tl2, tmax = checks[k]
        for ax in range(2):
            assert_parity(got_k, want, tl2, tmax, line_axis=ax, what="learned HJ u^%d" % k)
    assert abs(t[0] - ta) < max(1e-3 * ta, 2 * abs(tb - ta))
    assert 0 < fallbacks < evaluated
