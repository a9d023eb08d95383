"""GPU parity of the batched heat step (one persistent cooperative kernel per
time step over problems of uneven sizes, per-size-class autotuned tile shapes)
against the oracle and against the per-problem path, and the bounded grid
barrier's timeout status."""
import numpy as np
import pytest

from oracle import schemes
from paper_2007_03041_gb300 import molt as M
from paper_2007_03041_gb300 import workloads
from tests.gpu_util import need_gpu, rel_l2, to_dev, assert_grid_parity

pytestmark = pytest.mark.gpu


def _descs(sides):
    out = []
    for n in sides:
        h = 1.0 / n
        out.append(M.make_desc((n, n), P=3, quad_points=3, beta=0.6, pde=M.PDE_HEAT, dt=h / 2,
                               prec=M.PREC_F32_F64UPDATE))
    return out


def _run_batch(sides, nsteps, stream=True):
    import torch
    u0 = workloads.batched_heat(sides=sides)
    s = torch.cuda.Stream() if stream else None
    ctx = M.molt_create(_descs(sides), stream=s)
    try:
        us = [to_dev(x, torch.float64) for x in u0]
        torch.cuda.synchronize()
        t = M.molt_step(ctx, us, None, nsteps=nsteps, t=[0.0] * len(sides))
        torch.cuda.synchronize()
        shapes = [(M.molt_batch_tile_shape(ctx, i, 0), M.molt_batch_tile_shape(ctx, i, 1)) for i in range(len(sides))]
        return u0, [x.cpu().numpy() for x in us], t, shapes
    finally:
        M.molt_destroy(ctx)


def test_batched_heat_matches_oracle():
    need_gpu()
    sides = [128, 256, 512, 128, 1024, 256]
    u0, got, t, shapes = _run_batch(sides, 2)
    for n, a, b in zip(sides, u0, got):
        want = a
        for _ in range(2):
            want = schemes.heat_step(want, [1.0 / n] * 2, 0.5 / n, 1.0, 0.6, None, 3, 3)
        assert_grid_parity(b, want, 1e-5, what=str(n), ends=False)
    for n, ti in zip(sides, t):
        assert abs(ti - 2 * 0.5 / n) < 1e-15
    for n, (sx, sy) in zip(sides, shapes):
        for E, nwl, W in (sx, sy):
            assert E in (4, 8, 16) and nwl * W == 16 and 32 * nwl * E == n


def test_batched_matches_per_problem_path_large_sides():
    import torch
    need_gpu()
    sides = [2048, 1024, 512, 2048, 256]
    u0, got, _, _ = _run_batch(sides, 1, stream=False)   # legacy stream: direct launches
    for n, a, b in zip(sides, u0, got):
        ctx = M.molt_create(_descs([n])[0])
        try:
            u = to_dev(a, torch.float64)
            M.molt_step(ctx, u, None, nsteps=1, t=[0.0])
            ref = u.cpu().numpy()
        finally:
            M.molt_destroy(ctx)
        assert_grid_parity(b, ref, 1e-6, what=str(n))


def test_grid_barrier_wait_runs_out_and_context_stays_usable():
    import torch
    need_gpu()
    sides = [256, 128, 512]
    u0 = workloads.batched_heat(sides=sides)
    ctx = M.molt_create(_descs(sides))
    try:
        us = [to_dev(x, torch.float64) for x in u0]
        M.molt_set_option(ctx, M.OPT_WAIT_LIMIT, 2_000_000)     # about a millisecond
        M.molt_set_option(ctx, M.OPT_TEST_SKIP_ARRIVE, 1)
        with pytest.raises(M.MoltError) as ei:
            M.molt_step(ctx, us, None, nsteps=1, t=[0.0] * 3)
        assert ei.value.status == M.MOLT_ETIMEOUT
        # back to normal: the next step completes and matches the oracle
        M.molt_set_option(ctx, M.OPT_TEST_SKIP_ARRIVE, 0)
        M.molt_set_option(ctx, M.OPT_WAIT_LIMIT, 2_000_000_000)
        start = [x.cpu().numpy() for x in us]
        M.molt_step(ctx, us, None, nsteps=1, t=[0.0] * 3)
        got = [x.cpu().numpy() for x in us]
    finally:
        M.molt_destroy(ctx)
    for n, a, b in zip(sides, start, got):
        want = schemes.heat_step(a, [1.0 / n] * 2, 0.5 / n, 1.0, 0.6, None, 3, 3)
        assert_grid_parity(b, want, 1e-5, ends=False)
