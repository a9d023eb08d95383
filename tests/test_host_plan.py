"""Tile plans of the sweeps, on the host (molt_plan_sweep; no GPU): for
every line length 1..8192 in FP32 and FP64, and for grids with few and many
lines, the planned tile covers the line with no idle warp, stays within 512
threads and the shared-memory budget, and its grid covers every line; lines
past 8192 points are refused.  A wrong tile here is a wrong kernel launch
there, so the whole range is checked."""
import os

import pytest

from paper_2007_03041_gb300 import molt as M


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not os.path.exists(M.LIB_PATH):
        from paper_2007_03041_gb300 import build
        build.build()
    return M.load_library()


def _check(plan, n, nlines, elem):
    E, nwl, W = plan["points_per_lane"], plan["warps_per_line"], plan["lines_per_cta"]
    assert E in (4, 8, 16)
    assert 32 * E * nwl >= n > 32 * E * (nwl - 1), (n, plan)          # covers the line, no idle warp
    assert W >= 1 and W & (W - 1) == 0
    assert plan["threads_per_cta"] == 32 * nwl * W <= 512
    assert plan["ctas"] * W >= nlines > (plan["ctas"] - 1) * W
    assert plan["exact_fit"] == (1 if n == 32 * E * nwl else 0)
    assert W * n * elem <= plan["smem_bytes"] <= 200 * 1024


@pytest.mark.parametrize("prec,elem", [(M.PREC_F32, 4), (M.PREC_F64, 8)])
def test_every_line_length_of_a_1d_problem(prec, elem):
    for n in range(1, 8193):
        d = M.make_desc((n,), prec=prec)
        plan = M.molt_plan_sweep(d, 0, M.OP_0, 2, 0.7 * n)
        _check(plan, n, 1, elem)


@pytest.mark.parametrize("prec,elem", [(M.PREC_F32, 4), (M.PREC_F64, 8), (M.PREC_F32_F64UPDATE, 4)])
@pytest.mark.parametrize("bc", [M.BC_PERIODIC, M.BC_DIRICHLET])
def test_grids_with_few_and_many_lines(prec, elem, bc):
    for n in (7, 96, 255, 256, 257, 511, 512, 1000, 1024, 2048, 2053, 4096, 5277, 8191, 8192):
        for other in (1, 3, 64, 4096):
            d = M.make_desc((n, other), bc=[bc, M.BC_PERIODIC], prec=prec)
            _check(M.molt_plan_sweep(d, 0, M.OP_R, 1, 2.0 * n), n, other, elem)
            d = M.make_desc((other, n), bc=[M.BC_PERIODIC, bc], prec=prec)
            _check(M.molt_plan_sweep(d, 1, M.OP_L, 3, 2.0 * n), n, other, elem)


def test_the_preferred_tiles():
    """FP32: 16 points per lane whenever a line of whole warps allows it;
    FP64 grids with few lines: fewer points per lane (more warps per line
    against the FP64 pipe's latency), many lines: 16."""
    f32 = M.molt_plan_sweep(M.make_desc((512, 256, 512), prec=M.PREC_F32), 0, M.OP_0, 2, 100.0)
    assert f32["points_per_lane"] == 16 and f32["exact_fit"] == 1
    few = M.molt_plan_sweep(M.make_desc((256, 256), prec=M.PREC_F64), 0, M.OP_0, 3, 60.0)
    assert few["points_per_lane"] == 4 and few["warps_per_line"] == 2
    many = M.molt_plan_sweep(M.make_desc((4096, 4096), prec=M.PREC_F64), 0, M.OP_0, 1, 600.0)
    assert many["points_per_lane"] == 16


def test_fp64_points_per_lane_of_grids_with_few_lines():
    """The FP64 rule for grids with few lines (one sweep at a time; the SM
    count taken as 152 without a GPU): the measured-fastest points per lane
    of the heat steps, 256^2 -> 4 (two warps a line), 512^2 -> 8 (two warps
    a line, not one of 16 points a lane), 1024^2 and 2048^2 -> 16."""
    want = {256: (4, 2), 512: (8, 2), 1024: (16, 2), 2048: (16, 4)}
    for n, (E, nwl) in want.items():
        for axis in (0, 1):
            plan = M.molt_plan_sweep(M.make_desc((n, n), P=3, quad_points=3, prec=M.PREC_F64), axis, M.OP_0, 3,
                                     0.6 * n)
            assert (plan["points_per_lane"], plan["warps_per_line"]) == (E, nwl), (n, axis, plan)


def test_refused_plans():
    with pytest.raises(M.MoltError):
        M.molt_plan_sweep(M.make_desc((8193,)), 0, M.OP_0, 1, 100.0)          # longer than 8192 points
    with pytest.raises(M.MoltError):
        M.molt_plan_sweep(M.make_desc((64,)), 1, M.OP_0, 1, 10.0)             # axis out of range
    with pytest.raises(M.MoltError):
        M.molt_plan_sweep(M.make_desc((64,)), 0, 7, 1, 10.0)                  # unknown op
    with pytest.raises(M.MoltError):
        M.molt_plan_sweep(M.make_desc((64,)), 0, M.OP_0, 1, -1.0)             # alpha h must be positive
    with pytest.raises(M.MoltError):
        M.molt_plan_sweep(M.make_desc((64,), quad_points=5, weights=M.W_LEARNED, prec=M.PREC_F32), 0,
                          M.OP_R, 1, 10.0)                                     # learned: planned with the network
