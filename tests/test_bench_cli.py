"""The bench's command-line contract without a GPU: the reference arm (the
FP64 oracle on a bounded sample of the 3-D wave workload) prints one JSON
line with the contract's keys, alone and under torchrun with two ranks
(rank 0 prints, the other rank exits 0 without work)."""
import json
import os
import socket
import subprocess
import sys

import pytest

from tests.conftest import ROOT

KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"}


def _json_lines(out):
    return [json.loads(l) for l in out.splitlines() if l.strip().startswith("{")]


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    line = lines[0]
    assert KEYS <= set(line)
    assert line["impl"] == "reference" and line["higher_is_better"] is True and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.slow
def test_reference_arm_under_torchrun_two_ranks():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1 and lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2


def test_paper_configs_build_the_sec51_problems():
    """The paper_ex* bench workloads are the Sec. 5.1 test problems on the
    paper's 5277^2 grid (FP64, P = 1, 6-point rule, CFL 1, beta 1)."""
    import math
    import bench
    from paper_2007_03041_gb300 import molt as M
    d1, u1 = bench._problem("paper_ex1_advection")
    d2, u2 = bench._problem("paper_ex2_diffusion")
    d3, u3 = bench._problem("paper_ex3_hj")
    for d in (d1[0], d2[0], d3[0]):
        assert (d.n[0], d.n[1], d.P, d.quad_points, d.beta, d.prec) == (5277, 5277, 1, 6, 1.0, M.PREC_F64)
        assert abs(d.hi[0] - 2 * math.pi) < 1e-15
    assert (d1[0].pde, d1[0].hamiltonian, tuple(d1[0].velocity)[:2], d1[0].cfl) == (M.PDE_HJ, M.H_LINEAR, (1.0, 1.0), 1.0)
    assert (d2[0].pde, d2[0].integrator) == (M.PDE_HEAT, M.INT_EULER)
    assert abs(d2[0].dt - 2 * math.pi / 5277) < 1e-18
    assert (d3[0].hamiltonian, d3[0].h0) == (M.H_AFFINE_SQ, 1.0)
    assert u1[0].shape == (5277, 5277) and float(abs(u3[0]).max()) == 0.0
    assert abs(float(u2[0][5277 // 4, 0]) - 1.0) < 1e-3      # sin(x) + sin(y) at y ~ pi/2, x = 0 ([y][x])


def test_advdiff_bench_workload():
    """The viscous Burgers workload: 4096^2 FP32, WENO-Z, forward Euler, and a
    splitting bound c above max |u| of the initial state."""
    import math
    import bench
    from paper_2007_03041_gb300 import molt as M
    d, u = bench._problem("advdiff_burgers4096")
    d = d[0]
    assert (d.pde, d.flux, d.weights, d.quad_points, d.integrator, d.prec) == \
        (M.PDE_ADVDIFF, M.FLUX_BURGERS, M.W_WENOZ, 5, M.INT_EULER, M.PREC_F32)
    assert d.c > float(abs(u[0]).max())
    assert abs(d.dt - 0.5 * (2 * math.pi / 4096) / d.c) < 1e-18
