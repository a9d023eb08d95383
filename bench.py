"""Benchmark: DOF updates/s of the method-of-lines-transpose wave step.

Workload (one step = every sweep of the method's hot path over the grid):
3-D linear wave u_tt = c^2 Lap u, c = 1, on [0,1]^3 with Dirichlet
boundaries, 512^3 nodes, P = 2 successive-convolution terms, 6-point
quadrature, dt = 2h, beta = 0.8, sweeps in FP32 with the boundary solve and
the leapfrog update in FP64; u0 = 16 seeded Gaussian bumps (synthetic).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--config C] [--headline-only]

Prints one JSON line.  ``value`` is device-timed (inputs resident in HBM,
no instrumentation in the timed region), ``e2e`` goes through the same C-ABI
call with pinned host buffers copied in and the new state copied out every
step.  ``error_vs_oracle`` states the error of the result against the FP64
oracle: the first 10 steps on the full 512^3 grid and all 50 steps of the
run on a 256^3 grid, both compared in full (the oracle's axis sums as dense
matrices, oracle/dense.py).  Unless --headline-only, ``other_configs`` carries
the lines of the other workloads (2-D heat 256^2 FP64, 64 batched heat
problems, Hamilton-Jacobi 4096^2 WENO-Z, and 8192^2 with WENO-Z and with the
learned weights), each with its own clock record, roofline, oracle error and
speedup over the plain FP64 GPU form.  ``--impl reference`` times the FP64
CPU oracle on the host's cores on a bounded sample of the wave workload.
Under torchrun (N > 1) every rank advances its own replica (the path does not
shard across GPUs: replicas only); rank 0 prints.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N = 512
P = 2
QUAD = 6
BETA = 0.8
METRIC = "DOF updates/sec (3-D wave, 512^3, P=2) on GB300"
UNIT = "DOF/s"
TOL_F32 = 1e-5   # stated tolerance of the FP32-sweep forms (relative L2 vs the FP64 oracle)
TOL_F64 = 1e-12  # FP64 forms
WORKLOAD = {
    "workload": "wave3d_dirichlet_512^3_P2_quad6_beta0.8_dt2h",
    "grid": [N, N, N],
    "P": P,
    "quad_points": QUAD,
    "precision": "FP32 sweeps, FP64 boundary solve and leapfrog update",
    "l2": "inputs larger than L2 (2 x 1.07 GB FP64 state + 0.5 GB FP32 copy)",
}
# algorithmic bytes per DOF of each launch kind: x sweep: read the FP32 copy
# of u^n, write the FP32 accumulator; y (and z) sweeps: read copy + acc,
# write acc; last sweep with the FP64 leapfrog update: read copy + acc + u^n
# + u^{n-1} (FP64), write u^{n+1} (FP64) + its FP32 copy; separate update:
# read acc + u^n + u^{n-1}, write u^{n+1} + copy
BYTES_PER_DOF = {"x": 8, "yz": 12, "last_update": 36, "update": 32}
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per DOF per launch
# from one ncu capture of each kernel on the 512^3 step itself (one-pass
# metrics); a kernel changed since its capture has no entry
TRAFFIC_PER_DOF = {"wave_update_kernel (FP64 leapfrog update)": 31.65,
                   "lanes_sweep_kernel ACC_ADD (y lines)": 11.61}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def cpu_info():
    """(cores, CPU model) of the host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return os.cpu_count() or 1, model


def error_stats(got, want):
    """Relative L2, largest pointwise error over the largest value, largest
    pointwise error (numpy arrays)."""
    import numpy as np
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    den = float(np.linalg.norm(want))
    err = np.abs(got - want)
    amax = float(np.abs(want).max()) if want.size else 0.0
    return {"rel_l2": float(np.linalg.norm(got - want)) / (den if den > 0 else 1.0),
            "linf_rel": float(err.max()) / (amax if amax > 0 else 1.0), "linf": float(err.max())}


# ------------------------------------------------------------ oracle legs
def _oracle_sample(k, pool=None):
    """The FP64 oracle on a bounded sample of the wave workload: S_2 along x
    and y on k complete z-planes of the 512^3 grid, S_2 along z on k x 512
    complete z-lines, and the FP64 leapfrog update of those k x 512^2 points.
    pool: an oracle.parallel.LinePool (lines split among its processes) or
    None (one core).  Returns the elapsed seconds."""
    import numpy as np
    from oracle import sweep
    from paper_2007_03041_gb300 import workloads
    h = 1.0 / (N - 1)
    alpha = BETA / (2 * h)
    g = workloads.rng(7)
    slab = g.standard_normal((k, N, N))
    zl = g.standard_normal((N, k, N))
    ps = pool.partial_sum if pool is not None else sweep.partial_sum
    t0 = time.perf_counter()
    sx = ps(slab, 2, alpha, h, "0", "dirichlet", QUAD, P)
    sy = ps(slab, 1, alpha, h, "0", "dirichlet", QUAD, P)
    sz = ps(zl, 0, alpha, h, "0", "dirichlet", QUAD, P)
    new = 2.0 * slab - slab - BETA * BETA * (sx + sy + np.moveaxis(sz, 0, 1).reshape(slab.shape))
    el = time.perf_counter() - t0
    del new
    return el


def _sample_desc(k):
    return ("S_2 along x and y on %d complete 512^2 z-planes, along z on %d complete z-lines, and the leapfrog "
            "update (%d DOF of the 512^3 grid)" % (k, k * N, k * N * N))


def cpu_baseline(budget_s=8.0):
    """The oracle, as it stands, on the host: on every core (its lines split
    among one process per core) and on one core."""
    from oracle.parallel import LinePool
    cores, model = cpu_info()
    k_all = max(cores, 2)
    with LinePool(cores) as pool:
        _oracle_sample(1, pool)                  # worker start-up
        pts, el, reps = 0, 0.0, 0
        while el < budget_s or reps < 2:
            el += _oracle_sample(k_all, pool)
            pts += k_all * N * N
            reps += 1
    v_all = pts / el
    pts1, el1, reps1 = 0, 0.0, 0
    while el1 < budget_s / 2 or reps1 < 2:
        el1 += _oracle_sample(1)
        pts1 += N * N
        reps1 += 1
    return {"value": v_all, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": model,
            "sample": "%d repetitions of: %s; lines split among %d processes (one per core)"
                      % (reps, _sample_desc(k_all), cores),
            "one_core": {"value": pts1 / el1, "unit": UNIT, "cores": 1,
                         "sample": "%d repetitions of: %s" % (reps1, _sample_desc(1))}}


def run_reference(args):
    """The FP64 oracle as it stands on the host's cores: each step is the
    bounded sample above with as many z-planes as cores."""
    from oracle.parallel import LinePool
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    cores, model = cpu_info()
    k = max(cores, 2)
    with LinePool(cores) as pool:
        for _ in range(max(args.warmup, 1)):
            _oracle_sample(k, pool)
        tot = 0.0
        for _ in range(args.steps):
            tot += _oracle_sample(k, pool)
    value = args.steps * k * N * N / tot
    desc = _sample_desc(k) + "; lines split among %d processes (one per core)" % cores
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(WORKLOAD, sample=desc),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": model,
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def wave_error_vs_oracle(n, nsteps, stream):
    """Runs the wave workload on an n^3 grid (the seeded bumps, from rest) for
    nsteps steps and compares the final state in full with the FP64 oracle
    (oracle/dense.py: the oracle's S_2 as per-axis matrices)."""
    import numpy as np
    import torch
    from oracle import dense
    from paper_2007_03041_gb300 import molt as M
    from paper_2007_03041_gb300 import workloads
    h = 1.0 / (n - 1)
    dt = 2 * h
    u0 = workloads.wave_bumps(n)
    d = M.make_desc((n, n, n), bc=[M.BC_DIRICHLET] * 3, P=P, quad_points=QUAD, beta=BETA, pde=M.PDE_WAVE,
                    c=1.0, dt=dt, prec=M.PREC_F32_F64UPDATE)
    ctx = M.molt_create(d, stream)
    try:
        u = torch.tensor(u0, device="cuda")
        up = torch.empty_like(u)
        t = M.molt_step(ctx, u, up, nsteps=1, t=[0.0])
        if nsteps > 1:
            M.molt_step(ctx, u, up, nsteps=nsteps - 1, t=t)
        got = u.cpu().numpy()
        del u, up
    finally:
        M.molt_destroy(ctx)
    t0 = time.perf_counter()
    mats = dense.wave_matrices(u0.shape, [h] * 3, dt, 1.0, BETA, ["dirichlet"] * 3, QUAD, P)
    prev, cur = None, u0
    for k in range(nsteps):
        prev, cur = cur, dense.wave_step(cur, prev, mats, BETA, from_rest=(k == 0))
    out = error_stats(got, cur)
    out.update(grid=[n, n, n], steps=nsteps, compared="every grid point", oracle_s=time.perf_counter() - t0,
               tolerance_rel_l2=TOL_F32)
    return out


# ------------------------------------------------------------ headline
def run_ours(args):
    import torch
    from paper_2007_03041_gb300 import molt as M
    from paper_2007_03041_gb300 import workloads

    ws, rank, local = dist_env()
    dist = ws > 1
    if dist:
        import torch.distributed as tdist
        tdist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nx, ny, nz = args.grid
    hs = [1.0 / (nx - 1), 1.0 / (ny - 1), 1.0 / (nz - 1)]
    dt = 2 * min(hs)
    d = M.make_desc((nx, ny, nz), bc=[M.BC_DIRICHLET] * 3, P=P, quad_points=QUAD, beta=BETA, pde=M.PDE_WAVE,
                    c=1.0, dt=dt, prec=M.PREC_F32_F64UPDATE)
    stream = torch.cuda.current_stream(dev)
    ctx = M.molt_create(d, stream)
    # synthetic initial state (the seeded bumps of workloads.wave_bumps,
    # evaluated on the device)
    cen, wid = workloads.wave_bump_params()
    xs = [torch.arange(m, device=dev, dtype=torch.float64) / (m - 1) for m in (nx, ny, nz)]
    u = torch.zeros((nz, ny, nx), device=dev, dtype=torch.float64)
    for (cx, cy, cz), s in zip(cen, wid):
        gx = torch.exp(-(xs[0] - cx) ** 2 / (2 * s * s))
        gy = torch.exp(-(xs[1] - cy) ** 2 / (2 * s * s))
        gz = torch.exp(-(xs[2] - cz) ** 2 / (2 * s * s))
        u += gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    for ax in range(3):
        u.select(ax, 0).zero_()
        u.select(ax, u.shape[ax] - 1).zero_()
    u0 = u.clone() if args.compare else None
    up = torch.empty_like(u)
    # the clock sampler starts before the warm-up, so that the GPU is busy
    # (and its clocks up) when the timed region begins
    clocks = ClockSampler(local)
    clocks.start()
    t = M.molt_step(ctx, u, up, nsteps=1, t=[0.0])       # start from rest
    t = M.molt_step(ctx, u, up, nsteps=args.warmup, t=t)  # warm-up
    torch.cuda.synchronize()

    def form_run(prec, nsteps):
        """(ms per step, final state) of the start step plus nsteps timed
        steps of one precision form, from the same initial state."""
        dd = M.make_desc((nx, ny, nz), bc=[M.BC_DIRICHLET] * 3, P=P, quad_points=QUAD, beta=BETA, pde=M.PDE_WAVE,
                         c=1.0, dt=dt, prec=prec)
        cx = M.molt_create(dd, stream)
        try:
            a, b = u0.clone(), torch.empty_like(u0)
            tt = M.molt_step(cx, a, b, nsteps=1, t=[0.0])
            torch.cuda.synchronize()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            M.molt_step(cx, a, b, nsteps=nsteps, t=tt)
            f1.record(stream)
            torch.cuda.synchronize()
            return f0.elapsed_time(f1) / nsteps, a
        finally:
            M.molt_destroy(cx)

    def barrier():
        if dist:
            tdist.barrier()
        torch.cuda.synchronize()

    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    t = M.molt_step(ctx, u, up, nsteps=args.steps, t=t)
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    if dist:
        tt = torch.tensor([ms], device=dev)
        tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
        ms = float(tt.item())

    # five more trials of the same length, each in its own event pair:
    # fastest, mean and spread of the step time
    trial_ms = []
    for _ in range(5 if args.steps else 0):
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        t = M.molt_step(ctx, u, up, nsteps=args.steps, t=t)
        f1.record(stream)
        torch.cuda.synchronize()
        trial_ms.append(f0.elapsed_time(f1) / args.steps)

    # per-kernel averages from a second run of the same length with an event
    # pair around every launch (the headline region above runs without them)
    M.molt_set_option(ctx, M.OPT_PROFILE, 1)
    t = M.molt_step(ctx, u, up, nsteps=args.steps, t=t)
    per_kernel, kernel_names, launches = {}, {}, {}
    for name, kinds in (("x", ((M.KERNEL_XLINES_ACC_SET, "xline_sweep_kernel ACC_SET (x lines, one warp per line)"),
                               (M.KERNEL_LANES_ACC_SET, "lanes_sweep_kernel ACC_SET (x lines)"),
                               (M.KERNEL_ACC_SET, "sweep_tma_kernel ACC_SET (x lines)"))),
                        ("yz", ((M.KERNEL_LANES_ACC_ADD, "lanes_sweep_kernel ACC_ADD (y lines)"),
                                (M.KERNEL_ACC_ADD, "sweep_tma_kernel ACC_ADD (y and z lines)"))),
                        ("last_update", ((M.KERNEL_LANES_WAVE_FINAL,
                                          "lanes_sweep_kernel WAVE_FINAL (z lines + FP64 leapfrog update)"),)),
                        ("update", ((M.KERNEL_UPDATE, "wave_update_kernel (FP64 leapfrog update)"),))):
        for kind, kname in kinds:
            tot, cnt = M.molt_profile_read(ctx, kind)
            if cnt:
                per_kernel[name] = tot / cnt
                kernel_names[name] = kname
                launches[name] = cnt / args.steps
                break
    M.molt_set_option(ctx, M.OPT_PROFILE, 0)

    # end to end: every step copies its inputs (u^n, u^{n-1}) in from pinned
    # host memory and its result u^{n+1} back out.  Two device buffer sets
    # are double-buffered: the H2D copy of step k+1's inputs and the D2H copy
    # of step k's result run on their own streams, overlapping step k's (or
    # k+1's) sweeps; each step is an independent problem read from the host.
    e2e_steps = 0 if args.no_e2e else max(4, min(args.steps, 8))
    e2e_s = 1e-9
    if e2e_steps:
        hu = torch.empty_like(u, device="cpu").pin_memory()
        hup = torch.empty_like(u, device="cpu").pin_memory()
        hout = [torch.empty_like(u, device="cpu").pin_memory() for _ in range(2)]
        hu.copy_(u)
        hup.copy_(up)
        bufs = [(u, up), (torch.empty_like(u), torch.empty_like(u))]
        s_in = torch.cuda.Stream(dev)
        s_out = torch.cuda.Stream(dev)
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]
        ev_free = [torch.cuda.Event() for _ in range(2)]

        def copy_in(b):
            with torch.cuda.stream(s_in):
                s_in.wait_event(ev_free[b])
                bufs[b][0].copy_(hu, non_blocking=True)
                bufs[b][1].copy_(hup, non_blocking=True)
                ev_in[b].record(s_in)

        def pipelined(nsteps, t):
            for b in range(2):
                ev_free[b].record(s_out)
            if nsteps:
                copy_in(0)
            for k in range(nsteps):
                b = k % 2
                if k + 1 < nsteps:
                    copy_in(1 - b)
                stream.wait_event(ev_in[b])
                t = M.molt_step(ctx, bufs[b][0], bufs[b][1], nsteps=1, t=t)
                ev_done[b].record(stream)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ev_done[b])
                    hout[b].copy_(bufs[b][0], non_blocking=True)
                    ev_free[b].record(s_out)
            torch.cuda.synchronize()
            return t

        t = pipelined(2, t)    # warm-up of the copy path
        barrier()
        e0 = time.perf_counter()
        t = pipelined(e2e_steps, t)
        barrier()
        e2e_s = max(time.perf_counter() - e0, 1e-9)
        del hu, hup, hout, bufs
    M.molt_destroy(ctx)

    dof = nx * ny * nz
    value = ws * dof * args.steps / (ms / 1e3)
    e2e = None if args.no_e2e else {"value": ws * dof * e2e_steps / e2e_s, "unit": UNIT,
                                    "h2d_bytes_per_step": 2 * 8 * dof, "d2h_bytes_per_step": 8 * dof,
                                    "steps": e2e_steps, "ms_per_step": 1e3 * e2e_s / e2e_steps,
                                    "pipelining": "double-buffered H2D/D2H on copy streams"}
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    # dominant kernel: the largest share of the step's device time
    share = {k: per_kernel[k] * launches[k] for k in per_kernel}
    dom = max(share, key=share.get)
    achieved = BYTES_PER_DOF[dom] * dof / (per_kernel[dom] / 1e3) / 1e9
    traffic = TRAFFIC_PER_DOF.get(kernel_names[dom])
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic and traffic * dof,
                "kernel": kernel_names[dom], "peak_source": "measured" if peaks else "fallback",
                "per_kernel_ms": per_kernel, "per_kernel_name": kernel_names,
                "per_kernel_gbs": {k: BYTES_PER_DOF[k] * dof / (per_kernel[k] / 1e3) / 1e9 for k in per_kernel},
                "per_kernel_frac": {k: BYTES_PER_DOF[k] * dof / (per_kernel[k] / 1e3) / 1e9 / peak
                                    for k in per_kernel},
                "launches_per_step": launches,
                "algorithmic_bytes_per_dof": {k: BYTES_PER_DOF[k] for k in per_kernel},
                "step_bytes_per_dof": sum(BYTES_PER_DOF[k] * launches[k] for k in per_kernel),
                "per_kernel_source": "CUDA events around each launch, a second run of the same length",
                "peak_nominal_gbs": HBM_NOMINAL_GBS, "frac_nominal": achieved / HBM_NOMINAL_GBS}
    if rank != 0:
        return None
    compare = None
    if args.compare:
        nst = max(2, min(args.steps, 10))
        ms32, a32 = form_run(M.PREC_F32_F64UPDATE, nst)
        ms64, a64 = form_run(M.PREC_F64, nst)
        compare = {"fp64_value": dof / (ms64 / 1e3), "fp64_ms_per_step": ms64, "mixed_ms_per_step": ms32,
                   "speedup": ms64 / ms32, "steps_compared": nst + 1,
                   "rel_l2_vs_fp64": float(torch.linalg.norm(a32 - a64) / torch.linalg.norm(a64))}
        del a32, a64
    del u, up, u0
    torch.cuda.empty_cache()
    err = None
    if not args.no_oracle and ws == 1 and [nx, ny, nz] == [N, N, N]:
        err = {"full_grid_first_steps": wave_error_vs_oracle(N, 10, stream),
               "half_grid_whole_run": wave_error_vs_oracle(N // 2, 50, stream)}
    cpu = cpu_baseline() if (ws == 1 and not args.no_cpu) else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": dict(WORKLOAD, grid=[nx, ny, nz], parallelism="replicas" if ws > 1 else "1gpu"),
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": int(round(sum(launches.values()) * args.steps)) + 1, "clocks": clk,
        "error_vs_oracle": err,
    }
    if trial_ms:
        mean = sum(trial_ms) / len(trial_ms)
        line["trials"] = {"n": len(trial_ms), "steps_each": args.steps, "min_ms_per_step": min(trial_ms),
                          "mean_ms_per_step": mean,
                          "std_ms_per_step": (sum((x - mean) ** 2 for x in trial_ms) / len(trial_ms)) ** 0.5,
                          "note": "five further timed regions of the same length after the headline one"}
    if compare:
        line["vs_plain_fp64_gpu"] = compare
    return line


# --------------------------------------------------------------- other configs
# The default line is the 3-D wave workload above.  ``--config`` times the other
# workloads of the method on the same contract (device-timed DOF/s, step-level
# algorithmic bytes, a clock record), with the error against the FP64 oracle
# and the plain FP64 GPU form of the same problem (its DOF/s, the speedup of
# the measured form over it, the relative L2 difference of the final states).
CONFIGS = {
    # heat 256^2: FP64 thread-instructions per DOF and step from one ncu
    # capture (6 sweeps x 77.3 + 3 stage updates x 4.0); the state stays in L2
    "heat256": dict(metric="DOF updates/sec (2-D heat, 256^2, P=3, FP64, SSP-RK3) on GB300",
                    bytes_per_dof=168, bound="fp64", dtype="f64", flush_l2=True, fp64_inst_per_dof=476.0,
                    dram_per_dof=None),
    "batch64": dict(metric="DOF updates/sec (64 batched 2-D heat problems, sides 128..2048, P=3) on GB300",
                    bytes_per_dof=156, bound="hbm", dtype="f32",
                    l2="inputs larger than L2 (60M points: 0.48 GB FP64 state, 1.9 GB with the stage buffers)"),
    "hj4096": dict(metric="DOF updates/sec (2-D Hamilton-Jacobi, 4096^2, WENO-Z, FP32) on GB300",
                   bytes_per_dof=20, bound="hbm", dtype="f32", flush_l2=True),
    "hj8192": dict(metric="DOF updates/sec (2-D Hamilton-Jacobi, 8192^2, WENO-Z, FP32) on GB300",
                   bytes_per_dof=20, bound="hbm", dtype="f32", l2="inputs larger than L2 (FP32 state 268 MB)"),
    "hj8192_learned": dict(metric="DOF updates/sec (2-D Hamilton-Jacobi, 8192^2, learned WENO weights, FP32) on GB300",
                           bytes_per_dof=20, bound="tensor+alu", dtype="f32",
                           l2="inputs larger than L2 (FP32 state 268 MB)"),
    # the paper's own test problems (Sec. 5.1) on its 5277^2 grid: P = 1,
    # 6-point linear quadrature, forward Euler, FP64
    "paper_ex1_advection": dict(metric="DOF updates/sec (Sec. 5.1 Example 1, 2-D linear advection, 5277^2, FP64) on GB300",
                                bytes_per_dof=40, bound="fp64", dtype="f64", fp64_inst_per_dof=54.2,
                                dram_per_dof=41.0),
    "paper_ex2_diffusion": dict(metric="DOF updates/sec (Sec. 5.1 Example 2, 2-D diffusion, 5277^2, FP64) on GB300",
                                bytes_per_dof=40, bound="fp64", dtype="f64", fp64_inst_per_dof=45.6,
                                dram_per_dof=48.0),
    # Sec. 2.5 flux-split advection-diffusion: 2-D viscous Burgers, FP32,
    # WENO-Z, forward Euler with P = 1; per step and axis: split fluxes (read
    # u, write g+, g-), three accumulating sweeps (12 B each), plus the memset
    # of acc and the update (read acc + u, write u)
    "advdiff_burgers4096": dict(metric="DOF updates/sec (2-D viscous Burgers, 4096^2, flux-split, WENO-Z, FP32) on GB300",
                                bytes_per_dof=112, bound="hbm", dtype="f32", flush_l2=True),
    "paper_ex3_hj": dict(metric="DOF updates/sec (Sec. 5.1 Example 3, 2-D Hamilton-Jacobi with source, 5277^2, FP64) on GB300",
                         bytes_per_dof=80, bound="fp64", dtype="f64", fp64_inst_per_dof=65.2, dram_per_dof=104.4),
}
# FP64-bound lines: FP64 thread-instructions (DFMA + DADD + DMUL) and DRAM bytes
# per DOF per step from one ncu capture of the step's sweeps at 4096^2 (both
# scale with the points); peak = the nominal 1.25 TFLOP/s FP64 rate as thread-
# instructions: 2 per SM per cycle, 304 over the GPU, at the 2070 MHz maximum
# SM clock
FP64_PEAK_GINST = 304 * 2.070
# GB300 HBM3e nominal bandwidth (context next to the measured copy peak)
HBM_NOMINAL_GBS = 7900.0
# grid side of the paper_ex* configs: the paper's 5277 (--size overrides it for
# profiling at other sizes; the final-time errors are reported at 5277 only)
PAPER_N = 5277
# Sec. 4.5 / Sec. 5: the paper's sustained rate on one CPU node (2 x Xeon Gold
# 6148) for these test problems; a context figure from other hardware
PAPER_NODE_DOF_PER_S = 1e8


def _problem(config, prec=None):
    """(descs, initial states as numpy arrays, u_prev needed) of a config."""
    import math
    import numpy as np
    from paper_2007_03041_gb300 import molt as M
    from paper_2007_03041_gb300 import workloads
    if config == "heat256":
        n = 256
        d = M.make_desc((n, n), P=3, quad_points=3, beta=0.6, pde=M.PDE_HEAT, dt=0.5 / n,
                        prec=M.PREC_F64 if prec is None else prec)
        return [d], [workloads.heat_modes(n)]
    if config.startswith("paper_ex"):
        n = PAPER_N
        h = 2 * math.pi / n
        # prec: FP64 as the paper, or the reduced-precision form (FP32 state
        # for Hamilton-Jacobi, FP32 sweeps with the FP64 update for heat)
        if config == "paper_ex2_diffusion":
            d = M.make_desc((n, n), lo=[0, 0], hi=[2 * math.pi] * 2, P=1, quad_points=6, beta=1.0, pde=M.PDE_HEAT,
                            dt=h, prec=M.PREC_F64 if prec is None else prec, integrator=M.INT_EULER)
            return [d], [workloads.diffusion_initial(n)]
        ex1 = config == "paper_ex1_advection"
        d = M.make_desc((n, n), lo=[0, 0], hi=[2 * math.pi] * 2, P=1, quad_points=6, beta=1.0, pde=M.PDE_HJ,
                        cfl=1.0, dt=0.0, prec=M.PREC_F64 if prec is None else prec,
                        hamiltonian=M.H_LINEAR if ex1 else M.H_AFFINE_SQ, velocity=(1.0, 1.0), h0=0.0 if ex1 else 1.0)
        return [d], [workloads.advection_initial(n) if ex1 else np.zeros((n, n))]
    if config == "advdiff_burgers4096":
        n = 4096
        h = 2 * math.pi / n
        d = M.make_desc((n, n), lo=[0, 0], hi=[2 * math.pi] * 2, P=1, quad_points=5, weights=M.W_WENOZ, beta=0.6,
                        pde=M.PDE_ADVDIFF, c=1.2, diffusivity=2e-3, dt=0.5 * h / 1.2,
                        prec=M.PREC_F32 if prec is None else prec, flux=M.FLUX_BURGERS, integrator=M.INT_EULER)
        return [d], [workloads.burgers_initial(n)]
    if config == "batch64":
        sides = workloads.batched_sides()
        descs = [M.make_desc((n, n), P=3, quad_points=3, beta=0.6, pde=M.PDE_HEAT, dt=0.5 / n,
                             prec=M.PREC_F32_F64UPDATE if prec is None else prec) for n in sides]
        return descs, workloads.batched_heat(sides=sides)
    n = 4096 if config == "hj4096" else 8192
    weights = M.W_LEARNED if config == "hj8192_learned" else M.W_WENOZ
    if prec == M.PREC_F64:
        weights = M.W_WENOZ
    seed = workloads.SEED_HJ if config == "hj4096" else workloads.SEED_HJ_LARGE
    d = M.make_desc((n, n), lo=[0, 0], hi=[2 * math.pi] * 2, P=1, quad_points=5, weights=weights, beta=1.0,
                    pde=M.PDE_HJ, cfl=1.5, dt=0.0, prec=M.PREC_F32 if prec is None else prec)
    return [d], [workloads.hj_initial(n, seed=seed)]


L2_FLUSH_BYTES = 512 << 20   # written between timed steps whose state fits in L2 (129 MB)


def _timed_steps(config, steps, warmup, prec=None, blob=None, profile_kinds=(), clocks=False, flush_l2=False):
    """Runs a config on the device: returns (ms per step, final states (device
    tensors), per-kind device ms per step, learned-weight stats, clock record
    of the timed region).  flush_l2: L2_FLUSH_BYTES are written on the stream
    right before the timed molt_step call (states that fit in L2 stay there
    across the steps of one call, as in any run of that size)."""
    import torch
    from paper_2007_03041_gb300 import molt as M
    descs, u0 = _problem(config, prec)
    f32 = descs[0].prec == M.PREC_F32
    stream = torch.cuda.Stream()
    clk = None
    with torch.cuda.stream(stream):
        ctx = M.molt_create(descs, stream)
        try:
            if blob is not None and descs[0].weights == M.W_LEARNED:
                M.molt_set_mlp(ctx, blob)
            if config == "paper_ex3_hj":
                from paper_2007_03041_gb300 import workloads
                M.molt_set_source(ctx, 0, torch.tensor(workloads.manufactured_hj_source(int(descs[0].n[0])),
                                                       device="cuda", dtype=torch.float32 if f32 else torch.float64))
            us = [torch.tensor(a, dtype=torch.float32 if f32 else torch.float64, device="cuda") for a in u0]
            # sampler first, then the warm-up: the timed steps follow busy ones
            sampler = ClockSampler(0) if clocks else None
            if sampler:
                sampler.start()
            t = M.molt_step(ctx, us, None, nsteps=warmup, t=[0.0] * len(us)) if warmup else [0.0] * len(us)
            if blob is not None and descs[0].weights == M.W_LEARNED:
                M.molt_mlp_stats(ctx, reset=True)
            stream.synchronize()
            if flush_l2:
                junk = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
                junk.fill_(1.0)
                del junk
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            t = M.molt_step(ctx, us, None, nsteps=steps, t=t)
            e1.record(stream)
            stream.synchronize()
            ms = e0.elapsed_time(e1) / steps
            if sampler:
                clk = sampler.stop()
            stats = M.molt_mlp_stats(ctx) if (blob is not None and descs[0].weights == M.W_LEARNED) else None
            # per-kind device times from a separate profiled run of the same
            # length (event pairs around each launch; no graph replay)
            kinds = {}
            if profile_kinds:
                M.molt_set_option(ctx, M.OPT_PROFILE, 1)
                pu = [x.clone() for x in us]
                M.molt_step(ctx, pu, None, nsteps=steps, t=list(t))
                for name, kind in profile_kinds:
                    tot, cnt = M.molt_profile_read(ctx, kind)
                    if cnt:
                        kinds[name] = tot / steps
                M.molt_set_option(ctx, M.OPT_PROFILE, 0)
                del pu
        finally:
            M.molt_destroy(ctx)
    return ms, us, kinds, stats, clk


def _rk3(z):
    return 1.0 + z + z * z / 2.0 + z ** 3 / 6.0


def _modal_heat(n, seed, nsteps, iy, ix, beta=0.6, npts=3, P=3):
    """Closed-form discrete solution of the periodic heat step (dt = h/2) at
    the points (iy, ix): every Fourier mode of u0 is multiplied by the RK3
    polynomial of its exact discrete symbol (oracle/stability.py) per step.
    The oracle's line-by-line step matches it to 1e-14 (tests/test_oracle_schemes.py)."""
    import math
    import numpy as np
    from oracle import stability
    from paper_2007_03041_gb300 import workloads
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


def _hj_first_step_error(n, seed, weights, blob=None, theta=None, samples=256):
    """Error of u^1 of the 2-D Hamilton-Jacobi run at sampled points against
    the oracle, which needs only the x and y lines of u^0 through each point
    (weights "wenoz" or "learned" with the same BF16 network)."""
    import math
    import numpy as np
    import torch
    from oracle import mlp, schemes, sweep
    from oracle.quadrature import QuadratureRule
    from paper_2007_03041_gb300 import molt as M
    from paper_2007_03041_gb300 import workloads
    h = 2 * math.pi / n
    u0 = workloads.hj_initial(n, seed=seed).astype(np.float32)
    d = M.make_desc((n, n), lo=[0, 0], hi=[2 * math.pi] * 2, P=1, quad_points=5,
                    weights=M.W_LEARNED if weights == "learned" else M.W_WENOZ, beta=1.0, pde=M.PDE_HJ, cfl=1.5,
                    dt=0.0, prec=M.PREC_F32)
    ctx = M.molt_create(d)
    try:
        if blob is not None:
            M.molt_set_mlp(ctx, blob)
        u = torch.tensor(u0, device="cuda")
        t = M.molt_step(ctx, u, None, nsteps=1, t=[0.0])
        u1 = u.cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    g = workloads.rng(5)
    iy, ix = g.integers(0, n, samples), g.integers(0, n, samples)
    alpha = 1.0 / (1.5 * h)
    fn = None
    if weights == "learned":
        fn = mlp.learned_weight_fn(np.asarray(theta, dtype=np.float64), QuadratureRule(1.0 / 1.5, 5),
                                   emulate_bf16=True)
    u064 = u0.astype(np.float64)
    ders = []
    for lines, pos in ((u064[iy, :], ix), (u064[:, ix].T, iy)):
        dm = alpha * sweep.partial_sum(lines, 1, alpha, h, "R", "periodic", 5, 1, weights, fn)
        dp = -alpha * sweep.partial_sum(lines, 1, alpha, h, "L", "periodic", 5, 1, weights, fn)
        r = np.arange(len(pos))
        ders.append((dm[r, pos], dp[r, pos]))
    Hh, _ = schemes.hj_hamiltonian(ders)
    want = u064[iy, ix] - t[0] * Hh
    out = error_stats(u1[iy, ix], want)
    inc = error_stats(u1[iy, ix].astype(np.float64) - u064[iy, ix], -t[0] * Hh)
    out.update(steps=1, grid=[n, n], compared="%d sampled points (the x and y lines of u^0 through each)" % samples,
               increment_rel_l2=inc["rel_l2"], tolerance_rel_l2=TOL_F32,
               note="dt is the device's lagged step (the oracle step uses the same dt)")
    return out


def _hj_first_steps_error(n, seed, nsteps):
    """Error after the first nsteps steps of the 2-D Hamilton-Jacobi run
    (WENO-Z, FP32) against the oracle on the whole grid (the oracle's line
    sums split among one process per core)."""
    import math
    import numpy as np
    import torch
    from oracle.parallel import LinePool
    from paper_2007_03041_gb300 import molt as M
    from paper_2007_03041_gb300 import workloads
    h = 2 * math.pi / n
    u0 = workloads.hj_initial(n, seed=seed).astype(np.float32)
    d = M.make_desc((n, n), lo=[0, 0], hi=[2 * math.pi] * 2, P=1, quad_points=5, weights=M.W_WENOZ, beta=1.0,
                    pde=M.PDE_HJ, cfl=1.5, dt=0.0, prec=M.PREC_F32)
    ctx = M.molt_create(d)
    try:
        u = torch.tensor(u0, device="cuda")
        t = M.molt_step(ctx, u, None, nsteps=nsteps, t=[0.0])
        got = u.cpu().numpy()
    finally:
        M.molt_destroy(ctx)
    t0 = time.perf_counter()
    uu = u0.astype(np.float64)
    tt = 0.0
    with LinePool() as pool:
        sp = pool.hj_initial_speeds(uu, [h, h])
        for _ in range(nsteps):
            uu, dt, sp = pool.hj_step(uu, [h, h], sp)
            tt += dt
    out = error_stats(got, uu)
    out.update(steps=nsteps, grid=[n, n], compared="every grid point", t_gpu=t[0], t_oracle=tt,
               oracle_s=time.perf_counter() - t0, tolerance_rel_l2=TOL_F32)
    return out


# FP32-issue bound of the Hamilton-Jacobi WENO-Z steps: thread instructions
# per DOF and step of the sweeps (x pass 204, y pass on the transposed state
# 232, from one ncu capture at 4096^2) against 128 thread instructions per SM
# per cycle (4 schedulers x 32 lanes) x 152 SMs x 2070 MHz
HJ_INST_PER_DOF = 436.0
ISSUE_PEAK_GINST = 128 * 152 * 2.070


# Sec. 5.1 figure caption: L-infinity errors on the 5277^2 grid
PAPER_LINF = {"paper_ex1_advection": 2.874e-3, "paper_ex2_diffusion": 4.010e-4, "paper_ex3_hj": 2.674e-4}


def _paper_final_error(config, prec=None):
    """Runs a Sec. 5.1 test problem from t = 0 to its final time (2 pi, 1,
    0.5) and returns (L-infinity error against the exact solution, final t,
    steps)."""
    import math
    import torch
    from paper_2007_03041_gb300 import molt as M
    from paper_2007_03041_gb300 import workloads
    descs, u0 = _problem(config, prec)
    dt_ = torch.float32 if descs[0].prec == M.PREC_F32 else torch.float64
    n = int(descs[0].n[0])
    h = 2 * math.pi / n
    ctx = M.molt_create(descs)
    try:
        if config == "paper_ex3_hj":
            M.molt_set_source(ctx, 0, torch.tensor(workloads.manufactured_hj_source(n), device="cuda", dtype=dt_))
        u = torch.tensor(u0[0], device="cuda", dtype=dt_)
        if config == "paper_ex3_hj":
            t, steps = [0.0], 0
            while t[0] < 0.5:
                t = M.molt_step(ctx, [u], None, nsteps=1, t=t)
                steps += 1
            exact = workloads.manufactured_hj_solution(n, t[0])
        elif config == "paper_ex1_advection":
            steps = n                                # dt = h: T = 2 pi
            t = M.molt_step(ctx, [u], None, nsteps=steps, t=[0.0])
            exact = workloads.advection_solution(n, t[0])
        else:
            steps = round(1.0 / h)
            t = M.molt_step(ctx, [u], None, nsteps=steps, t=[0.0])
            exact = workloads.diffusion_solution(n, t[0])
        err = float((u.double() - torch.tensor(exact, device="cuda")).abs().max())
    finally:
        M.molt_destroy(ctx)
    return err, t[0], steps


NONUNIFORM_CONFIGS = ("nonuniform4096", "nonuniform4096_wenoz", "nonuniform4096_dirichlet")


def nonuniform_line(name, steps, warmup, error=True):
    """S_2 = D_0 + D_0^2 along x, then along y, of a 4096^2 FP32 field on a
    stretched non-uniform grid (point-local weights): periodic axes with the
    6-point linear rule, or WENO-Z on the 5-point rule with point-local d_r
    (_wenoz), or Dirichlet axes whose nodes include both ends (_dirichlet);
    a step is the two applications.  Error against the FP64 oracle on four
    sampled x lines of the timed step's first pass and four y lines of one
    more y pass over the input (untimed)."""
    import math
    import numpy as np
    import torch
    from paper_2007_03041_gb300 import molt as M
    from paper_2007_03041_gb300 import workloads
    n, L = 4096, 2 * math.pi
    weno = name.endswith("_wenoz")
    dirichlet = name.endswith("_dirichlet")
    if dirichlet:
        t = np.linspace(0.0, 1.0, n)
        nodes = L * (t + 0.3 * np.sin(2 * np.pi * t) / (2 * np.pi))
        nodes[0], nodes[-1] = 0.0, L
    else:
        xi = L * np.arange(n) / n
        nodes = xi + 0.3 * np.sin(xi)
    npts = 5 if weno else 6
    bc = M.BC_DIRICHLET if dirichlet else M.BC_PERIODIC
    d = M.make_desc((n, n), lo=[0, 0], hi=[L, L], bc=[bc, bc], P=2, quad_points=npts, prec=M.PREC_F32,
                    weights=M.W_WENOZ if weno else M.W_LINEAR)
    alpha = 0.6 * n / L
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = M.molt_create(d, stream)
        try:
            M.molt_set_grid_axis(ctx, 0, 0, nodes)
            M.molt_set_grid_axis(ctx, 0, 1, nodes)
            u0 = workloads.hj_initial(n).astype(np.float32)
            u = torch.tensor(u0, dtype=torch.float32, device="cuda")
            a, b = torch.empty_like(u), torch.empty_like(u)

            def step():
                M.molt_apply_D(ctx, 0, 0, M.OP_0, 2, alpha, u, a)
                M.molt_apply_D(ctx, 0, 1, M.OP_0, 2, alpha, a, b)
            clocks = ClockSampler(0)
            clocks.start()
            for _ in range(warmup):
                step()
            stream.synchronize()
            # the 67 MB input fits in L2: flush it before every timed step
            junk = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
            pairs = []
            for _ in range(steps):
                junk.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step()
                e1.record(stream)
                pairs.append((e0, e1))
            stream.synchronize()
            clk = clocks.stop()
            ms = sum(x.elapsed_time(y) for x, y in pairs) / steps
            del junk
            err = None
            if error:
                rows = [0, 1, n // 2, n - 1]
                gx = a.cpu().numpy()[rows]
                M.molt_apply_D(ctx, 0, 1, M.OP_0, 2, alpha, u, b)
                gy = b.cpu().numpy()[:, rows].T
                err = _nonuniform_error(u0.astype(np.float64), rows, nodes, None if dirichlet else L, alpha, npts,
                                        "wenoz" if weno else "linear", gx, gy)
        finally:
            M.molt_destroy(ctx)
    dof = n * n
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = 16 * dof / (ms / 1e3) / 1e9
    kind = "Dirichlet" if dirichlet else "periodic"
    line = {
        "metric": "DOF updates/sec (S_2 along x and y, 4096^2 non-uniform %s grid, FP32%s) on GB300"
                  % (kind, ", WENO-Z" if weno else ""),
        "value": dof / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": {"workload": name, "dof": dof, "bc": kind.lower(),
                                        "grid": ("x = L (t + 0.3 sin(2 pi t)/(2 pi)), t = i/(n-1)" if dirichlet
                                                 else "x = xi + 0.3 sin xi, xi = 2 pi i/n"),
                                        "weights": "wenoz" if weno else "linear",
                                        "l2": "L2 flushed (%d MB written) before every timed step" %
                                              (L2_FLUSH_BYTES >> 20)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "scope": "two apply_D calls per step (x: one sweep; y: transpose, sweep, transpose), "
                              "8 algorithmic B/DOF each",
                     "peak_source": "measured" if peaks else "fallback"},
        "gpu_launches": 4 * steps, "clocks": clk,
    }
    if err is not None:
        line["error_vs_oracle"] = err
    return line


def _nonuniform_error(u, rows, nodes, L, alpha, npts, weights, gx, gy):
    """Error of sampled x lines (rows of S_x[u]) and y lines (columns of
    S_y[u]) against the FP64 oracle."""
    import numpy as np
    from oracle import nonuniform
    tables = nonuniform.weights(nodes, L, alpha, npts)
    weno = nonuniform.weno_tables(nodes, L, alpha, npts) if weights == "wenoz" else None
    wx = np.stack([nonuniform.partial_sum(u[j], nodes, L, alpha, "0", npts, 2, weights, tables, weno) for j in rows])
    wy = np.stack([nonuniform.partial_sum(u[:, i], nodes, L, alpha, "0", npts, 2, weights, tables, weno)
                   for i in rows])
    st = error_stats(np.concatenate([gx.ravel(), gy.ravel()]), np.concatenate([wx.ravel(), wy.ravel()]))
    st["sample"] = "x lines %s of S_x[u] and y lines %s of S_y[u] (4096 points each)" % (rows, rows)
    return st


def config_line(name, steps, warmup, compare=True, error=True, size=None):
    import torch
    from paper_2007_03041_gb300 import molt as M
    from paper_2007_03041_gb300 import workloads
    global PAPER_N
    if size:
        PAPER_N = size
    cfg = dict(CONFIGS[name])
    if name.startswith("paper_ex"):
        cfg["metric"] = cfg["metric"].replace("5277^2", "%d^2" % PAPER_N)
    descs, u0s = _problem(name)
    dof = sum(int(d.n[0] * d.n[1] * d.n[2]) for d in descs)
    extra = {}
    blob = theta = None
    if name == "hj8192_learned":
        from paper_2007_03041_gb300 import learned
        t0 = time.perf_counter()
        x, y, dlin = learned.harvest(n=4096, steps=500, snapshots=5, count=10_000_000)
        t1 = time.perf_counter()
        xe, ye = x[-500_000:], y[-500_000:]
        theta, blob, hist = learned.train(x[:-500_000], y[:-500_000], epochs=3, batch=16384, lr=3e-3, lr_final=3e-4)
        t2 = time.perf_counter()
        loss, fb = learned.evaluate(blob, xe, ye, dlin)
        extra["training"] = {"stencils": int(x.shape[0]), "harvest_s": t1 - t0, "train_s": t2 - t1,
                             "epochs": 3, "batch": 16384, "heldout_loss": loss, "heldout_fallback": fb,
                             "source": "4096^2 WENO-Z Hamilton-Jacobi run, 500 steps, 5 snapshots"}
        del x, y, xe, ye
    kinds = {"heat256": (("sweep_final", M.KERNEL_HEAT_FINAL), ("sweep_acc", M.KERNEL_ACC_SET),
                         ("update", M.KERNEL_UPDATE)),
             "batch64": (("batch_step", M.KERNEL_BATCH),),
             "hj4096": (("hj_x", M.KERNEL_HJ_X), ("hj_y", M.KERNEL_HJ_Y), ("transpose", M.KERNEL_TRANSPOSE)),
             "hj8192": (("hj_x", M.KERNEL_HJ_X), ("hj_y", M.KERNEL_HJ_Y), ("transpose", M.KERNEL_TRANSPOSE)),
             "hj8192_learned": (("hj_x", M.KERNEL_HJ_X), ("hj_y", M.KERNEL_HJ_Y), ("transpose", M.KERNEL_TRANSPOSE)),
             "paper_ex1_advection": (("hj_x", M.KERNEL_HJ_X), ("hj_y", M.KERNEL_HJ_Y),
                                     ("transpose", M.KERNEL_TRANSPOSE)),
             "paper_ex2_diffusion": (("sweep_final", M.KERNEL_HEAT_FINAL), ("sweep_acc", M.KERNEL_ACC_SET)),
             "advdiff_burgers4096": (("flux", M.KERNEL_FLUX), ("sweeps", M.KERNEL_ACC_ADD),
                                     ("sweeps_lanes", M.KERNEL_LANES_ACC_ADD), ("update", M.KERNEL_UPDATE)),
             "paper_ex3_hj": (("hj_x", M.KERNEL_HJ_X), ("hj_y", M.KERNEL_HJ_Y))}[name]
    flush = bool(cfg.get("flush_l2"))
    ms, us, per_kind, stats, clk = _timed_steps(name, steps, warmup, blob=blob, profile_kinds=kinds, clocks=True,
                                                flush_l2=flush)
    if flush:
        l2 = ("state smaller than L2: L2 flushed (%d MB written) before the timed molt_step call; the state stays "
              "in L2 across the steps of the call, as in any run of this size" % (L2_FLUSH_BYTES >> 20))
    else:
        l2 = cfg.get("l2", "inputs larger than L2")
    value = dof / (ms / 1e3)
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = cfg["bytes_per_dof"] * dof / (ms / 1e3) / 1e9
    line = {
        "metric": cfg["metric"], "value": value, "unit": UNIT, "n_gpus": 1, "steps": steps,
        "warmup": warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": cfg["dtype"], "data": "synthetic",
        "config": {"workload": name, "dof": dof, "l2": l2},
        "roofline": {"bound": cfg["bound"], "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "scope": "whole step, algorithmic bytes",
                     "algorithmic_bytes_per_dof_step": cfg["bytes_per_dof"],
                     "per_kind_ms_per_step": per_kind,
                     "peak_source": "measured" if peaks else "fallback"},
        "clocks": clk,
    }
    if cfg["bound"] == "fp64":
        ach = cfg["fp64_inst_per_dof"] * dof / (ms / 1e3) / 1e9
        line["roofline"] = {"bound": "fp64", "achieved": ach, "peak": FP64_PEAK_GINST,
                            "unit": "G FP64 thread-instructions/s", "frac": ach / FP64_PEAK_GINST,
                            "traffic": cfg["dram_per_dof"] * dof if cfg["dram_per_dof"] else None,
                            "scope": "whole step",
                            "fp64_inst_per_dof_step": cfg["fp64_inst_per_dof"],
                            "hbm_gbs_algorithmic": achieved, "per_kind_ms_per_step": per_kind,
                            "peak_source": "nominal (ncu sustained FP64 rate x maximum SM clock)"}
    if name in ("hj4096", "hj8192"):
        ach = HJ_INST_PER_DOF * dof / (ms / 1e3) / 1e9
        line["roofline"]["issue_bound"] = {"achieved": ach, "peak": ISSUE_PEAK_GINST,
                                          "unit": "G thread-instructions/s", "frac": ach / ISSUE_PEAK_GINST,
                                          "inst_per_dof_step": HJ_INST_PER_DOF,
                                          "note": "instruction issue binds before HBM for WENO-Z"}
    # error of the result against the FP64 oracle
    if error:
        import numpy as np
        if name == "heat256":
            # relative error after 10 steps (the slowest mode keeps 2% of its
            # amplitude), and after the whole run (every mode has decayed to
            # the rounding level) against the initial amplitude
            from oracle import dense
            n = int(descs[0].n[0])
            mats = dense.heat_matrices((n, n), [1.0 / n] * 2, 0.5 / n, 1.0, 0.6, None, 3, 3)
            ms10, us10 = _timed_steps(name, 10, 0)[:2]
            w = u0s[0]
            w10 = None
            for k in range(warmup + steps):
                w = dense.heat_step(w, mats, 0.6)
                if k == 9:
                    w10 = w
            e = error_stats(us10[0].cpu().numpy(), w10)
            ef = error_stats(us[0].cpu().numpy(), w)
            e.update(steps=10, grid=[n, n], compared="every grid point", tolerance_rel_l2=TOL_F64,
                     whole_run={"steps": warmup + steps,
                                "linf_vs_initial_amplitude": ef["linf"] / float(np.abs(u0s[0]).max())})
            line["error_vs_oracle"] = e
        elif name == "batch64":
            g = workloads.rng(77)
            gots, wants, worst = [], [], 0.0
            for i, (n, a0, x) in enumerate(zip([int(d.n[0]) for d in descs], u0s, us)):
                iy, ix = g.integers(0, n, 256), g.integers(0, n, 256)
                want = _modal_heat(n, 3000 + i, warmup + steps, iy, ix)
                got = x.cpu().numpy()[iy, ix]
                gots.append(got)
                wants.append(want)
                worst = max(worst, float(np.abs(got - want).max()) / float(np.abs(a0).max()))
            e = error_stats(np.concatenate(gots), np.concatenate(wants))
            e.update(steps=warmup + steps, problems=len(descs), tolerance_rel_l2=TOL_F32,
                     worst_problem_linf_vs_initial_amplitude=worst,
                     compared="256 sampled points of every problem together, against the closed-form discrete "
                              "solution (every mode times the RK3 polynomial of its exact discrete symbol)")
            line["error_vs_oracle"] = e
        elif name == "hj4096":
            line["error_vs_oracle"] = _hj_first_steps_error(4096, workloads.SEED_HJ, 2)
        elif name == "hj8192":
            line["error_vs_oracle"] = _hj_first_step_error(8192, workloads.SEED_HJ_LARGE, "wenoz")
        elif name == "hj8192_learned":
            line["error_vs_oracle"] = _hj_first_step_error(8192, workloads.SEED_HJ_LARGE, "learned", blob,
                                                           theta.cpu().numpy())
    if name.startswith("paper_ex") and PAPER_N == 5277:
        err, tf, nst = _paper_final_error(name)
        extra["final_error"] = {"linf_vs_exact": err, "t_final": tf, "steps": nst,
                                "paper_linf_5277": PAPER_LINF[name]}
        line["vs_baseline"] = value / PAPER_NODE_DOF_PER_S
        extra["vs_baseline_note"] = ("value / the paper's sustained 1e8 DOF/node/s for its Sec. 5.1 test problems "
                                     "on one CPU node (2 x Xeon Gold 6148); other hardware, context only")
    if stats is not None:
        extra["learned_stats"] = {"stencils": stats[0], "fallbacks": stats[1],
                                  "fallback_fraction": stats[1] / max(stats[0], 1)}
    if compare and name.startswith("paper_ex"):
        # the reduced-precision form of the same problem: speed and final error
        rp = M.PREC_F32_F64UPDATE if name == "paper_ex2_diffusion" else M.PREC_F32
        ms_r = _timed_steps(name, steps, warmup, prec=rp)[0]
        extra["reduced_precision_form"] = {
            "prec": "f32 sweeps + f64 update" if rp == M.PREC_F32_F64UPDATE else "f32",
            "value": dof / (ms_r / 1e3), "ms_per_step": ms_r, "speedup_vs_fp64": ms / ms_r}
        if PAPER_N == 5277:
            err_r, tf_r, _ = _paper_final_error(name, rp)
            extra["reduced_precision_form"].update(linf_vs_exact=err_r, t_final=tf_r)
    elif compare and name != "heat256":
        ms64, us64 = _timed_steps(name, steps, warmup, prec=M.PREC_F64, flush_l2=flush)[:2]
        num = sum(float(torch.linalg.norm(a.double() - b.double()) ** 2) for a, b in zip(us, us64))
        den = sum(float(torch.linalg.norm(b.double()) ** 2) for b in us64)
        extra["vs_plain_fp64_gpu"] = {"fp64_value": dof / (ms64 / 1e3), "fp64_ms_per_step": ms64,
                                      "speedup": ms64 / ms, "rel_l2_vs_fp64": (num / max(den, 1e-300)) ** 0.5,
                                      "steps_compared": warmup + steps}
        del us64
    if compare and name == "hj8192_learned":
        ms32 = _timed_steps("hj8192", steps, warmup)[0]
        extra["vs_plain_fp32_wenoz_gpu"] = {"wenoz_ms_per_step": ms32, "speedup": ms32 / ms,
                                            "note": "the same 8192^2 problem with the WENO-Z formula in FP32"}
    line.update(extra)
    del us
    torch.cuda.empty_cache()
    return line


# workloads nested in the default line: the 256^2 FP64 heat problem, the 64
# batched heat problems, the 4096^2 and 8192^2 Hamilton-Jacobi problems with
# WENO-Z and with learned weights, and the 4096^2 non-uniform sweeps
DEFAULT_OTHER = (("heat256", 100, 3), ("batch64", 20, 3), ("hj4096", 20, 3), ("hj8192", 10, 2),
                 ("hj8192_learned", 10, 2), ("nonuniform4096", 20, 3), ("nonuniform4096_wenoz", 20, 3),
                 ("nonuniform4096_dirichlet", 20, 3))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end timing")
    ap.add_argument("--no-oracle", action="store_true", help="skip the error statements against the oracle")
    ap.add_argument("--headline-only", action="store_true", help="do not run the other workloads")
    ap.add_argument("--grid", type=lambda t: [int(v) for v in t.split(",")], default=[N, N, N],
                    help="nx,ny,nz (smaller grids are for profiler captures; the metric is quoted at 512^3)")
    ap.add_argument("--config", default="wave512", choices=["wave512"] + list(NONUNIFORM_CONFIGS) + sorted(CONFIGS),
                    help="workload (default: the 3-D wave step the metric is quoted on)")
    ap.add_argument("--size", type=int, default=None,
                    help="grid side of the paper_ex* configs (default: the paper's 5277)")
    ap.add_argument("--no-compare", dest="compare", action="store_false",
                    help="skip the plain FP64 GPU form (speedup and difference)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.config in NONUNIFORM_CONFIGS:
        print(json.dumps(nonuniform_line(args.config, args.steps, args.warmup, not args.no_oracle)))
    elif args.config != "wave512":
        print(json.dumps(config_line(args.config, args.steps, args.warmup, args.compare, not args.no_oracle,
                                     args.size)))
    else:
        line = run_ours(args)
        if line is None:
            return
        ws = dist_env()[0]
        if not args.headline_only and ws == 1 and args.grid == [N, N, N]:
            line["other_configs"] = [
                nonuniform_line(nm, st, wu, not args.no_oracle) if nm in NONUNIFORM_CONFIGS
                else config_line(nm, st, wu, args.compare, not args.no_oracle) for nm, st, wu in DEFAULT_OTHER]
        print(json.dumps(line))


if __name__ == "__main__":
    main()
