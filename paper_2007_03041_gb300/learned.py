"""Training of the WENO-weight network of the learned weight path.

The paper has no learned component.  The network (5 -> 32 -> 32 -> 3, GELU,
softmax; BF16 weights, FP32 accumulation) stands in for the WENO-Z weight
formula of the nonlinear local integrals (Sec. 2.4), and the sweep falls back
to WENO-Z wherever the two differ by more than 1e-2.  This module only
drives the library's kernels: harvesting stencils from Hamilton-Jacobi runs
with WENO-Z weights (molt_step + molt_mlp_harvest), and minibatch Adam on the
mean-squared distance to the WENO-Z weights (molt_mlp_loss_grad +
molt_mlp_adam).  PyTorch only holds the device buffers.
"""
import math

import numpy as np

from . import molt as M
from . import workloads


def hj_desc(n, weights, cfl=1.5, beta=1.0):
    """2-D periodic Hamilton-Jacobi problem on [0, 2 pi]^2 (n x n, FP32, P=1,
    5-point rule, lagged adaptive dt)."""
    return M.make_desc((n, n), lo=[0.0, 0.0], hi=[2 * math.pi] * 2, P=1, quad_points=5, weights=weights,
                       beta=beta, pde=M.PDE_HJ, cfl=cfl, dt=0.0, prec=M.PREC_F32)


def linear_weights(cfl=1.5, beta=1.0):
    """d_r of the 5-point rule at nu = alpha h = beta / cfl (square grids)."""
    return M.molt_weno_linear_weights(beta / cfl)


def harvest(n=4096, steps=500, snapshots=5, count=10_000_000, seed=workloads.SEED_MLP, cfl=1.5, beta=1.0,
            u0=None):
    """Stencils and WENO-Z targets from a WENO-Z Hamilton-Jacobi run.

    Runs the n x n problem from ``u0`` (default: the seeded -cos x - cos y +
    noise state) for ``steps`` steps and harvests, at ``snapshots`` evenly
    spaced step counts (the first at step 0, the last at ``steps``), count /
    (4 snapshots) stencils for each axis and side at seeded random positions.
    The rows of every (snapshot, axis, side) class are interleaved, so any
    contiguous slice is a balanced minibatch.  Returns device tensors
    x (count, 5), y (count, 3) and the linear weights."""
    import torch
    classes = 4 * snapshots
    per = count // classes
    total = per * classes
    d = linear_weights(cfl, beta)
    x = torch.empty((total, 5), dtype=torch.float32, device="cuda")
    y = torch.empty((total, 3), dtype=torch.float32, device="cuda")
    ctx = M.molt_create(hj_desc(n, M.W_WENOZ, cfl, beta))
    try:
        u = torch.tensor(workloads.hj_initial(n) if u0 is None else u0, dtype=torch.float32, device="cuda")
        marks = [round(k * steps / max(snapshots - 1, 1)) for k in range(snapshots)]
        done, t = 0, [0.0]
        for k, mark in enumerate(marks):
            if mark > done:
                t = M.molt_step(ctx, u, None, nsteps=mark - done, t=t)
                done = mark
            for axis in (0, 1):
                for side in (0, 1):
                    cls = 4 * k + 2 * axis + side
                    pos = torch.tensor(workloads.mlp_positions(per, n, n, seed + cls), device="cuda")
                    M.molt_mlp_harvest(u, pos, axis, side, x[cls:], y[cls:], d, stride=classes)
        torch.cuda.synchronize()
    finally:
        M.molt_destroy(ctx)
    return x, y, d


def train(x, y, epochs=2, batch=16384, lr=3e-3, lr_final=3e-4, seed=workloads.SEED_MLP, log_every=0):
    """Minibatch Adam on the network from the seeded initial parameters.
    The learning rate decays geometrically from ``lr`` to ``lr_final``.
    Returns (theta FP32 master parameters, BF16 blob, [(step, loss), ...])."""
    import torch
    dev = x.device
    theta = torch.tensor(workloads.mlp_initial_params(seed), device=dev)
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    grad = torch.zeros_like(theta)
    loss = torch.zeros(4, dtype=torch.float32, device=dev)
    blob = torch.empty(M.MLP_BLOB_BYTES, dtype=torch.uint8, device=dev)
    M.molt_mlp_pack(theta, blob)
    n = x.shape[0]
    batch = max(16, batch - batch % 4)
    per_epoch = n // batch
    total = max(1, epochs * per_epoch)
    history = []
    step = 0
    for _ in range(epochs):
        for b in range(per_epoch):
            r0 = b * batch
            M.molt_mlp_loss_grad(blob, x[r0:r0 + batch], y[r0:r0 + batch], grad, loss)
            step += 1
            rate = lr * (lr_final / lr) ** ((step - 1) / max(total - 1, 1))
            M.molt_mlp_adam(theta, m, v, grad, step, rate, blob)
            if log_every and (step % log_every == 0 or step == total):
                history.append((step, float(loss[0].item())))
    torch.cuda.synchronize()
    return theta, blob, history


def evaluate(blob, x, y, d):
    """(mean-squared loss, fallback fraction) of a network on stencils x with
    WENO-Z targets y."""
    import torch
    grad = torch.zeros(M.MLP_PARAMS, dtype=torch.float32, device=x.device)
    loss = torch.zeros(4, dtype=torch.float32, device=x.device)
    M.molt_mlp_loss_grad(blob, x, y, grad, loss)
    w = torch.empty_like(y)
    fb = torch.zeros(1, dtype=torch.int64, device=x.device)
    M.molt_mlp_forward(blob, x, w, d=d, fallbacks=fb)
    torch.cuda.synchronize()
    return float(loss[0].item()), float(fb.item()) / max(1, x.shape[0])
