"""Oracle: the partial sums on blocks of lines in a process pool.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__``.

S_P acts on every grid line independently (dimensional splitting, Sec. 2.2),
so splitting an axis's lines among worker processes and concatenating their
results is the oracle's own computation (``sweep.partial_sum_lines`` on each
block).  ``hj_step`` composes the oracle's Hamilton-Jacobi step from those
sums exactly as ``schemes.hj_step`` does (pinned against it in
tests/test_oracle_parallel.py).  Learned weights travel as the network's
parameter vector; each worker builds the oracle's weight function
(``mlp.learned_weight_fn``) from it.  The pool is started with ``spawn`` so
that no worker is forked from a process that has touched the GPU.  No method
arithmetic of its own."""
import multiprocessing as mp
import os

import numpy as np

from . import mlp, schemes, sweep
from .quadrature import QuadratureRule


def _block_partial_sum(args):
    lines, alpha, dx, op, bc, npts, P, weights, theta = args
    fn = None
    if weights == "learned":
        fn = mlp.learned_weight_fn(theta, QuadratureRule(alpha * dx, npts), emulate_bf16=True)
    return sweep.partial_sum_lines(lines, alpha, dx, op, bc, npts, P, weights, fn)


class LinePool:
    def __init__(self, procs=None):
        self.nproc = max(1, procs or os.cpu_count() or 1)
        self.pool = mp.get_context("spawn").Pool(self.nproc)

    def close(self):
        self.pool.close()
        self.pool.join()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def partial_sum(self, u, axis, alpha, dx, op, bc, npts, P, weights="linear", theta=None):
        """``sweep.partial_sum`` with the lines split among the workers
        (weights "learned": the network ``theta``, BF16-emulated forward)."""
        ua = np.moveaxis(np.asarray(u, dtype=np.float64), axis, -1)
        shape = ua.shape
        lines = np.ascontiguousarray(ua.reshape(-1, shape[-1]))
        blocks = np.array_split(lines, min(self.nproc, len(lines)))
        out = self.pool.map(_block_partial_sum, [(b, alpha, dx, op, bc, npts, P, weights, theta) for b in blocks])
        return np.moveaxis(np.concatenate(out).reshape(shape), -1, axis)

    def hj_step(self, u, dxs, lagged_speeds, cfl=1.5, beta=1.0, npts=5, weights="wenoz", theta=None):
        """``schemes.hj_step`` (H = |grad u|^2/2, no source, uniform axes)."""
        alpha = beta / (cfl * min(dxs))
        dt = schemes.hj_dt(lagged_speeds, dxs, cfl)
        ders = []
        for ax in range(u.ndim):
            dm = alpha * self.partial_sum(u, ax, alpha, dxs[ax], "R", sweep.BC_PERIODIC, npts, 1, weights, theta)
            dp = -alpha * self.partial_sum(u, ax, alpha, dxs[ax], "L", sweep.BC_PERIODIC, npts, 1, weights, theta)
            ders.append((dm, dp))
        Hh, speeds = schemes.hj_hamiltonian(ders)
        return u - dt * Hh, dt, speeds

    def hj_initial_speeds(self, u, dxs, cfl=1.5, beta=1.0, npts=5, weights="wenoz", theta=None):
        """``schemes.hj_initial_speeds``: the speeds of u itself."""
        return self.hj_step(u, dxs, [1.0] * u.ndim, cfl, beta, npts, weights, theta)[2]
