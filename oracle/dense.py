"""Oracle: the partial sums S_P of one axis as a dense matrix, for the linear schemes.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__``.

S_P = sum_{p<=P} D^p along a line (Sec. 2.1-2.4, computed line by line in
``sweep.partial_sum_lines``) is a linear map of the line's values.  Its matrix
M, (S_P v)_i = sum_j M_ij v_j, is the image of the identity: row j of
partial_sum_lines(I) is S_P[e_j], the j-th column of M.  The linear time
integrators of ``schemes`` -- the central-difference wave step (Sec. 2.1) and
the SSP-RK3 heat step (Sec. 2.5) -- apply S_P along every axis of the grid;
here that is a matrix product along the axis.  Same map, other evaluation
order: the results agree with ``schemes`` to rounding (pinned in
tests/test_oracle_dense.py), at a cost set by matrix products instead of
Python loops over points, so whole 512^3 runs are within reach.
"""
import numpy as np

from .sweep import partial_sum_lines, BC_PERIODIC
from .schemes import SSPRK3


def axis_matrix(n, alpha, dx, op, bc, npts, P):
    """M with (S_P v)_i = sum_j M_ij v_j on a line of n stored points."""
    return np.ascontiguousarray(partial_sum_lines(np.eye(n), alpha, dx, op, bc, npts, P).T)


def apply_axis(M, u, ax):
    """M applied to every line of u along numpy axis ``ax``."""
    u = np.asarray(u, dtype=np.float64)
    if ax == u.ndim - 1:
        return np.matmul(u, M.T)
    if ax == 0:
        return (M @ u.reshape(u.shape[0], -1)).reshape(u.shape)
    ua = np.moveaxis(u, ax, -2)
    return np.moveaxis(np.matmul(M, ua), -2, ax)


def wave_matrices(shape, dxs, dt, c=1.0, beta=0.8, bc=None, npts=6, P=2):
    """Per numpy axis, the matrix of S_P with alpha = beta/(c dt) (Sec. 2.1)."""
    bc = bc or [BC_PERIODIC] * len(shape)
    alpha = beta / (c * dt)
    return [axis_matrix(shape[ax], alpha, dxs[ax], "0", bc[ax], npts, P) for ax in range(len(shape))]


def wave_step(u, u_prev, mats, beta=0.8, from_rest=False):
    """The central-difference wave step of ``schemes.wave_step`` with the axis
    sums as matrix products: u^{n+1} = 2u^n - u^{n-1} - beta^2 sum_d S_{P,d}[u^n]
    (Taylor start from rest: u^0 - beta^2/2 sum_d S_{P,d}[u^0])."""
    S = np.zeros_like(u, dtype=np.float64)
    for ax, M in enumerate(mats):
        S += apply_axis(M, u, ax)
    if from_rest:
        return u - 0.5 * beta * beta * S
    return 2.0 * u - u_prev - beta * beta * S


def heat_matrices(shape, dxs, dt, kappa=1.0, beta=0.6, bc=None, npts=3, P=3):
    """Per numpy axis, the matrix of S_P with alpha = beta/sqrt(kappa dt) (Sec. 2.1)."""
    bc = bc or [BC_PERIODIC] * len(shape)
    alpha = beta / np.sqrt(kappa * dt)
    return [axis_matrix(shape[ax], alpha, dxs[ax], "0", bc[ax], npts, P) for ax in range(len(shape))]


def heat_step(u, mats, beta=0.6):
    """The SSP-RK3 heat step of ``schemes.heat_step`` with dt F(u) =
    -beta^2 sum_d S_{P,d}[u] as matrix products (Shu-Osher stages)."""
    un = np.asarray(u, dtype=np.float64)
    us = un
    for a0, a1 in SSPRK3:
        F = np.zeros_like(un)
        for ax, M in enumerate(mats):
            F += apply_axis(M, us, ax)
        us = a0 * un + a1 * (us - beta * beta * F)
    return us
