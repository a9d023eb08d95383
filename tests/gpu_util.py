"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

TOL_F64 = 1e-12   # relative L2, FP64 sweeps
TOL_F32 = 1e-5    # relative L2, FP32 sweeps


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2007_03041_gb300 import molt
    molt.load_library()


def rel_l2(got, want):
    want = np.asarray(want)
    den = np.linalg.norm(want)
    return np.linalg.norm(np.asarray(got) - want) / (den if den > 0 else 1.0)


def np_axis(ndim, axis):
    """numpy axis of the C-ABI axis (0 = x = last numpy axis)."""
    return ndim - 1 - axis


def to_dev(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def tol_for(prec):
    from paper_2007_03041_gb300 import molt as M
    return TOL_F64 if prec == M.PREC_F64 else TOL_F32


def state_dtype(prec):
    from paper_2007_03041_gb300 import molt as M
    return torch.float32 if prec == M.PREC_F32 else torch.float64


# Element-wise bound next to the relative L2 norm: the largest pointwise error
# over the largest value.  An error confined to a few points of a long line
# (the ghost-affected ends) is diluted in the L2 norm but not here.  FP32:
# D = v - L^{-1}[v] loses about 2^-24 / nu^2 of |v| to cancellation at small
# nu (1.1e-5 at nu = 0.075, the heat problems' 128^2 grid with dt = h/2), and
# the largest point of a field sits a few times above its RMS, so 5e-5; an
# error at the line ends from a wrong ghost or boundary term is 1e-3 or more.
MAX_F64 = 1e-11
MAX_F32 = 5e-5


def max_for(prec):
    from paper_2007_03041_gb300 import molt as M
    return MAX_F64 if prec == M.PREC_F64 else MAX_F32


def max_rel(got, want):
    want = np.asarray(want)
    den = np.abs(want).max() if want.size else 0.0
    return np.abs(np.asarray(got) - want).max() / (den if den > 0 else 1.0) if want.size else 0.0


def assert_parity(got, want, tol_l2, tol_max, line_axis=None, what=""):
    """rel-L2 <= tol_l2, max-abs <= tol_max * max|want|, and the first and
    last 4 points of every line along ``line_axis`` (numpy axis) held to the
    same max-abs bound on their own."""
    got = np.asarray(got)
    want = np.asarray(want)
    e2 = rel_l2(got, want)
    em = max_rel(got, want)
    assert e2 <= tol_l2, "%s rel-L2 %.3e > %.1e" % (what, e2, tol_l2)
    assert em <= tol_max, "%s max-abs %.3e > %.1e (x max|want|)" % (what, em, tol_max)
    if line_axis is not None and got.shape[line_axis] > 0:
        den = np.abs(want).max()
        den = den if den > 0 else 1.0
        g = np.moveaxis(got, line_axis, -1)
        w = np.moveaxis(want, line_axis, -1)
        k = min(4, g.shape[-1])
        for sl, name in ((np.s_[..., :k], "first"), (np.s_[..., -k:], "last")):
            ee = np.abs(g[sl] - w[sl]).max() / den
            assert ee <= tol_max, "%s %s %d points of the lines: %.3e > %.1e" % (what, name, k, ee, tol_max)
    return e2, em



def max_bound(tol_l2):
    """The element-wise bound (over max|want|) that goes with a relative-L2
    bound: the FP64 one for FP64 tolerances, else five times the L2 bound
    (the ratio of MAX_F32 to TOL_F32)."""
    return MAX_F64 if tol_l2 <= TOL_F64 else 5.0 * tol_l2


def assert_grid_parity(got, want, tol_l2, what="", ends=True):
    """assert_parity with the element-wise bound of ``tol_l2`` and, with
    ``ends``, the first and last 4 points of the lines along every axis of
    the grid (sampled points: ends=False)."""
    want = np.asarray(want)
    for ax in (range(want.ndim) if ends and want.ndim else [None]):
        assert_parity(got, want, tol_l2, max_bound(tol_l2), line_axis=ax, what=what)
