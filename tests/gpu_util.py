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
