"""Descriptor validation and argument checks of the C ABI, on the host: every
rejected descriptor makes molt_create return its status and name the reason
(molt_last_error(NULL)) before any device work, and the entry points reject
a null context.  No GPU needed: none of these calls reaches CUDA."""
import ctypes
import math
import os

import pytest

from paper_2007_03041_gb300 import molt as M


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(M.LIB_PATH):
        from paper_2007_03041_gb300 import build
        build.build()
    return M.load_library()


def _create(lib, descs):
    arr = (M.molt_desc * len(descs))(*descs)
    ctx = ctypes.c_void_p()
    st = lib.molt_create(arr, len(descs), None, ctypes.byref(ctx))
    msg = lib.molt_last_error(None)
    assert not ctx.value, "a rejected descriptor must not return a context"
    return st, (msg.decode() if msg else "")


def _desc(**kw):
    shape = kw.pop("shape", (16, 16))
    return M.make_desc(shape, **kw)


def _set(**fields):
    def f(d):
        for k, v in fields.items():
            if isinstance(v, tuple):
                getattr(d, k)[v[0]] = v[1]
            else:
                setattr(d, k, v)
        return d
    return f


CASES = [
    # (descriptor keywords, mutation, status, words of the reason)
    ({}, _set(ndim=0), M.MOLT_EINVAL, "ndim"),
    ({}, _set(ndim=4), M.MOLT_EINVAL, "ndim"),
    ({}, _set(n=(1, 0)), M.MOLT_EINVAL, "n must be >= 1"),
    ({}, _set(n=(0, (1 << 20) + 1)), M.MOLT_EINVAL, "2^20"),
    ({}, _set(bc=(0, 7)), M.MOLT_EINVAL, "boundary"),
    ({"shape": (1,), "bc": [M.BC_DIRICHLET]}, None, M.MOLT_EINVAL, "Dirichlet axes need n >= 2"),
    ({}, _set(hi=(1, 0.0)), M.MOLT_EINVAL, "hi must exceed lo"),
    ({"shape": (16,)}, _set(n=(2, 5)), M.MOLT_EINVAL, "unused axes"),
    ({"P": 0}, None, M.MOLT_EINVAL, "P must be in 1..64"),
    ({"P": 65}, None, M.MOLT_EINVAL, "P must be in 1..64"),
    ({"quad_points": 4}, None, M.MOLT_EINVAL, "quad_points"),
    ({"weights": 3}, None, M.MOLT_EINVAL, "unknown weights"),
    ({"weights": M.W_WENOZ, "quad_points": 6}, None, M.MOLT_EINVAL, "quad_points = 5"),
    ({"prec": 3}, None, M.MOLT_EINVAL, "precision"),
    ({"pde": 4}, None, M.MOLT_EINVAL, "unknown pde"),
    ({"flux": 2}, None, M.MOLT_EINVAL, "unknown flux"),
    ({"beta": 0.0}, None, M.MOLT_EINVAL, "beta must be positive"),
    ({"beta": float("nan")}, None, M.MOLT_EINVAL, "beta must be positive"),
    ({"hamiltonian": 3}, None, M.MOLT_EINVAL, "hamiltonian"),
    ({"velocity": (math.inf, 0.0)}, None, M.MOLT_EINVAL, "velocity must be finite"),
    ({"h0": math.nan}, None, M.MOLT_EINVAL, "h0 must be finite"),
    ({"integrator": 3}, None, M.MOLT_EINVAL, "integrator"),
    ({"pde": M.PDE_WAVE, "integrator": M.INT_RK3}, None, M.MOLT_EINVAL, "leapfrog"),
    ({"pde": M.PDE_HJ, "bc": [M.BC_PERIODIC, M.BC_DIRICHLET]}, None, M.MOLT_EUNSUPPORTED, "periodic axes"),
    ({"pde": M.PDE_HJ, "shape": (8, 8, 8)}, None, M.MOLT_EUNSUPPORTED, "1-D and 2-D"),
    ({"pde": M.PDE_HJ, "prec": M.PREC_F32_F64UPDATE}, None, M.MOLT_EUNSUPPORTED, "Hamilton-Jacobi runs in"),
    ({"pde": M.PDE_HJ, "cfl": 0.0}, None, M.MOLT_EINVAL, "cfl must be positive"),
    ({"weights": M.W_LEARNED, "quad_points": 5, "prec": M.PREC_F64}, None, M.MOLT_EUNSUPPORTED, "MOLT_PREC_F32"),
    ({"weights": M.W_LEARNED, "quad_points": 5, "prec": M.PREC_F32, "hamiltonian": M.H_LINEAR}, None,
     M.MOLT_EUNSUPPORTED, "learned weights run with H"),
    ({"pde": M.PDE_ADVDIFF, "bc": [M.BC_DIRICHLET, M.BC_PERIODIC]}, None, M.MOLT_EUNSUPPORTED, "periodic axes"),
    ({"pde": M.PDE_ADVDIFF, "c": 0.0}, None, M.MOLT_EUNSUPPORTED, "splitting bound"),
    ({"pde": M.PDE_ADVDIFF, "diffusivity": -1.0}, None, M.MOLT_EUNSUPPORTED, "diffusivity"),
    ({"pde": M.PDE_ADVDIFF, "weights": M.W_WENOZ, "quad_points": 5, "prec": M.PREC_F32_F64UPDATE}, None,
     M.MOLT_EUNSUPPORTED, "advection-diffusion runs"),
]


@pytest.mark.parametrize("kw,mutate,status,why", CASES)
def test_rejected_descriptors_name_their_reason(lib, kw, mutate, status, why):
    d = _desc(**kw)
    if mutate is not None:
        d = mutate(d)
    st, msg = _create(lib, [d])
    assert st == status, (st, msg)
    assert why in msg, msg


def test_the_reason_names_the_problem_of_a_batch(lib):
    good = _desc()
    bad = _desc(P=0)
    st, msg = _create(lib, [good, good, bad])
    assert st == M.MOLT_EINVAL
    assert msg.startswith("problem 2:"), msg


def test_null_arguments_and_contexts(lib):
    ctx = ctypes.c_void_p()
    assert lib.molt_create(None, 1, None, ctypes.byref(ctx)) == M.MOLT_EINVAL
    arr = (M.molt_desc * 1)(_desc())
    assert lib.molt_create(arr, 0, None, ctypes.byref(ctx)) == M.MOLT_EINVAL
    assert lib.molt_create(arr, 1, None, None) == M.MOLT_EINVAL
    assert lib.molt_apply_D(None, 0, 0, M.OP_0, 1, 1.0, None, None) == M.MOLT_EINVAL
    t = (ctypes.c_double * 1)(0.0)
    assert lib.molt_step(None, None, None, 1, t) == M.MOLT_EINVAL
    assert lib.molt_set_source(None, 0, None, 0) == M.MOLT_EINVAL
    assert lib.molt_set_grid_axis(None, 0, 0, None, 0) == M.MOLT_EINVAL
    assert lib.molt_set_mlp(None, None, 0) == M.MOLT_EINVAL
    assert lib.molt_destroy(None) == M.MOLT_OK
    assert b"null context" in lib.molt_last_error(None)


def test_host_table_entry_points_reject_bad_lines(lib):
    import numpy as np
    x = np.linspace(0.0, 1.0, 8, endpoint=False)
    with pytest.raises(M.MoltError):
        M.molt_nonuniform_weights(x, 1.0, 5.0, 4)            # no 4-point rule
    with pytest.raises(M.MoltError):
        M.molt_nonuniform_weights(x, 0.5, 5.0, 6)            # nodes wider than the period
    with pytest.raises(M.MoltError):
        M.molt_nonuniform_weno_weights(x, 1.0, -1.0)         # alpha must be positive
    with pytest.raises(M.MoltError):
        M.molt_nonuniform_weno_weights(np.r_[x[:4], x[3:]], 1.0, 5.0)   # repeated node
