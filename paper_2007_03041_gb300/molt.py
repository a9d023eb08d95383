"""Thin ctypes binding of the C ABI in include/molt.h (argument marshalling only).

Every computation runs in the CUDA kernels of ``libmolt.so``; there is no
fallback: if the library is missing or no GPU is present, the calls raise.
Arrays are torch CUDA tensors (dense, C-ordered [z][y][x]); ``axis`` follows
the C ABI (0 = x, the contiguous axis).
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmolt.so")

MOLT_OK, MOLT_EINVAL, MOLT_ENOMEM, MOLT_ECUDA, MOLT_ETIMEOUT, MOLT_ENONFINITE, MOLT_EUNSUPPORTED = range(7)
BC_PERIODIC, BC_DIRICHLET = 0, 1
OP_L, OP_R, OP_0 = 0, 1, 2
PREC_F64, PREC_F32_F64UPDATE, PREC_F32 = 0, 1, 2
PDE_HEAT, PDE_WAVE, PDE_HJ, PDE_ADVDIFF = 0, 1, 2, 3
FLUX_LINEAR, FLUX_BURGERS = 0, 1
W_LINEAR, W_WENOZ, W_LEARNED = 0, 1, 2
H_HALF_SQ, H_LINEAR, H_AFFINE_SQ = 0, 1, 2
INT_DEFAULT, INT_EULER, INT_RK3 = 0, 1, 2

EXPORTS = ("molt_create", "molt_apply_D", "molt_step", "molt_set_option", "molt_profile_read", "molt_destroy",
           "molt_last_error", "molt_wave_step_noalloc", "molt_batch_tile_shape", "molt_set_mlp", "molt_mlp_stats",
           "molt_weno_linear_weights", "molt_mlp_pack", "molt_mlp_forward", "molt_mlp_loss_grad", "molt_mlp_adam",
           "molt_mlp_harvest", "molt_quadrature_weights", "molt_set_source", "molt_set_grid_axis",
           "molt_nonuniform_weights", "molt_nonuniform_weno_weights", "molt_plan_sweep")
NU_WENO_SLOTS = 30
MLP_PARAMS = 1347
MLP_BLOB_BYTES = 3728
OPT_TMA, OPT_PROFILE, OPT_WAIT_LIMIT, OPT_TEST_SKIP_ARRIVE, OPT_LANES, OPT_AXIS_STREAMS, OPT_XLINES = 0, 1, 2, 3, 4, 5, 6
(KERNEL_STORE, KERNEL_ACC_SET, KERNEL_ACC_ADD, KERNEL_HEAT_FINAL, KERNEL_WAVE_FINAL, KERNEL_HJ_X, KERNEL_HJ_Y,
 KERNEL_UPDATE, KERNEL_BATCH, KERNEL_TRANSPOSE, KERNEL_FLUX, KERNEL_LANES_STORE, KERNEL_LANES_ACC_SET,
 KERNEL_LANES_ACC_ADD, KERNEL_LANES_WAVE_FINAL, KERNEL_XLINES_STORE, KERNEL_XLINES_ACC_SET,
 KERNEL_XLINES_ACC_ADD) = range(18)


class molt_desc(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("n", ctypes.c_int64 * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("bc", ctypes.c_int * 3),
        ("P", ctypes.c_int),
        ("quad_points", ctypes.c_int),
        ("weights", ctypes.c_int),
        ("beta", ctypes.c_double),
        ("pde", ctypes.c_int),
        ("c", ctypes.c_double),
        ("diffusivity", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("prec", ctypes.c_int),
        ("hamiltonian", ctypes.c_int),
        ("velocity", ctypes.c_double * 3),
        ("h0", ctypes.c_double),
        ("integrator", ctypes.c_int),
        ("flux", ctypes.c_int),
    ]


class molt_sweep_plan(ctypes.Structure):
    _fields_ = [
        ("points_per_lane", ctypes.c_int32),
        ("warps_per_line", ctypes.c_int32),
        ("lines_per_cta", ctypes.c_int32),
        ("threads_per_cta", ctypes.c_int32),
        ("ctas", ctypes.c_int64),
        ("smem_bytes", ctypes.c_int64),
        ("exact_fit", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class MoltError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("molt status %d: %s" % (status, msg))
        self.status = status


_lib = None


def load_library(path=LIB_PATH):
    """Load libmolt.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("libmolt.so not built: run __graft_entry__.build() (needs nvcc)")
        lib = ctypes.CDLL(path)
        lib.molt_create.argtypes = [ctypes.POINTER(molt_desc), ctypes.c_int, ctypes.c_void_p,
                                    ctypes.POINTER(ctypes.c_void_p)]
        lib.molt_apply_D.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
        lib.molt_step.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                  ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        lib.molt_set_option.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64]
        lib.molt_profile_read.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_int64)]
        lib.molt_destroy.argtypes = [ctypes.c_void_p]
        lib.molt_batch_tile_shape.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int] + \
            [ctypes.POINTER(ctypes.c_int)] * 3
        lib.molt_batch_tile_shape.restype = ctypes.c_int
        lib.molt_wave_step_noalloc.argtypes = [ctypes.POINTER(molt_desc), ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
        lib.molt_wave_step_noalloc.restype = ctypes.c_int
        vp, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
        lib.molt_set_mlp.argtypes = [vp, vp, ctypes.c_size_t]
        lib.molt_set_source.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int]
        lib.molt_set_grid_axis.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(dbl), i64]
        lib.molt_nonuniform_weights.argtypes = [ctypes.POINTER(dbl), i64, dbl, dbl, ctypes.c_int,
                                                ctypes.POINTER(dbl), ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
        lib.molt_nonuniform_weno_weights.argtypes = [ctypes.POINTER(dbl), i64, dbl, dbl, ctypes.POINTER(dbl),
                                                     ctypes.POINTER(dbl)]
        lib.molt_plan_sweep.argtypes = [ctypes.POINTER(molt_desc), ctypes.c_int, ctypes.c_int, ctypes.c_int, dbl,
                                        ctypes.POINTER(molt_sweep_plan)]
        lib.molt_mlp_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.c_int]
        lib.molt_weno_linear_weights.argtypes = [dbl, ctypes.POINTER(dbl)]
        lib.molt_quadrature_weights.argtypes = [ctypes.c_int, dbl, ctypes.POINTER(dbl), ctypes.POINTER(dbl),
                                                ctypes.POINTER(dbl)]
        lib.molt_mlp_pack.argtypes = [vp, vp, vp]
        lib.molt_mlp_forward.argtypes = [vp, vp, i64, ctypes.POINTER(dbl), vp, vp, vp]
        lib.molt_mlp_loss_grad.argtypes = [vp, vp, vp, i64, vp, vp, vp]
        lib.molt_mlp_adam.argtypes = [vp, vp, vp, vp, i64, dbl, dbl, dbl, dbl, vp, vp]
        lib.molt_mlp_harvest.argtypes = [vp, i64, i64, vp, i64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(dbl), vp,
                                         vp, i64, vp]
        for f in ("molt_set_mlp", "molt_set_source", "molt_set_grid_axis", "molt_nonuniform_weights", "molt_mlp_stats",
                  "molt_nonuniform_weno_weights", "molt_plan_sweep", "molt_weno_linear_weights", "molt_quadrature_weights",
                  "molt_mlp_pack", "molt_mlp_forward",
                  "molt_mlp_loss_grad", "molt_mlp_adam", "molt_mlp_harvest"):
            getattr(lib, f).restype = ctypes.c_int
        lib.molt_last_error.argtypes = [ctypes.c_void_p]
        lib.molt_last_error.restype = ctypes.c_char_p
        for f in ("molt_create", "molt_apply_D", "molt_step", "molt_set_option", "molt_profile_read", "molt_destroy"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def make_desc(shape_xyz, lo=None, hi=None, bc=None, P=1, quad_points=6, weights=W_LINEAR, beta=1.0,
              pde=PDE_HEAT, c=1.0, diffusivity=1.0, cfl=1.0, dt=0.0, prec=PREC_F64, hamiltonian=H_HALF_SQ,
              velocity=(0.0, 0.0, 0.0), h0=0.0, integrator=INT_DEFAULT, flux=FLUX_LINEAR):
    """Descriptor for a grid whose sizes are given x first (n_x, n_y, n_z)."""
    nd = len(shape_xyz)
    d = molt_desc()
    d.ndim = nd
    for i in range(3):
        d.n[i] = int(shape_xyz[i]) if i < nd else 1
        d.lo[i] = (lo[i] if lo is not None and i < nd else 0.0)
        d.hi[i] = (hi[i] if hi is not None and i < nd else 1.0)
        d.bc[i] = (bc[i] if bc is not None and i < nd else BC_PERIODIC)
    d.P, d.quad_points, d.weights, d.beta = P, quad_points, weights, beta
    d.pde, d.c, d.diffusivity, d.cfl, d.dt, d.prec = pde, c, diffusivity, cfl, dt, prec
    d.hamiltonian, d.h0, d.integrator, d.flux = hamiltonian, h0, integrator, flux
    for i in range(3):
        d.velocity[i] = velocity[i] if i < len(velocity) else 0.0
    return d


def _check(lib, ctx, st):
    if st != MOLT_OK:
        msg = lib.molt_last_error(ctx)
        raise MoltError(st, msg.decode() if msg else "")


def _ptr(t):
    if not t.is_cuda:
        raise ValueError("molt arrays must be CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("molt arrays must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def molt_create(descs, stream=None):
    """Create a context; ``stream`` is a torch.cuda.Stream (default: current)."""
    import torch
    lib = load_library()
    if isinstance(descs, molt_desc):
        descs = [descs]
    arr = (molt_desc * len(descs))(*descs)
    if stream is None:
        stream = torch.cuda.current_stream()
    ctx = ctypes.c_void_p()
    st = lib.molt_create(arr, len(descs), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(ctx))
    _check(lib, None, st)
    return ctx


def molt_apply_D(ctx, problem, axis, op, P, alpha, inp, out):
    lib = load_library()
    _check(lib, ctx, lib.molt_apply_D(ctx, problem, axis, op, P, float(alpha), _ptr(inp), _ptr(out)))


def molt_step(ctx, u, u_prev=None, nsteps=1, t=None):
    """Advance all problems; ``u``/``u_prev`` are lists of tensors (or one
    tensor); returns the list of times."""
    lib = load_library()
    if not isinstance(u, (list, tuple)):
        u = [u]
        if u_prev is not None:
            u_prev = [u_prev]
    n = len(u)
    up = (ctypes.c_void_p * n)(*[_ptr(x) for x in u])
    pp = None
    if u_prev is not None:
        pp = (ctypes.c_void_p * n)(*[(_ptr(x) if x is not None else None) for x in u_prev])
    tt = (ctypes.c_double * n)(*([0.0] * n if t is None else list(t)))
    _check(lib, ctx, lib.molt_step(ctx, up, pp, int(nsteps), tt))
    return list(tt)


def molt_set_option(ctx, option, value):
    lib = load_library()
    _check(lib, ctx, lib.molt_set_option(ctx, int(option), int(value)))


def molt_profile_read(ctx, kind):
    """(total device ms, launches) of the recorded sweeps of ``kind``; clears
    the records."""
    lib = load_library()
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(lib, ctx, lib.molt_profile_read(ctx, int(kind), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def molt_wave_step_noalloc(desc, u, u_prev, u_next, from_rest, stream=None):
    """One wave step with no device allocation (scratch in a static device
    array of the library); raises MoltError on a non-zero status."""
    import torch
    lib = load_library()
    if stream is None:
        stream = torch.cuda.current_stream()
    prev = _ptr(u_prev) if u_prev is not None else None
    st = lib.molt_wave_step_noalloc(ctypes.byref(desc), _ptr(u), prev, _ptr(u_next), int(from_rest),
                                    ctypes.c_void_p(stream.cuda_stream))
    if st != MOLT_OK:
        raise MoltError(st, "molt_wave_step_noalloc")


def molt_batch_tile_shape(ctx, problem, axis):
    """(points per lane, warps per line, lines per tile) the batched step's
    autotuner chose for (problem, axis)."""
    lib = load_library()
    v = [ctypes.c_int() for _ in range(3)]
    _check(lib, ctx, lib.molt_batch_tile_shape(ctx, problem, axis, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def molt_destroy(ctx):
    lib = load_library()
    _check(lib, ctx, lib.molt_destroy(ctx))


# ------------------------------------------------------------ learned weights
def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _status(st, what):
    if st != MOLT_OK:
        raise MoltError(st, what)


def _dvec3(d):
    return None if d is None else (ctypes.c_double * 3)(*[float(v) for v in d])


def molt_set_mlp(ctx, blob):
    """Install the BF16 network (a CUDA or CPU uint8 tensor of MLP_BLOB_BYTES)."""
    lib = load_library()
    if not blob.is_contiguous():
        raise ValueError("network blob must be contiguous")
    _check(lib, ctx, lib.molt_set_mlp(ctx, ctypes.c_void_p(blob.data_ptr()), blob.numel() * blob.element_size()))


def molt_set_source(ctx, problem, coef, degree=None):
    """Source F(x, t) = sum_k t^k coef[k] of a Hamilton-Jacobi problem: coef
    is a CUDA tensor of shape (degree+1, *state shape) in the state dtype
    (copied by the library), or None to remove the source."""
    lib = load_library()
    if coef is None:
        _check(lib, ctx, lib.molt_set_source(ctx, problem, None, 0))
        return
    if not coef.is_contiguous():
        raise ValueError("source coefficients must be contiguous")
    deg = coef.shape[0] - 1 if degree is None else degree
    _check(lib, ctx, lib.molt_set_source(ctx, problem, ctypes.c_void_p(coef.data_ptr()), deg))


def molt_set_grid_axis(ctx, problem, axis, x):
    """Non-uniform periodic axis from the node coordinates ``x`` of one period
    (a sequence of floats), or None for a uniform axis again."""
    lib = load_library()
    if x is None:
        _check(lib, ctx, lib.molt_set_grid_axis(ctx, problem, axis, None, 0))
        return
    arr = (ctypes.c_double * len(x))(*[float(v) for v in x])
    _check(lib, ctx, lib.molt_set_grid_axis(ctx, problem, axis, arr, len(x)))


def molt_nonuniform_weights(x, period, alpha, quad_points):
    """(cR (6, n), cL (6, n), q (n,)) point tables of a non-uniform periodic
    line, computed on the host by the library (no device work)."""
    import numpy as np
    lib = load_library()
    n = len(x)
    xs = (ctypes.c_double * n)(*[float(v) for v in x])
    cR, cL, q = (ctypes.c_double * (6 * n))(), (ctypes.c_double * (6 * n))(), (ctypes.c_double * n)()
    st = lib.molt_nonuniform_weights(xs, n, float(period), float(alpha), int(quad_points), cR, cL, q)
    if st != MOLT_OK:
        raise MoltError(st, "molt_nonuniform_weights")
    return (np.frombuffer(cR, dtype=np.float64).reshape(6, n).copy(),
            np.frombuffer(cL, dtype=np.float64).reshape(6, n).copy(), np.frombuffer(q, dtype=np.float64).copy())


def molt_nonuniform_weno_weights(x, period, alpha):
    """(wR (30, n), wL (30, n)) WENO-Z point tables (5-point rule) of a
    non-uniform periodic line, computed on the host by the library."""
    import numpy as np
    lib = load_library()
    n = len(x)
    xs = (ctypes.c_double * n)(*[float(v) for v in x])
    wR, wL = (ctypes.c_double * (NU_WENO_SLOTS * n))(), (ctypes.c_double * (NU_WENO_SLOTS * n))()
    st = lib.molt_nonuniform_weno_weights(xs, n, float(period), float(alpha), wR, wL)
    if st != MOLT_OK:
        raise MoltError(st, "molt_nonuniform_weno_weights")
    return (np.frombuffer(wR, dtype=np.float64).reshape(NU_WENO_SLOTS, n).copy(),
            np.frombuffer(wL, dtype=np.float64).reshape(NU_WENO_SLOTS, n).copy())


def molt_plan_sweep(desc, axis, op, P, alpha):
    """Tile plan of molt_apply_D(op, P, alpha) along ``axis`` (host only):
    dict of points_per_lane, warps_per_line, lines_per_cta, threads_per_cta,
    ctas, smem_bytes, exact_fit."""
    lib = load_library()
    out = molt_sweep_plan()
    st = lib.molt_plan_sweep(ctypes.byref(desc), int(axis), int(op), int(P), float(alpha), ctypes.byref(out))
    if st != MOLT_OK:
        msg = lib.molt_last_error(None)
        raise MoltError(st, msg.decode() if msg else "molt_plan_sweep")
    return {f: getattr(out, f) for f, _ in molt_sweep_plan._fields_ if f != "reserved"}


def molt_mlp_stats(ctx, reset=False):
    """(stencils evaluated, WENO-Z fallbacks) of the context's learned sweeps."""
    lib = load_library()
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(lib, ctx, lib.molt_mlp_stats(ctx, ctypes.byref(a), ctypes.byref(b), 1 if reset else 0))
    return a.value, b.value


def molt_weno_linear_weights(nu):
    """Linear weights (d_0, d_1, d_2) of the 5-point rule at nu = alpha*h."""
    lib = load_library()
    d = (ctypes.c_double * 3)()
    _status(lib.molt_weno_linear_weights(float(nu), d), "molt_weno_linear_weights")
    return tuple(d)


def molt_mlp_pack(theta, blob, stream=None):
    lib = load_library()
    _status(lib.molt_mlp_pack(_ptr(theta), _ptr(blob), _stream_ptr(stream)), "molt_mlp_pack")


def molt_mlp_forward(blob, x, w, d=None, fallbacks=None, stream=None):
    """Network weights w (n x 3) of raw stencils x (n x 5); with linear
    weights ``d`` the WENO-Z fallback applies (count added to ``fallbacks``,
    a CUDA int64 tensor of one element)."""
    lib = load_library()
    fb = _ptr(fallbacks) if fallbacks is not None else None
    _status(lib.molt_mlp_forward(_ptr(blob), _ptr(x), int(x.shape[0]), _dvec3(d), _ptr(w), fb, _stream_ptr(stream)),
            "molt_mlp_forward")


def molt_mlp_loss_grad(blob, x, y, grad, loss, stream=None):
    lib = load_library()
    _status(lib.molt_mlp_loss_grad(_ptr(blob), _ptr(x), _ptr(y), int(x.shape[0]), _ptr(grad), _ptr(loss),
                                   _stream_ptr(stream)), "molt_mlp_loss_grad")


def molt_mlp_adam(theta, m, v, grad, step, lr, blob, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    lib = load_library()
    _status(lib.molt_mlp_adam(_ptr(theta), _ptr(m), _ptr(v), _ptr(grad), int(step), float(lr), float(beta1),
                              float(beta2), float(eps), _ptr(blob), _stream_ptr(stream)), "molt_mlp_adam")


def molt_mlp_harvest(u, pos, axis, side, x, y=None, d=None, stride=1, stream=None):
    """Stencils at flat indices ``pos`` (int64) of the periodic 2-D FP32 state
    u (ny x nx) along ``axis`` (0: x, 1: y), side 0 (J_R) or 1 (J_L), into
    rows 0, stride, 2 stride, ... of x (n x 5); WENO-Z targets into the same
    rows of y (n x 3) with linear weights d.  x and y may be views that start
    at a row offset."""
    lib = load_library()
    ny, nx = u.shape
    _status(lib.molt_mlp_harvest(_ptr(u), int(nx), int(ny), _ptr(pos), int(pos.shape[0]), int(axis), int(side),
                                 _dvec3(d), ctypes.c_void_p(x.data_ptr()),
                                 ctypes.c_void_p(y.data_ptr()) if y is not None else None, int(stride),
                                 _stream_ptr(stream)), "molt_mlp_harvest")


def molt_quadrature_weights(quad_points, nu):
    """(c[6] on offsets -3..2, sub[3][4], d[3]) of the rule the sweeps use."""
    lib = load_library()
    c = (ctypes.c_double * 6)()
    sub = (ctypes.c_double * 12)()
    d = (ctypes.c_double * 3)()
    _status(lib.molt_quadrature_weights(int(quad_points), float(nu), c, sub, d), "molt_quadrature_weights")
    return list(c), [list(sub[4 * r:4 * r + 4]) for r in range(3)], list(d)
