/*
 * molt.h -- C ABI of the GB300 (sm_103a) library for the fast summation of
 * the method-of-lines-transpose convolution operator and the successive-
 * convolution partial sums it feeds (Christlieb, Guthrey, Sands,
 * Thavappiragasm, "Parallel Algorithms for Successive Convolution",
 * arXiv 2007.03041).
 *
 * The operators (Sec. 2.1, Eqs. "left/right-moving inverse op" and "second
 * derivative inverse op"), for a line [a, b] and a parameter alpha:
 *   L_R^{-1}[v](x) = alpha int_a^x e^{-alpha(x-s)} v(s) ds + A e^{-alpha(x-a)}
 *   L_L^{-1}[v](x) = alpha int_x^b e^{-alpha(s-x)} v(s) ds + B e^{-alpha(b-x)}
 *   L_0^{-1}[v](x) = alpha/2 int_a^b e^{-alpha|x-s|} v(s) ds
 *                    + A e^{-alpha(x-a)} + B e^{-alpha(b-x)}
 * D_* = I - L_*^{-1} (Eq. "D operators"), D^k = D(D^{k-1}) (Eq. "successive
 * relation for D"), and the partial sums sum_{p=1}^P D^p that represent
 * d_x^+ = -alpha sum D_L^p, d_x^- = alpha sum D_R^p, d_xx = -alpha^2 sum D_0^p
 * (Sec. 2.2).  Discretisation: local integrals J_R/J_L by polynomial
 * (optionally WENO-Z weighted) quadrature and the O(N) recurrences
 * I_R(x_i) = e^{-alpha dx} I_R(x_{i-1}) + J_R(x_i) (Sec. 2.4), boundary
 * constants A/B from periodicity (Sec. 2.3) or from the boundary values.
 *
 * Conventions shared by every entry point
 *   - Arrays are C-ordered [z][y][x] (x fastest, contiguous); axis 0 is x,
 *     axis 1 is y, axis 2 is z.  n[0], n[1], n[2] are the x, y, z sizes.
 *   - Periodic axes store the N unique points x_i = lo + i*h, h = (hi-lo)/N.
 *     Dirichlet axes store all nodes including both boundary nodes,
 *     h = (hi-lo)/(n-1).
 *   - All array pointers are DEVICE pointers, owned by the caller, dense and
 *     16-byte aligned.  Element type: double, except under MOLT_PREC_F32
 *     where it is float.
 *   - Work is enqueued on the CUDA stream given to molt_create; calls return
 *     before the GPU finishes, except where stated.
 *   - Every entry point returns a molt_status; nothing throws across the ABI.
 *     On failure, molt_last_error(ctx) describes the cause.  Unsupported
 *     combinations return MOLT_EUNSUPPORTED; there is no CPU fallback.
 *   - Entry points whose comment cites no section have no counterpart in the
 *     paper: lifecycle, options, profiling, tile planning, the allocation-free
 *     wave step and the learned local-integral weights.
 */
#ifndef MOLT_H
#define MOLT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MOLT_OK = 0,
  MOLT_EINVAL = 1,        /* bad argument or descriptor                       */
  MOLT_ENOMEM = 2,        /* device allocation failed                         */
  MOLT_ECUDA = 3,         /* a CUDA call failed                               */
  MOLT_ETIMEOUT = 4,      /* a device-side wait gave up (kernel returned)     */
  MOLT_ENONFINITE = 5,    /* a non-finite value reached the state             */
  MOLT_EUNSUPPORTED = 6   /* valid but not implemented combination            */
} molt_status;

typedef enum { MOLT_BC_PERIODIC = 0, MOLT_BC_DIRICHLET = 1 } molt_bc;
typedef enum { MOLT_OP_L = 0, MOLT_OP_R = 1, MOLT_OP_0 = 2 } molt_op;
typedef enum {
  MOLT_PREC_F64 = 0,            /* FP64 state, FP64 sweeps                         */
  MOLT_PREC_F32_F64UPDATE = 1,  /* FP64 state, FP32 sweeps, FP64 A/B and update    */
  MOLT_PREC_F32 = 2             /* FP32 state and sweeps, FP64 A/B                 */
} molt_prec;
typedef enum { MOLT_PDE_HEAT = 0, MOLT_PDE_WAVE = 1, MOLT_PDE_HJ = 2, MOLT_PDE_ADVDIFF = 3 } molt_pde;
/* Flux of the advection-diffusion problem u_t + sum_d d_d g_d(u) = kappa Lap u
 * (Sec. 2.5): MOLT_FLUX_LINEAR g_d = a_d u (a_d = velocity[d]),
 * MOLT_FLUX_BURGERS g_d = u^2/2 on every axis. */
typedef enum { MOLT_FLUX_LINEAR = 0, MOLT_FLUX_BURGERS = 1 } molt_flux;
typedef enum { MOLT_W_LINEAR = 0, MOLT_W_WENOZ = 1, MOLT_W_LEARNED = 2 } molt_weights;
/* Hamiltonian of the Hamilton-Jacobi step (Sec. 2.5, and the test problems
 * of Sec. 5.1: Example 1 is H = u_x + u_y, Example 3 H = (1 + u_x + u_y)^2/2),
 * a_d = velocity[d]:
 *   MOLT_H_HALF_SQ    H = |grad u|^2 / 2
 *   MOLT_H_LINEAR     H = sum_d a_d u_d                  (linear advection)
 *   MOLT_H_AFFINE_SQ  H = (h0 + sum_d a_d u_d)^2 / 2
 * The numerical Hamiltonian is local Lax-Friedrichs with r_d the largest
 * |dH/du_d| over the box of one-sided derivatives; the wave speed of axis d
 * is the grid maximum of r_d. */
typedef enum { MOLT_H_HALF_SQ = 0, MOLT_H_LINEAR = 1, MOLT_H_AFFINE_SQ = 2 } molt_hamiltonian;
/* Time integrator: MOLT_INT_DEFAULT (heat, advection-diffusion: 3-stage SSP
 * Runge-Kutta; wave: leapfrog; Hamilton-Jacobi: forward Euler),
 * MOLT_INT_EULER (forward Euler; heat, advection-diffusion and
 * Hamilton-Jacobi, the first-order coupling of the paper's test problems,
 * Sec. 5.1) or MOLT_INT_RK3 (3-stage SSP Runge-Kutta; for Hamilton-Jacobi
 * with P-term one-sided sums alpha sum_{p<=P} D_R^p, -alpha sum_{p<=P} D_L^p,
 * Sec. 2.5's coupling of an s-stage method with s-term sums). */
typedef enum { MOLT_INT_DEFAULT = 0, MOLT_INT_EULER = 1, MOLT_INT_RK3 = 2 } molt_integrator;

/* One problem: a grid, its boundary types, the quadrature and the PDE whose
 * time step molt_step advances.  Enumerations are stored as int. */
typedef struct {
  int ndim;              /* 1, 2 or 3                                            */
  int64_t n[3];          /* points per axis (x, y, z); unused axes = 1           */
  double lo[3], hi[3];   /* domain [lo, hi] per axis                             */
  int bc[3];             /* molt_bc per axis                                     */
  int P;                 /* terms of the partial sum, >= 1                       */
  int quad_points;       /* 3, 5 or 6 (J_R stencils {-1..1}, {-3..1}, {-3..2})   */
  int weights;           /* molt_weights; WENO-Z and learned need quad_points 5  */
  double beta;           /* alpha parameter (Sec. 2.1)                           */
  int pde;               /* molt_pde                                             */
  double c;              /* wave speed (wave)                                    */
  double diffusivity;    /* kappa (heat)                                         */
  double cfl;            /* CFL number (Hamilton-Jacobi)                         */
  double dt;             /* fixed time step; <= 0 selects the adaptive rule (HJ) */
  int prec;              /* molt_prec                                            */
  int hamiltonian;       /* molt_hamiltonian (Hamilton-Jacobi)                   */
  double velocity[3];    /* a_d of MOLT_H_LINEAR / MOLT_H_AFFINE_SQ              */
  double h0;             /* constant of MOLT_H_AFFINE_SQ                         */
  int integrator;        /* molt_integrator                                      */
  int flux;              /* molt_flux (advection-diffusion)                      */
} molt_desc;

typedef struct molt_ctx molt_ctx;

/* Create a context for `count` problems (count > 1: a batch advanced
 * together by molt_step).  `cuda_stream` is a cudaStream_t (NULL = legacy
 * default stream).  Validates every descriptor (n >= 1 per used axis,
 * Dirichlet axes n >= 2, P >= 1, quad_points in {3,5,6}, ...), builds the
 * quadrature tables (App. C weights by an independent moment series) and
 * allocates the workspace.  Synchronous.  On success *out owns all of it. */
molt_status molt_create(const molt_desc* descs, int count, void* cuda_stream, molt_ctx** out);

/* out = sum_{p=1}^{P} D_op^p[in] along `axis` of problem `problem`
 * (Eqs. "D operators", "successive relation for D", Sec. 2.2), with the
 * given alpha (nu = alpha*h), the problem's boundary type on that axis and
 * its quadrature/weights.  in and out: device arrays of the problem's full
 * grid; in == out is allowed.  The element type follows the precision
 * (double unless MOLT_PREC_F32); the sweeps run in FP32 unless MOLT_PREC_F64.
 * Asynchronous. */
molt_status molt_apply_D(molt_ctx* ctx, int problem, int axis, int op, int P, double alpha,
                         const void* in, void* out);

/* Advance every problem of the context by `nsteps` time steps.
 *   u[i]       device state of problem i (updated in place).
 *   u_prev[i]  wave: previous state u^{n-1} (updated to the state before the
 *              final one); NULL for heat / Hamilton-Jacobi.
 *   t_inout[i] time of problem i, host memory; advanced by the steps taken.
 *              Wave: t_inout[i] == 0 starts from rest (u_t = 0) with a
 *              second-order Taylor step and ignores u_prev[i] on entry.
 * Heat: 3-stage SSP Runge-Kutta on dt*F = -beta^2 sum_d S_{P,d}, alpha =
 * beta/sqrt(kappa dt).  Wave: u^{n+1} = 2u^n - u^{n-1} - beta^2 sum_d S_{P,d},
 * alpha = beta/(c dt); heat with MOLT_INT_EULER: u^{n+1} = u^n - beta^2
 * sum_d S_{P,d}[u^n].  Hamilton-Jacobi (H from desc.hamiltonian, periodic,
 * 1-D or 2-D): forward Euler u^{n+1} = u^n - dt (H^ - F(x, t_n)) with the
 * local Lax-Friedrichs numerical Hamiltonian H^, one-sided derivatives
 * alpha D_R, -alpha D_L, alpha = beta/(cfl min_d h_d), dt = cfl min_d h_d / c_d
 * with the wave speeds c_d of the previous step (Eq. "adaptive time rule",
 * Algorithm 1; the speeds of u^0 on the first step; at most 10 min_d h_d), and
 * the source F of molt_set_source (0 if none).
 * Advection-diffusion (periodic, 1-3 D, fixed dt): the flux split by global
 * Lax-Friedrichs, g = g^+ + g^-, g^{+-} = (g(u) +- c u)/2 with desc.c >=
 * max |g'(u)| over the run, upwind sums d^- g^+ = alpha sum_p D_R^p[g^+],
 * d^+ g^- = -alpha sum_p D_L^p[g^-] with alpha = beta/(c dt), and the
 * diffusion -kappa alpha_nu^2 sum_p D_0^p[u], alpha_nu = beta/sqrt(kappa dt),
 * so dt F = -(beta/c) sum_d (S_R[g_d^+] - S_L[g_d^-]) - beta^2 sum_d S_0[u];
 * 3-stage SSP Runge-Kutta (MOLT_INT_DEFAULT) or forward Euler.  Linear or
 * WENO-Z weights (WENO-Z: 5 points, MOLT_PREC_F64 or MOLT_PREC_F32).
 * Every problem may have non-uniform axes (molt_set_grid_axis): their
 * S_{P,d} are the point-local sums of molt_apply_D, the steps' formulas
 * unchanged; a Hamilton-Jacobi step with a non-uniform axis runs from the
 * one-sided sums of every axis and a pointwise stage kernel, with each
 * axis's spacing h_d its smallest cell (alpha = beta/(cfl min_d h_d), dt =
 * cfl min_d h_d / c_d).
 * Synchronous at the end (reads t and the device status). */
molt_status molt_step(molt_ctx* ctx, void* const* u, void* const* u_prev, int nsteps, double* t_inout);

/* Source term of a Hamilton-Jacobi problem, polynomial in time:
 *   F(x, t) = sum_{k=0}^{degree} t^k F_k(x),
 * as for a manufactured solution (Sec. 5.1, Example 3: u = t (sin x + sin y)
 * gives F = sin x + sin y + (1 + t cos x + t cos y)^2 / 2, degree 2).
 * coef: device array of degree+1 consecutive state-shaped arrays F_0 ..
 * F_degree (state element type, C order), copied into the context before
 * the call returns (the caller keeps ownership); coef == NULL removes the
 * source.  degree in 0..4.  MOLT_EINVAL: bad problem index, degree or
 * alignment, or a problem that is not Hamilton-Jacobi.  Synchronous. */
molt_status molt_set_source(molt_ctx* ctx, int problem, const void* coef, int degree);

/* Non-uniform axis: the n = desc.n[axis] nodes, host array, strictly
 * increasing; copied.  Periodic axis: the nodes of one period,
 * x[n-1] - x[0] < hi - lo (the period).  Dirichlet axis: every node of the
 * line, boundary nodes included, x[0] = a .. x[n-1] = b (n >= 4).
 * molt_apply_D along that axis then uses point-local quadrature weights
 * (each point's stencil nodes integrated against the exponential kernel,
 * the non-uniform case of Sec. 2.4) and cell decays e^{-alpha (x_i - x_{i-1})},
 * closed over the period with mu = e^{-alpha (hi - lo)} (Sec. 2.3), or on a
 * Dirichlet axis started at the ends, I_R(x_0) = I_L(x_{n-1}) = 0, with
 * ghost nodes mirrored about the ends holding the odd reflection of the
 * data, and the boundary constants that make L^{-1} take the boundary values
 * at a and b (mu = e^{-alpha (x_{n-1} - x_0)}; for L_0 the 2x2 system of
 * determinant 1 - mu^2).  With MOLT_W_WENOZ (5-point rule) the local
 * integrals are the WENO-Z combination of the substencil rules, with
 * point-local linear weights and smoothness indicators (see
 * molt_nonuniform_weno_weights); MOLT_W_LEARNED is MOLT_EUNSUPPORTED on
 * non-uniform axes.  molt_step runs every problem on such axes (see there).
 * x == NULL makes the axis uniform again.  The first call on a problem
 * allocates one state-sized array of the compute type (the axis sums of
 * molt_step), and for a Hamilton-Jacobi problem two state-sized arrays per
 * axis (its one-sided sums).  MOLT_EINVAL: bad index, count or nodes;
 * MOLT_ENOMEM.  Synchronous. */
molt_status molt_set_grid_axis(molt_ctx* ctx, int problem, int axis, const double* x, int64_t n);

/* The point tables of a non-uniform line (host only, no device work): for
 * nodes x[n] of one period of length `period` (> 0), or of a Dirichlet line
 * (period == 0: x[0] = a .. x[n-1] = b are both boundary nodes, n >= 4, and
 * the stencils reach ghost nodes mirrored about the ends, Sec. 2.3), alpha
 * and the rule: cR[6 n] and cL[6 n] (slot m of point i at m * n + i belongs
 * to offset m - 3: J_R(x_i) = sum_m cR v_{i+m-3}, J_L(x_i) = sum_m cL
 * v_{i-(m-3)}; unused slots 0) and q[n] (q_i = e^{-alpha (x_i - x_{i-1})}),
 * as the non-uniform sweeps use them.  On a Dirichlet line the recurrences
 * start at the ends: J_R(x_0) = J_L(x_{n-1}) = 0 and q_0 = 0.  MOLT_EINVAL on
 * bad arguments (nodes not strictly increasing or not finite, a periodic line
 * wider than its period). */
molt_status molt_nonuniform_weights(const double* x, int64_t n, double period, double alpha, int quad_points,
                                    double* cR, double* cL, double* q);

/* The WENO-Z point tables of a non-uniform line for the 5-point rule (host
 * only, no device work; Sec. 2.4: on a non-uniform mesh the linear weights
 * d_r are local to each point); `period` as for molt_nonuniform_weights (a
 * Dirichlet line's end points, where the recurrences start, get zero rules
 * and d_r = 1/3).  wR[30 n] (J_R) and wL[30 n] (J_L),
 * slot s of point i at s * n + i, with substencil r = 0..2 on the offsets
 * {r-3, r-2, r-1} (nodes x_{i+o} for J_R, x_{i-o} for J_L):
 *   slots 3r+j     c^{(r)}_j, the rule of substencil r:
 *                  J^{(r)} = sum_j c^{(r)}_j v(node j);
 *   slots 9+r      d_r, with sum_r d_r c^{(r)} the 5-point rule of the point;
 *   slots 12+3r+j  A_{rj}, slots 21+3r+j B_{rj}: with a = sum_j A_{rj} v,
 *                  b = sum_j B_{rj} v the substencil interpolant has
 *                  dp/dt = a + b t in the cell variable t in [-1, 0]
 *                  (t = (s - x_i)/dx_i on [x_{i-1}, x_i] for J_R,
 *                  t = (x_i - s)/dx_i on [x_i, x_{i+1}] for J_L), so its
 *                  smoothness indicator, the sum over l = 1, 2 of
 *                  dx_i^{2l-1} int_cell (d^l p/ds^l)^2 ds, is a^2 - a b + 4/3 b^2.
 * WENO-Z: w~_r = d_r (1 + tau/(1e-6 + beta_r)), tau = |beta_0 - beta_2|,
 * J = sum_r w~_r J^{(r)} / sum_r w~_r.  MOLT_EINVAL on bad arguments. */
molt_status molt_nonuniform_weno_weights(const double* x, int64_t n, double period, double alpha, double* wR,
                                         double* wL);

/* Tile plan of a sweep (host only, no device work): the tile shape that
 * molt_apply_D(op, P, alpha) along `axis` of a problem described by `d`
 * launches with the plain sweep kernel -- points per lane E, warps per line
 * (32 E warps_per_line >= n), lines per CTA (a power of two), threads per CTA
 * (<= 512), CTAs (ceil(lines / lines_per_cta)), dynamic shared memory per
 * CTA, and whether the line fills its lanes exactly (no masked points).
 * Where the array geometry meets the tensor-copy alignment rules the
 * persistent TMA kernel runs the same tiles with one CTA per SM.  The SM
 * count that sizes grids with few lines is the current device's (152 when
 * no device is present).  MOLT_EINVAL: an invalid descriptor or argument;
 * MOLT_EUNSUPPORTED: a line or tile the sweeps do not take, learned weights.
 * The reason is in molt_last_error(NULL). */
typedef struct {
  int32_t points_per_lane;
  int32_t warps_per_line;
  int32_t lines_per_cta;
  int32_t threads_per_cta;
  int64_t ctas;
  int64_t smem_bytes;
  int32_t exact_fit;
  int32_t reserved;
} molt_sweep_plan;

molt_status molt_plan_sweep(const molt_desc* d, int axis, int op, int P, double alpha, molt_sweep_plan* out);

/* Context options.
 *   MOLT_OPT_TMA      1 (default): sweeps whose lines are an exact fit and
 *                     whose arrays meet the tensor-copy alignment rules run
 *                     the persistent TMA-fed kernel; 0: always the plain
 *                     one-tile-per-CTA kernel.  Both compute the same values.
 *   MOLT_OPT_PROFILE  1: record a CUDA event pair around every sweep launch
 *                     (read back with molt_profile_read); 0 (default): off.
 * Returns MOLT_EINVAL for an unknown option or value. */
typedef enum {
  MOLT_OPT_TMA = 0,
  MOLT_OPT_PROFILE = 1,
  MOLT_OPT_WAIT_LIMIT = 2,        /* cycles a device-side wait may take before the
                                     kernel records MOLT_ETIMEOUT and returns
                                     (default 2e9, >= 1000)                      */
  MOLT_OPT_TEST_SKIP_ARRIVE = 3,  /* test hook: 1 makes one CTA of the batched step
                                     skip its first grid barrier, so the others'
                                     bounded waits run out (MOLT_ETIMEOUT)       */
  MOLT_OPT_LANES = 4,             /* line-per-lane FP32 sweeps (one lane per line,
                                     one warp per 16-point segment, difference
                                     form of the recurrences): 1 (default) when
                                     the line shape allows and nu*16 >= ~3.5;
                                     2 whenever the shape allows; 0 never.
                                     Both kernels compute the same values      */
  MOLT_OPT_AXIS_STREAMS = 5,      /* heat problems of up to 2^18 points in 2-D
                                     or 3-D: 1 (default) runs the x sweep of a
                                     stage on the context's stream and the y
                                     (and z) sweeps on a second stream at the
                                     same time, then one update kernel; 0 runs
                                     the axes one after another.  Same values */
  MOLT_OPT_XLINES = 6             /* x lines of the FP32 sweeps that
                                     MOLT_OPT_LANES admits: 1 (default) one
                                     warp per line group (lanes = 16-point
                                     segments, carries by warp shuffles), for
                                     any number of lines; 0 the line-per-lane
                                     tiles.  Same values up to FP32 rounding
                                     (the carries are summed in another order) */
} molt_option;
molt_status molt_set_option(molt_ctx* ctx, int option, int64_t value);

/* Kinds of sweep launches, by the work their epilogue does. */
typedef enum {
  MOLT_KERNEL_STORE = 0,       /* molt_apply_D                                */
  MOLT_KERNEL_ACC_SET = 1,     /* first axis of a step: acc = S               */
  MOLT_KERNEL_ACC_ADD = 2,     /* middle axis: acc += S                       */
  MOLT_KERNEL_HEAT_FINAL = 3,  /* last axis + Runge-Kutta stage update        */
  MOLT_KERNEL_WAVE_FINAL = 4,  /* last axis + leapfrog update                 */
  MOLT_KERNEL_HJ_X = 5,        /* Hamilton-Jacobi: first axes                 */
  MOLT_KERNEL_HJ_Y = 6,        /* Hamilton-Jacobi: last axis + update         */
  MOLT_KERNEL_UPDATE = 7,      /* FP64 state update of the FP32-sweep forms   */
  MOLT_KERNEL_BATCH = 8,       /* one persistent batched heat step            */
  MOLT_KERNEL_TRANSPOSE = 9,   /* state transposes of the 2-D Hamilton-Jacobi
                                  y pass on long lines                        */
  MOLT_KERNEL_FLUX = 10,       /* advection-diffusion: split fluxes g^+, g^-  */
  MOLT_KERNEL_LANES_STORE = 11,   /* line-per-lane sweeps (MOLT_OPT_LANES):      */
  MOLT_KERNEL_LANES_ACC_SET = 12, /*   STORE, ACC_SET, and ACC_ADD / the        */
  MOLT_KERNEL_LANES_ACC_ADD = 13, /*   advection-diffusion accumulations,       */
  MOLT_KERNEL_LANES_WAVE_FINAL = 14, /* and the last axis of the mixed-precision
                                     wave step with the FP64 leapfrog update  */
  MOLT_KERNEL_XLINES_STORE = 15,   /* warp-per-line x sweeps (MOLT_OPT_XLINES): */
  MOLT_KERNEL_XLINES_ACC_SET = 16, /*   STORE, ACC_SET, and ACC_ADD / the       */
  MOLT_KERNEL_XLINES_ACC_ADD = 17  /*   advection-diffusion accumulations       */
} molt_kernel_kind;

/* With MOLT_OPT_PROFILE on: synchronises the stream, returns the summed
 * device time (ms) and count of the recorded launches of `kind`, and clears
 * those records (setting MOLT_OPT_PROFILE, to either value, clears all
 * records).  Either output pointer may be NULL. */
molt_status molt_profile_read(molt_ctx* ctx, int kind, double* total_ms, int64_t* launches);

/* One wave time step that allocates no device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- code under a fixed device-memory budget, code inside a
 * framework whose caching allocator owns all of the device's memory, and
 * latency-critical code that cannot afford a first-use allocation.
 *   desc      one problem with pde = MOLT_PDE_WAVE, prec =
 *             MOLT_PREC_F32_F64UPDATE, linear weights, every used axis
 *             2..8192 points, at most 1,048,576 grid points in total;
 *             larger grids return MOLT_EINVAL, other PDEs/precisions
 *             MOLT_EUNSUPPORTED.
 *   u, u_prev u^n and u^{n-1}: device arrays of doubles (u_prev unused and
 *             may be NULL when from_rest != 0).
 *   u_next    receives u^{n+1} = 2u^n - u^{n-1} - beta^2 sum_d S_{P,d}[u^n]
 *             (from_rest: u^n - beta^2/2 sum_d S_{P,d}[u^n]).  It may be
 *             u_prev (the usual leapfrog rotation: each point of u^{n-1} is
 *             read by the thread that then writes that point), never u
 *             (MOLT_EINVAL).  All three 16-byte aligned.
 *   cuda_stream  cudaStream_t the work is enqueued on.
 * Scratch (the FP32 copy of u^n, the FP32 axis accumulator and a status
 * word, 8 MiB + 256 bytes) is a file-scope device array that every GPU
 * loading the library holds until the process exits.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with
 * the device current, and looks it up again whenever the current CUDA
 * context differs from the one it was looked up in (after cudaDeviceReset
 * the module loads again and the array may move); make the first call on a
 * device, and the first after a context reset, before any stream capture.
 * Every call on a device shares the array and clears the status word, so
 * calls that overlap on the GPU (other streams, other host threads) race.
 * Synchronous: returns after the step finished (MOLT_ENONFINITE if a
 * non-finite value reached u_next).  Allocates nothing, host or device. */
molt_status molt_wave_step_noalloc(const molt_desc* desc, const double* u, const double* u_prev, double* u_next,
                                   int from_rest, void* cuda_stream);

/* Batched step (count > 1; every problem 2-D heat, MOLT_PREC_F32_F64UPDATE,
 * linear weights, sides that tile exactly -- multiples of 128 up to 8192 in
 * power-of-two warps per line): molt_step advances all problems with ONE
 * persistent cooperative kernel per time step, captured in a CUDA graph when
 * the stream is not the legacy default stream.  Its phases (x sweeps, y
 * sweeps, FP64 update; three Runge-Kutta stages) are separated by grid
 * barriers with bounded waits.  The first molt_step autotunes, per size class
 * and axis, the line-tile shape (points per lane 16, 8 or 4, hence warps per
 * line and lines per 512-thread tile) by timing each candidate.  This call
 * reports the shape chosen for (problem, axis); MOLT_EUNSUPPORTED before the
 * first batched step or for contexts that do not batch. */
molt_status molt_batch_tile_shape(molt_ctx* ctx, int problem, int axis, int* points_per_lane, int* warps_per_line,
                                  int* lines_per_tile);

/* ---------------------------------------------------------------------------
 * Learned WENO weights.  The paper has no learned component: its nonlinear
 * local integrals use WENO-Z weights (Sec. 2.4).  Problems with weights =
 * MOLT_W_LEARNED (quad_points 5, MOLT_PREC_F32) replace the weight formula by
 * a small network -- 5 stencil values -> 32 -> 32 -> 3, GELU (tanh form) after
 * both hidden layers, softmax output -- evaluated on the tensor cores in BF16
 * with FP32 accumulation inside the sweep.  Network inputs are the stencil
 * values in J_R orientation (v_{e-3} .. v_{e+1}; J_L uses the mirrored
 * stencil v_{e+3} .. v_{e-1}) minus the middle value, divided by their
 * largest magnitude plus 1e-30.  Wherever the network's weights differ from
 * the WENO-Z weights by more than 1e-2 in any component (or are not finite),
 * the WENO-Z weights are used (fallback).
 *
 * Network blob (MOLT_MLP_BLOB_BYTES bytes, BF16, row-major, zero padded):
 *   W1[32][16] (inputs 0..4 used), W2[32][32], W3[8][32] (outputs 0..2 used),
 *   b1[32], b2[32], b3[8] (0..2 used).
 * FP32 master parameters (MOLT_MLP_PARAMS floats, training entry points):
 *   W1 (32x5), b1 (32), W2 (32x32), b2 (32), W3 (3x32), b3 (3), row-major.
 * ------------------------------------------------------------------------- */
#define MOLT_MLP_PARAMS 1347
#define MOLT_MLP_BLOB_BYTES 3728

/* Install the network used by the context's learned-weight problems.  blob:
 * host or device memory (unified addressing), `bytes` must equal
 * MOLT_MLP_BLOB_BYTES.  Synchronous (the blob may be reused on return).
 * MOLT_EINVAL if no problem of the context uses learned weights.  Sweeps of
 * learned-weight problems fail with MOLT_EINVAL until this has been called. */
molt_status molt_set_mlp(molt_ctx* ctx, const void* blob, size_t bytes);

/* Counters of the context's learned-weight sweeps since creation or the last
 * reset: stencils evaluated by the network and stencils that fell back to
 * WENO-Z.  Synchronous; reset != 0 clears both.  Either pointer may be NULL. */
molt_status molt_mlp_stats(molt_ctx* ctx, int64_t* stencils, int64_t* fallbacks, int reset);

/* The training and evaluation entry points below take no context: every
 * pointer is a DEVICE pointer (16-byte aligned) unless stated, work is
 * enqueued on `cuda_stream` (a cudaStream_t, NULL = legacy stream) and the
 * calls return before it finishes.  n == 0 does nothing; n < 0 or a NULL
 * required pointer returns MOLT_EINVAL. */

/* WENO linear weights d_0, d_1, d_2 of the 5-point rule at nu = alpha*h
 * (App. C construction; d_0 from the ratio of first coefficients, d_2 from
 * the ratio of last ones, d_1 = 1 - d_0 - d_2).  d: host array of 3.
 * Synchronous, host only. */
molt_status molt_weno_linear_weights(double nu, double* d);

/* The quadrature weights the sweeps use (App. C construction, from
 * exponential moments: a power series for nu <= 1, the integration-by-parts
 * recurrence above), host only and synchronous.  quad_points 3, 5 or 6;
 * nu = alpha*h > 0.  c[6]: weights of J_R(x_i) = sum_l c_l v_{i+l} on the
 * offsets l = -3..2 (zero where the rule has no node).  sub[12] (may be NULL):
 * substencil weights [r][j] for r = 0..2, node j of substencil r (5-point
 * rule: offsets -3+r..-1+r, j = 3 zero; 6-point: -3+r..r); d[3] (may be
 * NULL): the linear weights.  Both zero for the 3-point rule. */
molt_status molt_quadrature_weights(int quad_points, double nu, double* c, double* sub, double* d);

/* Round FP32 master parameters theta[MOLT_MLP_PARAMS] to the BF16 blob. */
molt_status molt_mlp_pack(const float* theta, void* blob, void* cuda_stream);

/* Network weights of n stencils.  x: n x 5 raw stencil values (J_R
 * orientation, not normalised; the call normalises).  w: n x 3 outputs.
 * d: NULL for the raw network outputs, or the host array of the 3 linear
 * weights -- then the WENO-Z fallback applies and, if `fallbacks` (device
 * unsigned 64-bit counter) is not NULL, the number of fallbacks is added. */
molt_status molt_mlp_forward(const void* blob, const float* x, int64_t n, const double* d, float* w,
                             unsigned long long* fallbacks, void* cuda_stream);

/* Mean-squared training loss L = (1/n) sum_i sum_r (p_ir - y_ir)^2 of the
 * network outputs p (as molt_mlp_forward with d = NULL) against targets y
 * (n x 3), and its gradient with respect to the FP32 master parameters
 * (through the BF16 forward pass; products of the backward pass in BF16 with
 * FP32 accumulation).  grad[MOLT_MLP_PARAMS] and *loss are overwritten. */
molt_status molt_mlp_loss_grad(const void* blob, const float* x, const float* y, int64_t n, float* grad, float* loss,
                               void* cuda_stream);

/* One Adam step (Kingma & Ba, 2015) on the FP32 master parameters with
 * moment buffers m, v (MOLT_MLP_PARAMS floats each, zero before step 1):
 * m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * theta -= lr (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps); then the
 * BF16 blob is rewritten from theta.  step >= 1. */
molt_status molt_mlp_adam(float* theta, float* m, float* v, const float* grad, int64_t step, double lr, double beta1,
                          double beta2, double eps, void* blob, void* cuda_stream);

/* Training stencils from a periodic 2-D FP32 state u (ny x nx, x fastest):
 * for each of `count` flat grid indices pos[i] (int64, 0 <= pos < nx*ny),
 * row i*stride of x (n x 5) receives the 5 values along `axis` (0: x, 1: y)
 * at offsets -3..1 (side 0, J_R) or +3..-1 (side 1, J_L), periodically
 * wrapped, and, if y is not NULL, row i*stride of y (n x 3) their WENO-Z
 * weights with linear weights d (host array of 3).  stride >= 1 interleaves
 * the stencils of several calls.  An index outside the grid yields a row of
 * NaNs. */
molt_status molt_mlp_harvest(const float* u, int64_t nx, int64_t ny, const int64_t* pos, int64_t count, int axis,
                             int side, const double* d, float* x, float* y, int64_t stride, void* cuda_stream);

/* Release everything the context owns.  Synchronises its stream first. */
molt_status molt_destroy(molt_ctx* ctx);

/* Text of the last error recorded on ctx ("" if none); valid until the next
 * call on ctx.  ctx may be NULL (then describes the last molt_create error). */
const char* molt_last_error(const molt_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* MOLT_H */
