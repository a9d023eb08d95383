// Fast summation on non-uniform lines (the point-local quadrature that
// Sec. 2.4 describes for non-uniform meshes): per point i the J_R / J_L
// weights of its own stencil nodes and the cell decay q_i = e^{-alpha (x_i -
// x_{i-1})}; the recurrences I_R(x_i) = q_i I_R(x_{i-1}) + J_R(x_i),
// I_L(x_i) = q_{i+1} I_L(x_{i+1}) + J_L(x_i) close over the period with
// mu = prod q_i = e^{-alpha L} (Sec. 2.3), or on a Dirichlet line start at
// the ends with the boundary constants fixed by the boundary values.
//
// Host side: build_nonuniform_tables() integrates the Lagrange basis of each
// point's stencil against the exponential by 16-point Gauss-Legendre
// quadrature (FP64).  Device side: one CTA per line, the line staged in
// shared memory and its scan positions split between the CTA's warps; per D
// application and direction each warp computes its segment's local integrals
// once (chunks of 32 x 4 points: per-lane affine maps (q, J), a warp scan of
// their compositions), the segment maps and the periodic closure give every
// segment its start value, and the warp replays its chunks from there.
#pragma once

#include <cmath>
#include <vector>

#include "sweep.cuh"

namespace molt {

// Device tables of one (axis, alpha, rule): structure of arrays.  Linear
// weights: slot m belongs to offset m - 3 (offsets -3..2; unused slots are
// 0).  WENO-Z: cR, cL hold the kNuWeno-slot tables of
// build_nonuniform_weno_tables.
template <typename T>
struct NuTables {
  const T* cR;   // [6][n]: J_R(x_i) = sum_m cR[m][i] v_{i + m - 3}   (WENO-Z: [30][n])
  const T* cL;   // [6][n]: J_L(x_i) = sum_m cL[m][i] v_{i - (m - 3)} (WENO-Z: [30][n])
  const T* q;    // [n]: q_i = e^{-alpha (x_i - x_{i-1})}
};

struct NuArgs {
  LineGeom g;
  int mode, P;
  int bc;               // 0 periodic, 1 Dirichlet (nodes x_0 = a .. x_{n-1} = b)
  double inv1mmu;       // periodic: 1/(1 - mu), mu = e^{-alpha L}
  double mu, kdir;      // Dirichlet: mu = e^{-alpha (b - a)}, kdir = 2/(1 - mu^2)
  const void* in;
  void* out;
  int* status;
};

// Roots and weights of the n-point Gauss-Legendre rule on [-1, 1] (Newton on
// the three-term recurrence of the Legendre polynomials).
inline void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      const double dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) {
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        break;
      }
      x[i] = z;
      w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
  }
}

// x_j for any j: periodic images (L > 0, x the nodes of one period), or for a
// Dirichlet line (L == 0, nodes x_0 = a .. x_{n-1} = b, n >= 4) the ghost
// nodes mirrored about the ends, x_{-j} = 2a - x_j, x_{N+j} = 2b - x_{N-j}
// (Sec. 2.3: the stencils reach odd-reflected data there).
inline double nu_node(const std::vector<double>& x, double L, long long j) {
  const long long n = static_cast<long long>(x.size());
  if (L > 0) {
    long long r = j % n;
    if (r < 0) r += n;
    return x[size_t(r)] + double((j - r) / n) * L;
  }
  const long long N = n - 1;
  if (j < 0) return 2.0 * x[0] - x[size_t(-j)];
  if (j > N) return 2.0 * x[size_t(N)] - x[size_t(2 * N - j)];
  return x[size_t(j)];
}

// cR, cL: 6*n (slot-major), q: n.  x: the n nodes of one period [x_0, x_0 + L),
// or (L == 0) of a Dirichlet line.  Dirichlet lines start their recurrences
// at the ends, I_R(x_0) = 0 and I_L(x_N) = 0: J_R(x_0) and J_L(x_N) are zero
// and q_0 = 0, so a scan over the whole line gives exactly those values.
inline void build_nonuniform_tables(const std::vector<double>& x, double L, double alpha, int npts,
                                    std::vector<double>* cR, std::vector<double>* cL, std::vector<double>* q) {
  const int n = int(x.size());
  int lo = -3, hi = 2;                 // J_R stencil offsets (6 points)
  if (npts == 5) hi = 1;
  if (npts == 3) { lo = -1; hi = 1; }
  const int k = hi - lo + 1;
  cR->assign(6 * size_t(n), 0.0);
  cL->assign(6 * size_t(n), 0.0);
  q->assign(n, 0.0);
  constexpr int kG = 16;
  double gx[kG], gw[kG];
  gauss_legendre(kG, gx, gw);
  auto node = [&](long long j) { return nu_node(x, L, j); };
  for (int i = 0; i < n; ++i) {
    const double xi = x[size_t(i)];
    for (int side = 0; side < 2; ++side) {
      // J_R: cell [x_{i-1}, x_i], nodes x_{i+l}; J_L: cell [x_i, x_{i+1}], nodes x_{i-l}
      const double a = side == 0 ? node(i - 1) : xi, b = side == 0 ? xi : node(i + 1);
      double t[6];
      for (int m = 0; m < k; ++m) t[m] = node(side == 0 ? i + lo + m : i - (lo + m)) - xi;
      for (int m = 0; m < k; ++m) {
        double sum = 0.0;
        for (int gq = 0; gq < kG; ++gq) {
          const double s = 0.5 * (b - a) * gx[gq] + 0.5 * (b + a);
          double ell = 1.0;
          for (int r = 0; r < k; ++r)
            if (r != m) ell *= ((s - xi) - t[r]) / (t[m] - t[r]);
          const double kern = side == 0 ? std::exp(-alpha * (xi - s)) : std::exp(-alpha * (s - xi));
          sum += 0.5 * (b - a) * gw[gq] * alpha * kern * ell;
        }
        (side == 0 ? *cR : *cL)[size_t(lo + m + 3) * n + i] = sum;
      }
    }
    (*q)[size_t(i)] = std::exp(-alpha * (xi - node(i - 1)));
  }
  if (!(L > 0)) {
    for (int m = 0; m < 6; ++m) {
      (*cR)[size_t(m) * n] = 0.0;
      (*cL)[size_t(m) * n + n - 1] = 0.0;
    }
    (*q)[0] = 0.0;
  }
}

// WENO-Z tables of the 5-point rule (quadratic substencils S_r = offsets
// {r-3, r-2, r-1}, Sec. 2.4), per point and direction, slot-major [kNuWeno][n]
// (periodic lines, or Dirichlet lines with L == 0 as above):
//   slots 3r+j       c^{(r)}_j: J^{(r)} = sum_j c^{(r)}_j v(node j of S_r)
//   slots 9+r        d_r, the linear weights with sum_r d_r c^{(r)} = c
//   slots 12+3r+j    A_{rj} = l_j'(0), slots 21+3r+j  B_{rj} = l_j''
// in the cell variable t in [-1, 0] (t = (s - x_i)/dx for J_R on
// [x_{i-1}, x_i], t = (x_i - s)/dx for J_L on [x_i, x_{i+1}]), l_j the
// Lagrange basis of S_r.  With a = sum A v and b = sum B v the interpolant has
// p_t = a + b t, so its smoothness indicator int_{-1}^0 p_t^2 + p_tt^2 dt is
// a^2 - a b + 4/3 b^2.  The node of slot j of S_r is x_{i + (r + j - 3)} for
// J_R and x_{i - (r + j - 3)} for J_L.  Since every rule integrates the
// constant exactly (weights summing to 1 - q), d_1 = 1 - d_0 - d_2 once the
// two outer nodes, each in one substencil only, fix d_0 and d_2.
constexpr int kNuWeno = 30;

inline void build_nonuniform_weno_tables(const std::vector<double>& x, double L, double alpha,
                                         std::vector<double>* wR, std::vector<double>* wL) {
  const int n = int(x.size());
  wR->assign(size_t(kNuWeno) * n, 0.0);
  wL->assign(size_t(kNuWeno) * n, 0.0);
  constexpr int kG = 16;
  double gx[kG], gw[kG];
  gauss_legendre(kG, gx, gw);
  auto node = [&](long long j) { return nu_node(x, L, j); };
  // nu int_{-1}^0 e^{nu t} l_m(t) dt for the Lagrange basis on nodes t[0..k)
  auto rule = [&](const double* t, int k, int m, double nu) {
    double sum = 0.0;
    for (int g = 0; g < kG; ++g) {
      const double tt = 0.5 * (gx[g] - 1.0);
      double ell = 1.0;
      for (int r = 0; r < k; ++r)
        if (r != m) ell *= (tt - t[r]) / (t[m] - t[r]);
      sum += 0.5 * gw[g] * nu * std::exp(nu * tt) * ell;
    }
    return sum;
  };
  for (int i = 0; i < n; ++i) {
    const double xi = x[size_t(i)];
    for (int side = 0; side < 2; ++side) {
      const double dx = side == 0 ? xi - node(i - 1) : node(i + 1) - xi;
      const double nu = alpha * dx;
      double t5[5];
      for (int k = 0; k < 5; ++k) {
        const int off = k - 3;
        t5[k] = side == 0 ? (node(i + off) - xi) / dx : (xi - node(i - off)) / dx;
      }
      std::vector<double>& w = side == 0 ? *wR : *wL;
      auto at = [&](int slot) -> double& { return w[size_t(slot) * n + i]; };
      for (int r = 0; r < 3; ++r) {
        const double* t = t5 + r;
        for (int j = 0; j < 3; ++j) {
          const double ta = t[(j + 1) % 3], tb = t[(j + 2) % 3];
          const double den = (t[j] - ta) * (t[j] - tb);
          at(3 * r + j) = rule(t, 3, j, nu);
          at(12 + 3 * r + j) = -(ta + tb) / den;
          at(21 + 3 * r + j) = 2.0 / den;
        }
      }
      const double d0 = rule(t5, 5, 0, nu) / at(0);
      const double d2 = rule(t5, 5, 4, nu) / at(8);
      at(9) = d0;
      at(10) = 1.0 - d0 - d2;
      at(11) = d2;
    }
  }
  if (!(L > 0)) {
    // Dirichlet ends: J_R(x_0) = J_L(x_N) = 0 (zero rules, equal weights)
    for (int side = 0; side < 2; ++side) {
      std::vector<double>& w = side == 0 ? *wR : *wL;
      const size_t i = side == 0 ? 0 : size_t(n - 1);
      for (int slot = 0; slot < kNuWeno; ++slot) w[size_t(slot) * n + i] = 0.0;
      for (int r = 0; r < 3; ++r) w[size_t(9 + r) * n + i] = 1.0 / 3.0;
    }
  }
}

// WENO-Z local integral of point i from its point tables tw ([30][n], layout
// of build_nonuniform_weno_tables), in difference form: returns
// (1 - q) v_i - J(x_i) = sum_r w_r sum_j c^{(r)}_j (v_i - v_j), exact since
// every substencil rule integrates the constant to 1 - q and the normalised
// weights sum to one.  The five stencil values are taken in the orientation
// of the direction (J_L reads the mirrored nodes); per substencil r its
// rule, a = p_t(0) and b = p_tt, beta_r = a^2 - a b + 4/3 b^2, and the
// WENO-Z map w~_r = d_r (1 + tau/(eps + beta_r)), tau = |beta_0 - beta_2|,
// eps = 1e-6 (Sec. 2.4).
template <typename T, bool LEFT>
__device__ __forceinline__ T nu_wenoz_defect(const T* tw, const T* v, int n, int i) {
  T w[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) w[k] = LEFT ? v[3 + i - (k - 3)] : v[3 + i + (k - 3)];
  T Jr[3], beta[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    T J = T(0), a = T(0), b = T(0);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      // differences from the centre: the derivative rows sum to zero, so a
      // and b change sign only (beta is even in (a, b)), and the centre's
      // term drops
      if (r + j == 3) continue;
      const T dj = w[3] - w[r + j];
      J = fma(tw[(3 * r + j) * n + i], dj, J);
      a = fma(tw[(12 + 3 * r + j) * n + i], dj, a);
      b = fma(tw[(21 + 3 * r + j) * n + i], dj, b);
    }
    Jr[r] = J;
    beta[r] = fma(a, a - b, T(4.0 / 3.0) * b * b);
  }
  const T tau = fabs(beta[0] - beta[2]);
  const T eps = T(1e-6);
  T num = T(0), sum = T(0);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const T d = tw[(9 + r) * n + i];
    const T wt = fma(d * tau, weight_rcp(eps + beta[r]), d);
    num = fma(wt, Jr[r], num);
    sum += wt;
  }
  return num * weight_rcp(sum);
}

// One direction, split over the `nw` warps of the line (segment `seg` <= 512
// scan positions each, R ascending, L descending), in difference form: the
// scan carries W = v - I, which obeys the recurrence of I with the forcing
// K_i = v_i - q_i v_{i-1} - J_R(x_i) = sum_l c_{i,l} (v_i - v_{i+l}) +
// q_i (v_i - v_{i-1}) (mirrored for L; the rules integrate constants to
// 1 - q_i), so W of constant data is exactly zero and on smooth data its
// rounding error scales with the differences, not with v.  Each warp
// computes K and the decays of its segment once (chunks of 32 x 4 points,
// kept in registers), the per-lane affine maps x -> q x + K composed by a
// warp scan per chunk; the segments' maps meet in shared memory
// (maps[2 * nw]) and give the line's end value from W = 0, `all`.  The value
// entering the line is then k1 * all + start0: the periodic closure (k1 =
// 1/(1 - mu), start0 = 0) or a Dirichlet line's boundary value of W (the
// recurrence starts at the end node, whose decay is taken as 1 so that the
// scan passes the start value on unchanged; K there is zero).  Each warp
// replays its chunks from its start value and stores by OUT: 0 nothing (the
// total only), 1 W in w (D_R or D_L, or W_R of L_0), 3 D_0 = (w + W)/2 in w
// (w holding W_R: the L pass of L_0).  Returns `all`.
template <typename T, bool LEFT, int OUT, bool WENO>
__device__ __forceinline__ T nu_direction(const NuTables<T>& tb, const T* v, T* w, int n, int nw, int part, int seg,
                                          double k1, double start0, bool dirichlet, T* maps, int lane) {
  constexpr int kPer = 4, kChunks = 4;          // seg <= kChunks * 32 * kPer
  const int s0 = min(n, part * seg), s1 = min(n, s0 + seg);
  T jk[kChunks][kPer], qk[kChunks][kPer];
  T Ae[kChunks], Be[kChunks], At[kChunks], Bt[kChunks];
  T sA = T(1), sB = T(0);                        // the segment's map
#pragma unroll
  for (int c = 0; c < kChunks; ++c) {
    const int c0 = s0 + c * 32 * kPer;
    T A = T(1), B = T(0);
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int step = c0 + lane * kPer + k;
      qk[c][k] = T(1);
      jk[c][k] = T(0);
      if (step < s1) {
        const int i = LEFT ? n - 1 - step : step;
        const T vc = v[3 + i];
        T K = T(0);
        if constexpr (WENO) {
          K = nu_wenoz_defect<T, LEFT>(LEFT ? tb.cL : tb.cR, v, n, i);
        } else {
#pragma unroll
          for (int m = 0; m < 6; ++m) {
            const int off = m - 3;
            if (off == 0) continue;          // the centre's difference is 0
            if (LEFT) K = fma(tb.cL[m * n + i], vc - v[3 + i - off], K);
            else K = fma(tb.cR[m * n + i], vc - v[3 + i + off], K);
          }
        }
        const T qi = LEFT ? tb.q[i + 1 < n ? i + 1 : 0] : tb.q[i];
        K = fma(qi, vc - v[3 + i + (LEFT ? 1 : -1)], K);
        qk[c][k] = (dirichlet && step == 0) ? T(1) : qi;
        jk[c][k] = K;
        B = fma(qk[c][k], B, K);
        A *= qk[c][k];
      }
    }
    // inclusive scan of the lane maps (later lanes apply after)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T Ap = __shfl_up_sync(0xffffffffu, A, o), Bp = __shfl_up_sync(0xffffffffu, B, o);
      if (lane >= o) {
        B = fma(A, Bp, B);
        A *= Ap;
      }
    }
    Ae[c] = __shfl_up_sync(0xffffffffu, A, 1);
    Be[c] = __shfl_up_sync(0xffffffffu, B, 1);
    if (lane == 0) {
      Ae[c] = T(1);
      Be[c] = T(0);
    }
    At[c] = __shfl_sync(0xffffffffu, A, 31);
    Bt[c] = __shfl_sync(0xffffffffu, B, 31);
    sB = fma(At[c], sB, Bt[c]);
    sA *= At[c];
  }
  if (lane == 0) {
    maps[2 * part] = sA;
    maps[2 * part + 1] = sB;
  }
  __syncthreads();
  // value before this segment from W = 0 before the line, and the line's end value
  T pre = T(0), all = T(0), gA = T(1);
  for (int j = 0; j < nw; ++j) {
    if (j == part) pre = all;
    if (j < part) gA *= maps[2 * j];
    all = fma(maps[2 * j], all, maps[2 * j + 1]);
  }
  if constexpr (OUT == 0) {
    __syncthreads();   // maps[] is reused by the next pass
    return all;
  }
  // the start value carried through the earlier segments
  // (the boundary algebra in FP64: 1/(1 - mu) and 2/(1 - mu^2) grow large as
  // alpha times the line length shrinks)
  T carry = fma(gA, T(fma(double(all), k1, start0)), pre);
#pragma unroll
  for (int c = 0; c < kChunks; ++c) {
    const int c0 = s0 + c * 32 * kPer;
    T y = fma(Ae[c], carry, Be[c]);
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int step = c0 + lane * kPer + k;
      if (step < s1) {
        y = fma(qk[c][k], y, jk[c][k]);
        const int i = LEFT ? n - 1 - step : step;
        if constexpr (OUT == 1) w[i] = y;
        if constexpr (OUT == 3) w[i] = T(0.5) * (w[i] + y);
      }
    }
    carry = fma(At[c], carry, Bt[c]);
  }
  __syncthreads();
  return all;
}

// S_P along non-uniform lines, periodic or Dirichlet: one CTA of `nw` warps per line (the
// scan positions split into nw segments of at most 512); shared memory: v
// (n + 6) and w (n) of T plus the segment maps.  WENO: local integrals by
// WENO-Z with the point-local tables, else the linear point weights.
template <typename T, typename TIO, bool WENO>
// FP32 lines take at most 64 registers (two 512-thread or four 256-thread
// CTAs per SM: the scans' shuffle chains wait on latency, so more resident
// warps keep the SM issuing; 4096^2: 1.14 -> 0.94 ms per S_2 step with the
// linear rule, 2.39 -> 2.20 with WENO-Z); FP64 keeps 128 (it would spill).
#ifndef MOLT_NU_MIN_BLOCKS_F32
#define MOLT_NU_MIN_BLOCKS_F32 2
#endif
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? MOLT_NU_MIN_BLOCKS_F32 : 1)
    nonuniform_kernel(const NuArgs a, const NuTables<T> tb) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int n = a.g.n;
  const int nw = blockDim.x >> 5, part = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long line = blockIdx.x;
  T* v = reinterpret_cast<T*>(smem_raw);
  T* w = v + n + 6;
  T* maps = w + n;
  const int seg = ((n + nw - 1) / nw + 127) / 128 * 128;
  const long long base = line_base(a.g, line);
  const long long st = a.g.stride;
  const TIO* in = static_cast<const TIO*>(a.in);
  TIO* out = static_cast<TIO*>(a.out);
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[3 + i] = T(in[base + i * st]);
  __syncthreads();
  const bool dir = a.bc == 1;
  const double k1 = dir ? 0.0 : a.inv1mmu;
  for (int p = 0; p < a.P; ++p) {
    if (threadIdx.x < 3) {
      const int j = threadIdx.x + 1;
      if (dir) {
        // odd reflection about the end values (mirrored ghost nodes, Sec. 2.3)
        v[3 - j] = T(2) * v[3] - v[3 + j];
        v[3 + n - 1 + j] = T(2) * v[3 + n - 1] - v[3 + n - 1 - j];
      } else {
        v[3 - j] = v[3 + ((n - j) % n + n) % n];
        v[3 + n - 1 + j] = v[3 + (j - 1) % n];
      }
    }
    __syncthreads();
    // D into w: R alone, L alone, or W_R first and then the L pass of L_0.
    // Dirichlet start values (Sec. 2.3, the 2x2 algebra of Sec. 3.3):
    // L_R^{-1}(a) = v(a) and L_L^{-1}(b) = v(b), so W starts from 0; for L_0
    // the passes start from 2A and 2B with [[1, mu], [mu, 1]] (A, B) =
    // (v(a) - I_0(a), v(b) - I_0(b)), which in terms of the W totals from
    // zero starts, W_R^0(b) and W_L^0(a), is W_R(a) = (kd/2) (mu W_R^0(b) -
    // W_L^0(a)) and W_L(b) = (kd/2) (mu W_L^0(a) - W_R^0(b)), kd =
    // 2/(1 - mu^2): the L total comes first
    if (a.mode == MODE_R) nu_direction<T, false, 1, WENO>(tb, v, w, n, nw, part, seg, k1, 0.0, dir, maps, lane);
    if (a.mode == MODE_L) nu_direction<T, true, 1, WENO>(tb, v, w, n, nw, part, seg, k1, 0.0, dir, maps, lane);
    if (a.mode == MODE_0) {
      if (!dir) {
        nu_direction<T, false, 1, WENO>(tb, v, w, n, nw, part, seg, k1, 0.0, false, maps, lane);
        nu_direction<T, true, 3, WENO>(tb, v, w, n, nw, part, seg, k1, 0.0, false, maps, lane);
      } else {
        const double hk = 0.5 * a.kdir, km = hk * a.mu;
        const double WL =
            double(nu_direction<T, true, 0, WENO>(tb, v, w, n, nw, part, seg, 0.0, 0.0, true, maps, lane));
        const double WR =
            double(nu_direction<T, false, 1, WENO>(tb, v, w, n, nw, part, seg, km, -hk * WL, true, maps, lane));
        nu_direction<T, true, 3, WENO>(tb, v, w, n, nw, part, seg, km, -hk * WR, true, maps, lane);
      }
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const T d = w[i];
      TIO* o = out + base + i * st;
      *o = p == 0 ? TIO(d) : TIO(T(*o) + d);
      v[3 + i] = d;
    }
    __syncthreads();
  }
}

}  // namespace molt
