// Host-side constants of one sweep: the quadrature weights and decay factors
// a kernel reads, from the FP64 table of csrc/coeffs.cpp (Sec. 2.3-2.4).
#pragma once

#include <cmath>

#include "coeffs.h"
#include "sweep.cuh"

namespace molt {

// Fills the weight and decay fields of `a` for lines of N intervals and E
// points per lane.  FP64 sweeps take the table as it is.  FP32 sweeps run
// their recurrences with q rounded to FP32 (q32); every constant they meet is
// made consistent with that ratio:
//   * the FP64 boundary constants use powers of q32 (mu = q32^N, ...), so the
//     periodic image sum and the Dirichlet solve close the recurrences the
//     kernel actually ran;
//   * each rule's FP32 weights are rescaled to sum to 1 - q32 (the moment
//     identity sum_l c_l = 1 - e^{-nu}, App. C), the last rounding residual
//     moved onto the largest weight, so that D[const] = 0 holds in the FP32
//     arithmetic.  Without this, the relative rounding of 1 - q32 (about
//     1e-6 at nu = 0.03) shifts the symbol of D by that amount at every
//     frequency, a systematic damping that a long run accumulates;
//   * alpha in FP32 (one-sided derivatives alpha D) is alpha * nu32 / nu.
#ifndef MOLT_FIT_F32_WEIGHTS
#define MOLT_FIT_F32_WEIGHTS 1
#endif
inline void set_line_constants(SweepArgs& a, const QuadTable& qt, int N, int E, bool f32_sweeps) {
  const bool f32 = f32_sweeps && MOLT_FIT_F32_WEIGHTS;
  for (int i = 0; i < 6; ++i) a.c[i] = qt.c[i];
  for (int r = 0; r < 3; ++r) {
    for (int j = 0; j < 4; ++j) a.sub[r][j] = qt.sub[r][j];
    a.d[r] = qt.d[r];
  }
  double q = qt.q, lq = -qt.nu;   // lq = log q
  if (f32) {
    q = double(float(qt.q));
    lq = std::log(q);
  }
  a.q = q;
  a.qE = std::exp(lq * double(E));
  a.invq = std::exp(-lq);
  a.mu = std::exp(lq * double(N));
  a.inv1mmu = 1.0 / (-std::expm1(lq * double(N)));
  a.invdet = 1.0 / (-std::expm1(2.0 * lq * double(N)));
  a.k2det = 2.0 * a.invdet;
  a.k2detq = a.k2det * a.invq;
  a.qf = float(q);
  a.qEf = float(a.qE);
  a.alphaf = float(f32 ? a.alpha * (-lq) / qt.nu : a.alpha);
  // FP32 weights summing to 1 - q32 (exact in FP64: q32 is a float)
  const double target = 1.0 - q;
  auto fit = [target](const double* c, int n, float* out) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += c[i];
    int imax = 0;
    for (int i = 0; i < n; ++i) {
      out[i] = float(s != 0.0 ? c[i] * (target / s) : c[i]);
      if (std::fabs(c[i]) > std::fabs(c[imax])) imax = i;
    }
    double got = 0.0;
    for (int i = 0; i < n; ++i) got += double(out[i]);
    out[imax] = float(double(out[imax]) + (target - got));
  };
  if (f32) {
    fit(qt.c, 6, a.cf);
    // the FP32 kernels read three substencil taps (the 5-point rule's)
    for (int r = 0; r < 3; ++r) {
      if (qt.npts == 5) {
        fit(qt.sub[r], 3, a.subf[r]);
      } else {
        for (int j = 0; j < 3; ++j) a.subf[r][j] = float(qt.sub[r][j]);
      }
    }
  } else {
    for (int i = 0; i < 6; ++i) a.cf[i] = float(qt.c[i]);
    for (int r = 0; r < 3; ++r)
      for (int j = 0; j < 3; ++j) a.subf[r][j] = float(qt.sub[r][j]);
  }
  for (int r = 0; r < 3; ++r) a.df[r] = float(qt.d[r]);
}

}  // namespace molt
