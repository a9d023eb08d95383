// Host-side quadrature tables for the local integrals J_R / J_L (Sec. 2.4,
// App. C of arXiv 2007.03041).
//
// With nu = alpha*h and s = x_i + t*h, the weight of node x_{i+l} in
// J_R(x_i) = alpha int_{x_{i-1}}^{x_i} e^{-alpha(x_i-s)} p(s) ds is
//   c_l(nu) = nu int_{-1}^{0} e^{nu t} ell_l(t) dt = sum_m L[l][m] M_m(nu),
// where ell_l(t) = sum_m L[l][m] t^m is the Lagrange basis on the integer
// offsets and M_m(nu) = nu int_{-1}^{0} e^{nu t} t^m dt are exponential
// moments.  The moments come from their power series for small nu (no
// cancellation; the App. C closed forms lose digits like nu^-3) and from the
// integration-by-parts recurrence M_m = -(-1)^m e^{-nu} - (m/nu) M_{m-1}
// for larger nu, where it is stable.
#pragma once

namespace molt {

struct QuadTable {
  int npts;           // 3, 5 or 6
  double nu;          // alpha*h
  double c[6];        // J_R weights on offsets -3..2 (zero where unused)
  double sub[3][4];   // substencil weights (5-pt: offsets -3+r .. -1+r; 6-pt: -3+r .. r)
  double d[3];        // linear weights, sum_r d_r sub_r = big stencil
  double q;           // e^{-nu}
};

// Fills t for the given stencil size; returns false if npts is unsupported
// or the linear weights do not reproduce the large-stencil rule.
bool build_quadrature(int npts, double nu, QuadTable* t);

// nu * int_{-1}^{0} e^{nu t} t^m dt for m = 0..mmax (mmax <= 7).
void exp_moments(double nu, int mmax, double* M);

}  // namespace molt
