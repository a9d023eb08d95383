// Quadrature tables for the local integrals (Sec. 2.4, App. C).  See coeffs.h.
#include "coeffs.h"

#include <cmath>
#include <cstring>

namespace molt {

void exp_moments(double nu, int mmax, double* M) {
  if (nu <= 1.0) {
    // M_m = nu * sum_k nu^k/k! * (-1)^(m+k) / (m+k+1): terms fall like nu^k/k!
    for (int m = 0; m <= mmax; ++m) {
      double term = 1.0, sum = 0.0;
      for (int k = 0; k < 60; ++k) {
        const double sgn = ((m + k) & 1) ? -1.0 : 1.0;
        sum += sgn * term / double(m + k + 1);
        term *= nu / double(k + 1);
        if (term < 1e-40) break;
      }
      M[m] = nu * sum;
    }
  } else {
    const double e = std::exp(-nu);
    M[0] = 1.0 - e;
    for (int m = 1; m <= mmax; ++m) {
      const double sgn = (m & 1) ? -1.0 : 1.0;
      M[m] = -sgn * e - (double(m) / nu) * M[m - 1];
    }
  }
}

// Monomial coefficients of the Lagrange basis polynomial for node j of the
// integer node set `nodes` (size n <= 6).
static void lagrange_monomials(const int* nodes, int n, int j, double* coef) {
  double p[8] = {1.0};
  int deg = 0;
  double denom = 1.0;
  for (int m = 0; m < n; ++m) {
    if (m == j) continue;
    // p *= (t - nodes[m])
    double np_[8] = {0};
    for (int k = 0; k <= deg; ++k) {
      np_[k + 1] += p[k];
      np_[k] -= double(nodes[m]) * p[k];
    }
    ++deg;
    std::memcpy(p, np_, sizeof(p));
    denom *= double(nodes[j] - nodes[m]);
  }
  for (int k = 0; k < n; ++k) coef[k] = p[k] / denom;
}

static void weights_on(const int* nodes, int n, const double* M, double* out) {
  for (int j = 0; j < n; ++j) {
    double coef[8];
    lagrange_monomials(nodes, n, j, coef);
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += coef[k] * M[k];
    out[j] = s;
  }
}

bool build_quadrature(int npts, double nu, QuadTable* t) {
  std::memset(t, 0, sizeof(*t));
  t->npts = npts;
  t->nu = nu;
  t->q = std::exp(-nu);
  double M[8];
  exp_moments(nu, 7, M);
  if (npts == 3) {
    const int nodes[3] = {-1, 0, 1};
    double w[3];
    weights_on(nodes, 3, M, w);
    for (int j = 0; j < 3; ++j) t->c[nodes[j] + 3] = w[j];
    return true;
  }
  if (npts != 5 && npts != 6) return false;
  const int n = npts;
  const int m = npts == 6 ? 4 : 3;  // substencil size
  int nodes[6];
  for (int j = 0; j < n; ++j) nodes[j] = -3 + j;
  double big[6];
  weights_on(nodes, n, M, big);
  for (int j = 0; j < n; ++j) t->c[j] = big[j];
  for (int r = 0; r < 3; ++r) {
    int sn[4];
    for (int j = 0; j < m; ++j) sn[j] = -3 + r + j;
    weights_on(sn, m, M, t->sub[r]);
  }
  // Linear weights: node -3 only in S_0, the last node only in S_2 (Sec. 2.4
  // definition); d_1 closes the partition of unity.
  t->d[0] = big[0] / t->sub[0][0];
  t->d[2] = big[n - 1] / t->sub[2][m - 1];
  t->d[1] = 1.0 - t->d[0] - t->d[2];
  // every node's weight must be reproduced
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int r = 0; r < 3; ++r) {
      const int k = j - r;
      if (k >= 0 && k < m) s += t->d[r] * t->sub[r][k];
    }
    if (std::fabs(s - big[j]) > 1e-12 * (std::fabs(big[j]) + nu)) return false;
  }
  return true;
}

}  // namespace molt
