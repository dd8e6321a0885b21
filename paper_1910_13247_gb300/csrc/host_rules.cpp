// 1D quadrature rules and Lagrange bases on [0, 1] (host, FP64).
//
// Gauss-Legendre points are the roots of P_n; Gauss-Lobatto nodes are
// {0, 1} and the roots of P_k'.  Both are found by Newton's method from
// Chebyshev-type starting values on [-1, 1]; only the lower half is iterated
// and the upper half is its mirror image, and an odd-count middle node is
// exactly 1/2 (Sec. 3.4: tensor-product Lagrange elements and Gauss
// quadrature).  The iteration runs in long double (64- or 113-bit
// significand) and each point is rounded to double once, after the affine map
// to [0, 1], so it is the double nearest to the root it is defined as (a
// double-precision iteration followed by the map loses up to three bits near
// the ends of the interval).  Weights are evaluated at the rounded points.
#include <cmath>
#include <limits>

#include "mfx_internal.h"

namespace mfx {

// P_n(t) and P_{n-1}(t) by Bonnet's recurrence.
template <typename R>
static void legendre(int n, R t, R* p, R* pm1) {
  R a = 1, b = t;
  if (n == 0) { *p = 1; *pm1 = 0; return; }
  for (int m = 2; m <= n; ++m) {
    R c = ((2 * m - 1) * t * b - (m - 1) * a) / m;
    a = b;
    b = c;
  }
  *p = b;
  *pm1 = a;
}

// Newton steps stop below a few units in the last place of long double
static const long double kNewtonTol = 8 * std::numeric_limits<long double>::epsilon();

void gauss_legendre(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  long double t[kMaxN * 2];
  int h = n / 2;
  for (int i = 0; i < h; ++i) {
    long double r = -std::cos(pi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      long double p, pm;
      legendre<long double>(n, r, &p, &pm);
      long double dp = n * (r * p - pm) / (r * r - 1);
      long double dr = p / dp;
      r -= dr;
      if (std::fabs(dr) < kNewtonTol) break;
    }
    t[i] = r;
    t[n - 1 - i] = -r;
  }
  if (n % 2) t[h] = 0;
  for (int i = 0; i < n; ++i) {
    x[i] = (double)(0.5L * (t[i] + 1));  // one rounding, after the map to [0, 1]
    const double tr = 2.0 * x[i] - 1.0;  // the rounded point in [-1, 1] (exact)
    double p, pm;
    legendre<double>(n, tr, &p, &pm);
    double dp = n * (tr * p - pm) / (tr * tr - 1.0);
    w[i] = 0.5 * (2.0 / ((1.0 - tr * tr) * dp * dp));
  }
}

void gauss_lobatto(int k, double* x) {
  const double pi = 3.14159265358979323846;
  long double t[kMaxN * 2];
  t[0] = -1;
  t[k] = 1;
  int interior = k - 1, h = interior / 2;
  for (int j = 0; j < h; ++j) {
    long double r = -std::cos(pi * (j + 1) / k);
    for (int it = 0; it < 100; ++it) {
      long double p, pm;
      legendre<long double>(k, r, &p, &pm);
      long double dp = k * (r * p - pm) / (r * r - 1);
      long double d2p = (2 * r * dp - k * (k + 1) * p) / (1 - r * r);
      long double dr = dp / d2p;
      r -= dr;
      if (std::fabs(dr) < kNewtonTol) break;
    }
    t[1 + j] = r;
    t[k - 1 - j] = -r;
  }
  if (interior % 2) t[1 + h] = 0;
  for (int i = 0; i <= k; ++i) x[i] = (double)(0.5L * (t[i] + 1));  // one rounding, after the map
}

double lagrange_value(int n, const double* nodes, int j, double x) {
  double v = 1.0;
  for (int m = 0; m < n; ++m)
    if (m != j) v = v * (x - nodes[m]) / (nodes[j] - nodes[m]);
  return v;
}

double lagrange_derivative(int n, const double* nodes, int j, double x) {
  double s = 0.0;
  for (int m = 0; m < n; ++m) {
    if (m == j) continue;
    double t = 1.0 / (nodes[j] - nodes[m]);
    for (int l = 0; l < n; ++l)
      if (l != j && l != m) t = t * (x - nodes[l]) / (nodes[j] - nodes[l]);
    s += t;
  }
  return s;
}

void make_basis(int k, BasisTables* t) {
  int n = k + 1;
  t->k = k;
  t->n = n;
  gauss_lobatto(k, t->gll);
  gauss_legendre(n, t->xq, t->wq);
  for (int q = 0; q < n; ++q)
    for (int j = 0; j < n; ++j) {
      t->S[q * n + j] = lagrange_value(n, t->gll, j, t->xq[q]);
      t->Sd[q * n + j] = lagrange_derivative(n, t->gll, j, t->xq[q]);
      t->D[q * n + j] = lagrange_derivative(n, t->xq, j, t->xq[q]);
    }
}

}  // namespace mfx
