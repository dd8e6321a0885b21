// 1D quadrature rules and Lagrange bases on [0, 1] (host, FP64).
//
// Gauss-Legendre points are the roots of P_n; Gauss-Lobatto nodes are
// {0, 1} and the roots of P_k'.  Both are found by Newton's method from
// Chebyshev-type starting values; only the lower half is iterated and the
// upper half is its mirror image, so the rules are exactly symmetric and an
// odd-count middle node is exactly 1/2 (Sec. 3.4: tensor-product Lagrange
// elements and Gauss quadrature).
#include <cmath>

#include "mfx_internal.h"

namespace mfx {

// P_n(t) and P_{n-1}(t) by Bonnet's recurrence.
static void legendre(int n, double t, double* p, double* pm1) {
  double a = 1.0, b = t;
  if (n == 0) { *p = 1.0; *pm1 = 0.0; return; }
  for (int m = 2; m <= n; ++m) {
    double c = ((2 * m - 1) * t * b - (m - 1) * a) / m;
    a = b;
    b = c;
  }
  *p = b;
  *pm1 = a;
}

void gauss_legendre(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  double t[kMaxN * 2];
  int h = n / 2;
  for (int i = 0; i < h; ++i) {
    double r = -std::cos(pi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, pm;
      legendre(n, r, &p, &pm);
      double dp = n * (r * p - pm) / (r * r - 1.0);
      double dr = p / dp;
      r -= dr;
      if (std::fabs(dr) < 1e-16) break;
    }
    t[i] = r;
    t[n - 1 - i] = -r;
  }
  if (n % 2) t[h] = 0.0;
  for (int i = 0; i < n; ++i) {
    double p, pm;
    legendre(n, t[i], &p, &pm);
    double dp = n * (t[i] * p - pm) / (t[i] * t[i] - 1.0);
    x[i] = 0.5 * (t[i] + 1.0);
    w[i] = 0.5 * (2.0 / ((1.0 - t[i] * t[i]) * dp * dp));
  }
}

void gauss_lobatto(int k, double* x) {
  const double pi = 3.14159265358979323846;
  double t[kMaxN * 2];
  t[0] = -1.0;
  t[k] = 1.0;
  int interior = k - 1, h = interior / 2;
  for (int j = 0; j < h; ++j) {
    double r = -std::cos(pi * (j + 1) / k);
    for (int it = 0; it < 100; ++it) {
      double p, pm;
      legendre(k, r, &p, &pm);
      double dp = k * (r * p - pm) / (r * r - 1.0);
      double d2p = (2.0 * r * dp - k * (k + 1) * p) / (1.0 - r * r);
      double dr = dp / d2p;
      r -= dr;
      if (std::fabs(dr) < 1e-16) break;
    }
    t[1 + j] = r;
    t[k - 1 - j] = -r;
  }
  if (interior % 2) t[1 + h] = 0.0;
  for (int i = 0; i <= k; ++i) x[i] = 0.5 * (t[i] + 1.0);
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
