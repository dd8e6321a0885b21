/*
 * FP64 CPU oracle kernels (test infrastructure only; never linked into the
 * GPU library).  Plain loops written to be checked against the method by eye.
 *
 * Element matrix (Eq. 1 with coefficient, assembled as in the step-4 cell
 * loop of Sec. 2.4):
 *   A_ij = sum_q a(x_q) (J_q^{-T} grad phi_i(xi_q)) . (J_q^{-T} grad phi_j(xi_q)) |det J_q| w_q
 * with phi_i(xi) = l_i1(xi_1) l_i2(xi_2) l_i3(xi_3) evaluated as a 3D function
 * at every 3D quadrature point (no sum factorisation), the Q1 (trilinear)
 * mapping of the cell's 8 vertices, and the coefficient evaluated at the
 * physical quadrature point x_q.
 *
 * Right-hand side b_i = sum_q phi_i(x_q) f(x_q) |det J_q| w_q (step-4 loop).
 * Mass matrix M_ij = sum_q phi_i phi_j |det J_q| w_q.
 *
 * Vertex v of a cell is corner (a, b, c) = (v & 1, (v >> 1) & 1, (v >> 2) & 1).
 * Local DoF i = i1 + n (i2 + n i3), n = k + 1.
 *
 * Coefficient kinds: 0 constant a = p0;
 *                    1 a = p0 + p1 sin(2 pi x) cos(2 pi y) z.
 * Forcing kinds (manufactured u = sin(pi x) sin(pi y) sin(pi z)):
 *                    0 f = -div(a grad u) for the coefficient above;
 *                    2 f given as values at the quadrature points.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static const double PI = 3.14159265358979323846;

/* l_j(x) by the product formula */
static double lag(int n, const double* nodes, int j, double x) {
  double v = 1.0;
  for (int m = 0; m < n; ++m)
    if (m != j) v = v * (x - nodes[m]) / (nodes[j] - nodes[m]);
  return v;
}

/* l_j'(x) = sum_{m != j} 1/(x_j - x_m) prod_{l != j,m} (x - x_l)/(x_j - x_l) */
static double lag_d(int n, const double* nodes, int j, double x) {
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

static double coef(int kind, const double* p, const double x[3]) {
  if (kind == 0) return p[0];
  return p[0] + p[1] * sin(2 * PI * x[0]) * cos(2 * PI * x[1]) * x[2];
}

/* f = -div(a grad u) for u = sin(pi x) sin(pi y) sin(pi z) */
static double forcing(int kind, const double* p, const double x[3]) {
  double sx = sin(PI * x[0]), sy = sin(PI * x[1]), sz = sin(PI * x[2]);
  double cx = cos(PI * x[0]), cy = cos(PI * x[1]), cz = cos(PI * x[2]);
  double u = sx * sy * sz;
  double lap_u = -3.0 * PI * PI * u;
  double a = coef(kind, p, x);
  if (kind == 0) return -a * lap_u;
  double gu[3] = {PI * cx * sy * sz, PI * sx * cy * sz, PI * sx * sy * cz};
  double ga[3] = {p[1] * 2 * PI * cos(2 * PI * x[0]) * cos(2 * PI * x[1]) * x[2],
                  -p[1] * 2 * PI * sin(2 * PI * x[0]) * sin(2 * PI * x[1]) * x[2],
                  p[1] * sin(2 * PI * x[0]) * cos(2 * PI * x[1])};
  return -(ga[0] * gu[0] + ga[1] * gu[1] + ga[2] * gu[2] + a * lap_u);
}

/* Q1 map at reference point xi: physical point x, Jacobian J[i][j] = dx_i/dxi_j (Sec. 3.4) */
static void q1_map(const double* V /* 8x3 */, const double xi[3], double x[3], double J[3][3]) {
  for (int i = 0; i < 3; ++i) {
    x[i] = 0;
    for (int j = 0; j < 3; ++j) J[i][j] = 0;
  }
  for (int v = 0; v < 8; ++v) {
    int c[3] = {v & 1, (v >> 1) & 1, (v >> 2) & 1};
    double N[3], dN[3];
    for (int d = 0; d < 3; ++d) {
      N[d] = c[d] ? xi[d] : 1.0 - xi[d];
      dN[d] = c[d] ? 1.0 : -1.0;
    }
    double shape = N[0] * N[1] * N[2];
    double grad[3] = {dN[0] * N[1] * N[2], N[0] * dN[1] * N[2], N[0] * N[1] * dN[2]};
    for (int i = 0; i < 3; ++i) {
      x[i] += shape * V[3 * v + i];
      for (int j = 0; j < 3; ++j) J[i][j] += V[3 * v + i] * grad[j];
    }
  }
}

static double inverse3(const double J[3][3], double Ji[3][3]) {
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
               J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  return det;
}

/* Quadrature-point data shared by the cell routines below. */
typedef struct {
  double x[3];    /* physical point */
  double JxW;     /* |det J| w */
  double Jit[3][3]; /* J^{-T} */
} qdata;

static void eval_q(const double* V, const double* xq, const double* wq, int nq, int q, qdata* d) {
  int q1 = q % nq, q2 = (q / nq) % nq, q3 = q / (nq * nq);
  double xi[3] = {xq[q1], xq[q2], xq[q3]};
  double J[3][3], Ji[3][3];
  q1_map(V, xi, d->x, J);
  double det = inverse3(J, Ji);
  d->JxW = fabs(det) * wq[q1] * wq[q2] * wq[q3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) d->Jit[i][j] = Ji[j][i];
}

/* reference gradient and value of phi_i at reference point xi */
static void shape(int k, const double* nodes, int i, const double xi[3], double* val, double g[3]) {
  int n = k + 1;
  int i1 = i % n, i2 = (i / n) % n, i3 = i / (n * n);
  double l1 = lag(n, nodes, i1, xi[0]), l2 = lag(n, nodes, i2, xi[1]), l3 = lag(n, nodes, i3, xi[2]);
  double d1 = lag_d(n, nodes, i1, xi[0]), d2 = lag_d(n, nodes, i2, xi[1]), d3 = lag_d(n, nodes, i3, xi[2]);
  *val = l1 * l2 * l3;
  g[0] = d1 * l2 * l3;
  g[1] = l1 * d2 * l3;
  g[2] = l1 * l2 * d3;
}

/*
 * Element matrices of `ncell` cells: out[c][i][j], i, j < n^3 (Eq. 1 by the
 * step-4 cell loop of Sec. 2.4).
 * rows: optional list of local rows to compute (nrows > 0); then out[c][r][j].
 */
int or_cell_matrices(int ncell, int k, int nq, const double* nodes, const double* xq,
                     const double* wq, const double* verts, int coef_kind, const double* cpar,
                     int nrows, const int* rows, double* out) {
  int n = k + 1, nd = n * n * n, NQ = nq * nq * nq;
  int nr = nrows > 0 ? nrows : nd;
#pragma omp parallel for schedule(dynamic)
  for (int c = 0; c < ncell; ++c) {
    double* A = out + (size_t)c * nr * nd;
    double* grad = (double*)malloc(sizeof(double) * 3 * nd);
    memset(A, 0, sizeof(double) * nr * nd);
    for (int q = 0; q < NQ; ++q) {
      qdata d;
      eval_q(verts + 24 * (size_t)c, xq, wq, nq, q, &d);
      int q1 = q % nq, q2 = (q / nq) % nq, q3 = q / (nq * nq);
      double xi[3] = {xq[q1], xq[q2], xq[q3]};
      double a = coef(coef_kind, cpar, d.x);
      for (int i = 0; i < nd; ++i) {
        double v, g[3];
        shape(k, nodes, i, xi, &v, g);
        for (int r = 0; r < 3; ++r)
          grad[3 * i + r] = d.Jit[r][0] * g[0] + d.Jit[r][1] * g[1] + d.Jit[r][2] * g[2];
      }
      for (int ri = 0; ri < nr; ++ri) {
        int i = nrows > 0 ? rows[ri] : ri;
        for (int j = 0; j < nd; ++j)
          A[(size_t)ri * nd + j] += a *
              (grad[3 * i] * grad[3 * j] + grad[3 * i + 1] * grad[3 * j + 1] +
               grad[3 * i + 2] * grad[3 * j + 2]) * d.JxW;
      }
    }
    free(grad);
  }
  return 0;
}

/* Element mass matrices out[c][i][j] = sum_q phi_i phi_j JxW (the loop of Sec. 2.4). */
int or_cell_mass(int ncell, int k, int nq, const double* nodes, const double* xq,
                 const double* wq, const double* verts, double* out) {
  int n = k + 1, nd = n * n * n, NQ = nq * nq * nq;
#pragma omp parallel for schedule(dynamic)
  for (int c = 0; c < ncell; ++c) {
    double* M = out + (size_t)c * nd * nd;
    double* val = (double*)malloc(sizeof(double) * nd);
    memset(M, 0, sizeof(double) * nd * nd);
    for (int q = 0; q < NQ; ++q) {
      qdata d;
      eval_q(verts + 24 * (size_t)c, xq, wq, nq, q, &d);
      int q1 = q % nq, q2 = (q / nq) % nq, q3 = q / (nq * nq);
      double xi[3] = {xq[q1], xq[q2], xq[q3]}, g[3];
      for (int i = 0; i < nd; ++i) shape(k, nodes, i, xi, &val[i], g);
      for (int i = 0; i < nd; ++i)
        for (int j = 0; j < nd; ++j) M[(size_t)i * nd + j] += val[i] * val[j] * d.JxW;
    }
    free(val);
  }
  return 0;
}

/*
 * Element right-hand sides out[c][i] = sum_q phi_i(x_q) f(x_q) JxW (step-4
 * loop, Sec. 2.4).
 * force_kind 0: manufactured forcing for coefficient (coef_kind, cpar);
 * force_kind 2: fq[c][q] given.
 */
int or_cell_rhs(int ncell, int k, int nq, const double* nodes, const double* xq,
                const double* wq, const double* verts, int coef_kind, const double* cpar,
                int force_kind, const double* fq, double* out) {
  int n = k + 1, nd = n * n * n, NQ = nq * nq * nq;
#pragma omp parallel for schedule(dynamic)
  for (int c = 0; c < ncell; ++c) {
    double* b = out + (size_t)c * nd;
    memset(b, 0, sizeof(double) * nd);
    for (int q = 0; q < NQ; ++q) {
      qdata d;
      eval_q(verts + 24 * (size_t)c, xq, wq, nq, q, &d);
      int q1 = q % nq, q2 = (q / nq) % nq, q3 = q / (nq * nq);
      double xi[3] = {xq[q1], xq[q2], xq[q3]}, g[3], v;
      double f = force_kind == 2 ? fq[(size_t)c * NQ + q] : forcing(coef_kind, cpar, d.x);
      for (int i = 0; i < nd; ++i) {
        shape(k, nodes, i, xi, &v, g);
        b[i] += v * f * d.JxW;
      }
    }
  }
  return 0;
}

/* Physical quadrature points out[c][q][3] and JxW[c][q]. */
int or_cell_qpoints(int ncell, int nq, const double* xq, const double* wq, const double* verts,
                    double* xout, double* jxw) {
  int NQ = nq * nq * nq;
  for (int c = 0; c < ncell; ++c)
    for (int q = 0; q < NQ; ++q) {
      qdata d;
      eval_q(verts + 24 * (size_t)c, xq, wq, nq, q, &d);
      for (int i = 0; i < 3; ++i) xout[((size_t)c * NQ + q) * 3 + i] = d.x[i];
      jxw[(size_t)c * NQ + q] = d.JxW;
    }
  return 0;
}

/*
 * Squared L2 error sum_c sum_q (u_h(x_q) - u(x_q))^2 JxW with the given rule
 * (xq, wq, nq) and u = sin(pi x) sin(pi y) sin(pi z); ucell[c][i] are the
 * cell's nodal values.
 */
double or_l2_error_sq(int ncell, int k, int nq, const double* nodes, const double* xq,
                      const double* wq, const double* verts, const double* ucell, int exact) {
  int n = k + 1, nd = n * n * n, NQ = nq * nq * nq;
  double total = 0.0;
#pragma omp parallel for reduction(+ : total) schedule(dynamic)
  for (int c = 0; c < ncell; ++c) {
    for (int q = 0; q < NQ; ++q) {
      qdata d;
      eval_q(verts + 24 * (size_t)c, xq, wq, nq, q, &d);
      int q1 = q % nq, q2 = (q / nq) % nq, q3 = q / (nq * nq);
      double xi[3] = {xq[q1], xq[q2], xq[q3]}, g[3], v, uh = 0.0;
      for (int i = 0; i < nd; ++i) {
        shape(k, nodes, i, xi, &v, g);
        uh += ucell[(size_t)c * nd + i] * v;
      }
      /* exact solution: 0 -> sin(pi x) sin(pi y) sin(pi z) (u = 0 on every face),
         1 -> sin(pi x) (u = 0 on the x faces, zero normal derivative on the others) */
      double u = exact == 1 ? sin(PI * d.x[0]) : sin(PI * d.x[0]) * sin(PI * d.x[1]) * sin(PI * d.x[2]);
      total += (uh - u) * (uh - u) * d.JxW;
    }
  }
  return total;
}

/* y = A x for a CSR matrix, plain row loop: the action the matrix-free operator of Sec. 3.6 computes. */
int or_csr_spmv(int64_t nrows, const int64_t* rowptr, const int64_t* col, const double* val,
                const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < nrows; ++r) {
    double s = 0.0;
    for (int64_t p = rowptr[r]; p < rowptr[r + 1]; ++p) s += val[p] * x[col[p]];
    y[r] = s;
  }
  return 0;
}
