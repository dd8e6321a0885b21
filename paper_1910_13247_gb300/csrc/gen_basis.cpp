// Build-time generator: writes the 1D matrices of every degree as C++ constants (the vmult
// kernels' S and D: the 1D shape functions and derivatives at the Gauss points on which the sum
// factorisation of Sec. 3.1 works; the SIPG double-float kernel's K1, M1 and end derivatives)
// (hexadecimal floating-point literals, exact FP64 values) for the vmult kernels,
// using the library's own quadrature and Lagrange routines (host_rules.cpp).
#include <cstdio>

#include "mfx_internal.h"

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  FILE* f = std::fopen(argv[1], "w");
  if (!f) return 1;
  std::fprintf(f, "// Generated at build time by gen_basis.cpp: S[q*N+j] = l_j(xi_q), D[q*N+p] = L_p'(xi_q),\n"
                 "// Sd[q*N+j] = l_j'(xi_q).\n");
  std::fprintf(f, "#pragma once\nnamespace mfx {\ntemplate <int N> struct BasisConst;\n");
  for (int k = 1; k <= mfx::kMaxDegree; ++k) {
    mfx::BasisTables t;
    mfx::make_basis(k, &t);
    const int n = k + 1;
    std::fprintf(f, "template <> struct BasisConst<%d> {\n", n);
    const char* names[3] = {"S", "D", "Sd"};
    const double* mats[3] = {t.S, t.D, t.Sd};
    for (int m = 0; m < 3; ++m) {
      std::fprintf(f, "  static __host__ __device__ constexpr double %s(int i) {\n    switch (i) {\n", names[m]);
      for (int i = 0; i < n * n; ++i) std::fprintf(f, "      case %d: return %a;\n", i, mats[m][i]);
      std::fprintf(f, "      default: return 0.0;\n    }\n  }\n");
    }
    std::fprintf(f, "};\n");
  }
  // SIPG tables on [0, 1]: K1 = Sd^T W Sd, M1 = S^T W S (exact with n-point Gauss), end derivatives
  std::fprintf(f, "template <int N> struct DgConst;\n");
  for (int k = 1; k <= mfx::kMaxDegree; ++k) {
    mfx::BasisTables t;
    mfx::make_basis(k, &t);
    const int n = k + 1;
    double K1[mfx::kMaxN * mfx::kMaxN], M1[mfx::kMaxN * mfx::kMaxN], e0[mfx::kMaxN], e1[mfx::kMaxN];
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double kk = 0.0, mm = 0.0;
        for (int q = 0; q < n; ++q) {
          kk += t.wq[q] * t.Sd[q * n + i] * t.Sd[q * n + j];
          mm += t.wq[q] * t.S[q * n + i] * t.S[q * n + j];
        }
        K1[i * n + j] = kk;
        M1[i * n + j] = mm;
      }
    for (int i = 0; i < n; ++i) {
      e0[i] = mfx::lagrange_derivative(n, t.gll, i, 0.0);
      e1[i] = mfx::lagrange_derivative(n, t.gll, i, 1.0);
    }
    std::fprintf(f, "template <> struct DgConst<%d> {\n", n);
    const char* names[4] = {"K1", "M1", "d0", "d1"};
    const double* mats[4] = {K1, M1, e0, e1};
    const int sizes[4] = {n * n, n * n, n, n};
    for (int m = 0; m < 4; ++m) {
      std::fprintf(f, "  static __host__ __device__ constexpr double %s(int i) {\n    switch (i) {\n", names[m]);
      for (int i = 0; i < sizes[m]; ++i) std::fprintf(f, "      case %d: return %a;\n", i, mats[m][i]);
      std::fprintf(f, "      default: return 0.0;\n    }\n  }\n");
    }
    std::fprintf(f, "};\n");
  }
  std::fprintf(f, "}  // namespace mfx\n");
  std::fclose(f);
  return 0;
}
