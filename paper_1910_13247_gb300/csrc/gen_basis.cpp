// Build-time generator: writes the 1D matrices of every degree as C++ constants
// (hexadecimal floating-point literals, exact FP64 values) for the vmult kernels,
// using the library's own quadrature and Lagrange routines (host_rules.cpp).
#include <cstdio>

#include "mfx_internal.h"

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  FILE* f = std::fopen(argv[1], "w");
  if (!f) return 1;
  std::fprintf(f, "// Generated at build time by gen_basis.cpp: S[q*N+j] = l_j(xi_q), D[q*N+p] = L_p'(xi_q).\n");
  std::fprintf(f, "#pragma once\nnamespace mfx {\ntemplate <int N> struct BasisConst;\n");
  for (int k = 1; k <= mfx::kMaxDegree; ++k) {
    mfx::BasisTables t;
    mfx::make_basis(k, &t);
    const int n = k + 1;
    std::fprintf(f, "template <> struct BasisConst<%d> {\n", n);
    const char* names[2] = {"S", "D"};
    const double* mats[2] = {t.S, t.D};
    for (int m = 0; m < 2; ++m) {
      std::fprintf(f, "  static __host__ __device__ constexpr double %s(int i) {\n    switch (i) {\n", names[m]);
      for (int i = 0; i < n * n; ++i) std::fprintf(f, "      case %d: return %a;\n", i, mats[m][i]);
      std::fprintf(f, "      default: return 0.0;\n    }\n  }\n");
    }
    std::fprintf(f, "};\n");
  }
  std::fprintf(f, "}  // namespace mfx\n");
  std::fclose(f);
  return 0;
}
