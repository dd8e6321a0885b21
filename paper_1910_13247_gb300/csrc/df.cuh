// Double-float arithmetic: a value as an unevaluated sum of two floats (hi + lo, about 48 significant
// bits).  Products with a constant are formed exactly by FMA-based error-free transformations (the
// product error of a*b is fma(a, b, -a*b), as in Ogita, Rump and Oishi's accurate dot product, 2005),
// sums by Knuth's two-sum; all operations use the round-to-nearest intrinsics, which the compiler
// never fuses, so the transformations stay exact.  Used by the FP64 operators, because GB300 runs FP64 FMAs at 1/62 of
// the FP32 rate.
#pragma once

namespace mfx {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_split(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_join(df a) { return (double)a.hi + (double)a.lo; }

// s + t with |s| >= |t| (or s = 0): normalised pair
__device__ __forceinline__ df df_fast_norm(float s, float t) {
  const float h = __fadd_rn(s, t);
  return {h, __fsub_rn(t, __fsub_rn(h, s))};
}

// (s, t) = x * c exactly up to the lo*lo term (first term of a sum)
__device__ __forceinline__ void df_prod(df x, float ch, float cl, float& s, float& t) {
  s = __fmul_rn(x.hi, ch);
  float e = __fmaf_rn(x.hi, ch, -s);
  e = __fmaf_rn(x.hi, cl, e);
  t = __fmaf_rn(x.lo, ch, e);
}

// (s, t) += x * c: two-sum of the high parts, error terms into t
__device__ __forceinline__ void df_prod_acc(df x, float ch, float cl, float& s, float& t) {
  const float p = __fmul_rn(x.hi, ch);
  float e = __fmaf_rn(x.hi, ch, -p);
  e = __fmaf_rn(x.hi, cl, e);
  e = __fmaf_rn(x.lo, ch, e);
  const float s2 = __fadd_rn(s, p);
  const float bv = __fsub_rn(s2, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(s2, bv)), __fsub_rn(p, bv));
  s = s2;
  t = __fadd_rn(t, __fadd_rn(err, e));
}

__device__ __forceinline__ df df_dot3(df a0, df b0, df a1, df b1, df a2, df b2) {
  float s, t;
  df_prod(b0, a0.hi, a0.lo, s, t);
  df_prod_acc(b1, a1.hi, a1.lo, s, t);
  df_prod_acc(b2, a2.hi, a2.lo, s, t);
  return df_fast_norm(s, t);
}

__device__ __forceinline__ df df_add(df a, df b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bv = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bv)), __fsub_rn(b.hi, bv));
  return df_fast_norm(s, __fadd_rn(err, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_add3(df a, df b, df c) { return df_add(df_add(a, b), c); }

// compile-time split of the 1D matrices
constexpr float split_hi(double v) { return (float)v; }
constexpr float split_lo(double v) { return (float)(v - (double)(float)v); }

}  // namespace mfx
