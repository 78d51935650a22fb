// Double-float ("FP32 pair", ~48 significand bits) arithmetic for the VIF
// residual covariance of the mixed form: products, sums, square root and
// e^{-x}, built on the error-free transformations of common.cuh (TwoSum,
// FMA TwoProduct).  The methods follow the double-double library of Hida,
// Li and Bailey ("Library for double-double and quad-double arithmetic",
// 2007), carried over to pairs of FP32 values:
//   * products: the exact product of the leading parts (FMA) plus the cross
//     terms, renormalised;
//   * square root: one Newton correction of the FP32 root;
//   * exp: Cody-Waite reduction x = n ln2 + r (ln2 in three parts, the first
//     with 15 significand bits so that n * part is exact for |n| < 2^9),
//     Taylor series of e^{r/16} to degree 6, squared four times, scaled by 2^n.
// Relative accuracy ~1e-12 (checked against FP64 on the GPU by the VIF
// parity tests), far below the FP32 rounding of the residual block it feeds.
#pragma once

#include "common.cuh"

namespace vst {

// s + e with |s| >= |e| (Dekker's fast TwoSum)
__device__ __forceinline__ df df_fast(float s, float e) {
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ df dfm_add(df a, df b) {
  const df s = df_two_sum(a.hi, b.hi);
  return df_fast(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ df dfm_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast(p, e);
}
__device__ __forceinline__ df dfm_scale(df a, float s) {  // s a power of two
  return {a.hi * s, a.lo * s};
}
// a >= 0
__device__ __forceinline__ df dfm_sqrt(df a) {
  if (!(a.hi > 0.f)) return {0.f, 0.f};
  const float y = sqrtf(a.hi);
  const float p = __fmul_rn(y, y);
  const float e = fmaf(y, y, -p);
  const float r = ((a.hi - p) - e) + a.lo;  // a - y^2 (a.hi - p is exact)
  return df_fast(y, r / (2.0f * y));
}

// 1 / j! as a double-float (leading part, remainder)
template <int J>
struct InvFact {
  static constexpr double v = InvFact<J - 1>::v / J;
  static constexpr float hi = (float)v;
  static constexpr float lo = (float)(v - (double)(float)v);
};
template <>
struct InvFact<0> {
  static constexpr double v = 1.0;
  static constexpr float hi = 1.0f;
  static constexpr float lo = 0.0f;
};

// e^{-x} for x >= 0 (0 below the FP32 range)
__device__ __forceinline__ df dfm_exp_neg(df x) {
  if (!(x.hi < 87.0f)) return {0.f, 0.f};
  constexpr float kInvLn2 = 1.4426950408889634f;
  constexpr double kLn2 = 0.6931471805599453094;
  constexpr float c1 = 0.693145751953125f;  // 15 significand bits
  constexpr float c2 = (float)(kLn2 - 0.693145751953125);
  constexpr float c3 = (float)(kLn2 - 0.693145751953125 - (double)(float)(kLn2 - 0.693145751953125));
  const df y = {-x.hi, -x.lo};
  const float n = rintf(y.hi * kInvLn2);
  // r = y - n ln2
  df r = df_two_sum(fmaf(-n, c1, y.hi), -n * c2);  // n c1 exact; y.hi - n c1 exact (Sterbenz)
  const float p2e = fmaf(-n, c2, n * c2);          // rounding error of n c2
  r = df_fast(r.hi, r.lo + (p2e - n * c3) + y.lo);
  // e^{r/16} by Horner, then square four times
  const df s = dfm_scale(r, 0.0625f);
  df t = {InvFact<6>::hi, InvFact<6>::lo};
  t = dfm_add(dfm_mul(t, s), df{InvFact<5>::hi, InvFact<5>::lo});
  t = dfm_add(dfm_mul(t, s), df{InvFact<4>::hi, InvFact<4>::lo});
  t = dfm_add(dfm_mul(t, s), df{InvFact<3>::hi, InvFact<3>::lo});
  t = dfm_add(dfm_mul(t, s), df{InvFact<2>::hi, InvFact<2>::lo});
  t = dfm_add(dfm_mul(t, s), df{1.0f, 0.0f});
  t = dfm_add(dfm_mul(t, s), df{1.0f, 0.0f});
#pragma unroll
  for (int q = 0; q < 4; ++q) t = dfm_mul(t, t);
  const int ni = (int)n;
  return {ldexpf(t.hi, ni), ldexpf(t.lo, ni)};
}

// Matern M_nu(x) for nu = 0.5, 1.5, 2.5 given E = e^{-x}
template <int NU>
__device__ __forceinline__ df dfm_matern(df x, df E) {
  if (NU == 0) return E;
  if (NU == 1) return dfm_mul(dfm_add(df{1.f, 0.f}, x), E);
  // 1 + x + x^2 / 3
  const df x2 = dfm_mul(x, x);
  constexpr float t_hi = (float)(1.0 / 3.0);
  constexpr float t_lo = (float)(1.0 / 3.0 - (double)(float)(1.0 / 3.0));
  const df q = dfm_add(dfm_add(df{1.f, 0.f}, x), dfm_mul(x2, df{t_hi, t_lo}));
  return dfm_mul(q, E);
}

}  // namespace vst
