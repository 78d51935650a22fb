// Device-side building blocks shared by the kernels of libvst.
//
// Covariance: the non-separable Gneiting form of Eq. (2) with d = 2,
//   C(h, u) = sigma1^2 psi(u)^{-(delta+gamma)} M_nu(c h psi(u)^{-gamma/2}),
//   psi(u)  = a |u|^{2 alpha} + 1,
// for the closed-form Matern orders nu in {0.5, 1.5, 2.5} (Sect. 4.5).
// Everything that depends on the time lag alone is tabulated once per call
// for integer lags ("lag table"); non-integer or very long lags fall back to
// evaluating psi directly in FP64.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "vst.h"

namespace vst {

constexpr int kLagTab = 1024;          // integer lags 0..kLagTab-1 are tabulated
// mixed form: default threshold of the condition estimate (max_j L_jj /
// min_j L_jj)^2 above which a row is redone in FP64
constexpr float kDefaultTau = 1.0e4f;
constexpr unsigned kFull = 0xffffffffu;

// Parameters as the kernels see them (by value in the kernel arguments).
struct DevTheta {
  double sigma1sq, c, a, gamma, nugget, alpha, delta, nu;
  double p;            // delta + gamma * d / 2 with d = 2
  float dg_hi, dg_lo;  // sigma1^2 + nugget as a double-float (mixed form's diagonal)
  // FP32 constants of the mixed form's gradient: 1/sigma1^2, 1/c, gamma/2, p
  float inv_s1f, inv_cf, hgf, pf;
};

// Derived fields of a DevTheta whose eight parameters are set.
__host__ __device__ inline void finish_dev_theta(DevTheta& d) {
  d.p = d.delta + d.gamma;  // delta + gamma d/2, d = 2
  const double dg = d.sigma1sq + d.nugget;
  d.dg_hi = (float)dg;
  d.dg_lo = (float)(dg - (double)d.dg_hi);
  d.inv_s1f = (float)(1.0 / d.sigma1sq);
  d.inv_cf = (float)(1.0 / d.c);
  d.hgf = (float)(0.5 * d.gamma);
  d.pf = (float)d.p;
}

// Padded size of the local (m+1) x (m+1) block: the row kernels are
// instantiated for PM = 8, 16, 24, 32 (multiples of the 16-byte FP32 row loads)
__host__ __device__ constexpr int padded_pm(int p) { return p <= 8 ? 8 : p <= 16 ? 16 : p <= 24 ? 24 : 32; }

// Precision codes accepted by the single-dataset entry points; the plain
// Vecchia path has one mixed form (VST_MIXED_BF16X3 only changes the VIF
// low-rank product).
inline bool valid_precision(int p) { return p == VST_FP64 || p == VST_MIXED || p == VST_MIXED_BF16X3; }
inline int plain_precision(int p) { return p == VST_MIXED_BF16X3 ? VST_MIXED : p; }

// Per-point record read by the mixed-precision row kernel, written once per
// call so that the per-row work has no FP64 arithmetic: coordinates and the
// response as double-floats (hi + lo), the day index and whether the time is
// an integer day (|t| < 1e9).
struct __align__(16) PrepPt {
  float xhi, xlo, yhi, ylo;
  float vhi, vlo;
  int td, tint;
};

// Per-lag factors of Eq. (2) and of its parameter derivatives:
//   P  = sigma1^2 psi^{-(delta+gamma)}   (amplitude at this lag)
//   G  = c psi^{-gamma/2}                (x = G h is the Matern argument)
//   Qa = |u|^{2 alpha} / psi             (d psi / d a, divided by psi)
//   L  = ln psi                          (d/d gamma of the psi powers)
struct LagD { double P, G, Qa, L; };
struct __align__(16) LagF { float P, G, Qa, L; };

__host__ __device__ inline LagD lag_factors(const DevTheta& th, double u) {
  u = fabs(u);
  const double au = (u == 0.0) ? 0.0 : pow(u, 2.0 * th.alpha);
  const double psi = th.a * au + 1.0;
  const double L = log(psi);
  LagD r;
  r.P = th.sigma1sq * exp(-th.p * L);
  r.G = th.c * exp(-0.5 * th.gamma * L);
  r.Qa = au / psi;
  r.L = L;
  return r;
}

// Matern part, NU = 0, 1, 2 for nu = 0.5, 1.5, 2.5; E = exp(-x).
template <int NU, typename T>
__device__ __forceinline__ T matern_M(T x, T E) {
  if (NU == 0) return E;
  if (NU == 1) return (T(1) + x) * E;
  return (T(1) + x + x * x * T(1.0 / 3.0)) * E;
}
// x * dM/dx
template <int NU, typename T>
__device__ __forceinline__ T matern_xdM(T x, T E) {
  if (NU == 0) return -x * E;
  if (NU == 1) return -x * x * E;
  return -(x * x * T(1.0 / 3.0)) * (T(1) + x) * E;
}

template <typename T> __device__ __forceinline__ T dexp(T x);
template <> __device__ __forceinline__ float dexp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double dexp<double>(double x) { return exp(x); }
template <typename T> __device__ __forceinline__ T drsqrt(T x);
// 1/sqrt(x) by the hardware approximation, denormal inputs and outputs
// flushed to zero (rsqrtf also handles denormal inputs, at the cost of a few
// instructions per call; the arguments here are variances and squared
// distances, and a zero or flushed one is handled where it occurs)
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
template <> __device__ __forceinline__ float drsqrt<float>(float x) { return rsqrt_ftz(x); }
// the smallest normal FP32 value: squared distances below it count as 0
constexpr float kFltMinNormal = 1.17549435e-38f;
template <> __device__ __forceinline__ double drsqrt<double>(double x) { return rsqrt(x); }
template <typename T> __device__ __forceinline__ T dsqrt(T x);
template <> __device__ __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }

// ---------------------------------------------------------------------------
// Double-float ("FP32 pair") arithmetic for the refinement residuals of the
// mixed-precision form.  Error-free transformations: TwoSum (Knuth, TAOCP
// vol. 2) and the FMA-based TwoProduct (the exact product error a*b - fl(a*b)
// is representable and one fused multiply-add computes it).
struct df { float hi, lo; };

__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float err = (a - (s - bb)) + (b - bb);
  return {s, err};
}
// s += a * b  (a float, b double-float), result not renormalised every step
__device__ __forceinline__ void df_fma_acc(df& s, float a, df b) {
  const float p = a * b.hi;
  const float pe = fmaf(a, b.hi, -p);
  const float q = fmaf(a, b.lo, pe);
  const df t = df_two_sum(s.hi, p);
  s.hi = t.hi;
  s.lo = s.lo + (t.lo + q);
}
// (ah + al) - (bh + bl) rounded to FP32: TwoSum of the leading parts plus the
// trailing parts; within an ulp or two of the exactly rounded difference.
__device__ __forceinline__ float df_diff(float ah, float al, float bh, float bl) {
  const df t = df_two_sum(ah, -bh);
  return t.hi + (t.lo + (al - bl));
}
// Two independent double-float sums (hi + lo, componentwise) on packed FP32
// pairs: hi + lo -= a * b exactly up to the final additions, the product
// split by one fused multiply-add (TwoProduct) and the sum by TwoSum.
__device__ __forceinline__ void df2_dot_sub(float2& hi, float2& lo, float2 a, float2 b) {
  const float2 p = __fmul2_rn(make_float2(-a.x, -a.y), b);
  const float2 pe = __ffma2_rn(make_float2(-a.x, -a.y), b, make_float2(-p.x, -p.y));
  const float2 sm = __fadd2_rn(hi, p);
  const float2 bb = __fadd2_rn(sm, make_float2(-hi.x, -hi.y));
  const float2 t = __fadd2_rn(sm, make_float2(-bb.x, -bb.y));
  const float2 e1 = __fadd2_rn(hi, make_float2(-t.x, -t.y));
  const float2 e2 = __fadd2_rn(p, make_float2(-bb.x, -bb.y));
  lo = __fadd2_rn(lo, __fadd2_rn(__fadd2_rn(e1, e2), pe));
  hi = sm;
}
__device__ __forceinline__ df df_split(double v) {
  const float hi = (float)v;
  return {hi, (float)(v - (double)hi)};
}
__device__ __forceinline__ double df_to_double(df v) { return (double)v.hi + (double)v.lo; }

// Warp-wide sum of a double-float, fixed xor tree (same order every call).
__device__ __forceinline__ df df_warp_sum(df v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(kFull, v.hi, o);
    const float ol = __shfl_xor_sync(kFull, v.lo, o);
    const df t = df_two_sum(v.hi, oh);
    v.hi = t.hi;
    v.lo = v.lo + ol + t.lo;
  }
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Workspace header written by the kernels (mirrors vst_ws_info).
struct WsHeader {
  int32_t status;
  int32_t reserved;
  unsigned long long bad_row;   // atomicMin target; ~0ull = none
  unsigned long long n_fallback;
  unsigned long long n_tie;
};

__device__ __forceinline__ void report_error(WsHeader* h, int code, long long row) {
  atomicCAS(&h->status, 0, code);
  atomicMin(&h->bad_row, (unsigned long long)row);
}

}  // namespace vst
