// Fused per-row Vecchia kernel: for each row i (one warp per row),
//   1. gather the |N(i)| <= m neighbours and row i itself (position PM-1),
//   2. evaluate the local (m+1) x (m+1) response covariance Sigma~ (Eq. (2)
//      plus the nugget on the diagonal, Sect. 3.1),
//   3. Cholesky-factor it with row j of the factor held in lane j's registers,
//   4. solve for A_i = Sigma~_{i,N} Sigma~_N^{-1} and D_i (Sect. 4.1) and the
//      whitened residual, giving the NLL term 1/2 log D_i + 1/2 r_i^2 / D_i,
//   5. (gradient) contract the adjoint weights dNLL_i/dSigma~ with the
//      covariance derivatives dSigma~/dtheta, recomputed pair by pair.
//
// The factor of the (m+1)-block with row i last contains everything:
// its last row is [w^T, sqrt(D_i)] with w = L_N^{-1} k, and A_i = L_N^{-T} w.
// Unused positions (rows with fewer than m neighbours) are padded with unit
// diagonal entries and zero cross-covariances, which leaves the factor of the
// used block unchanged.
//
// Adjoint of one row.  With a~ = (-A_i, 1) and b~ = (Sigma~_N^{-1} y_N, 0) on
// the positions (N(i), i), r = y_i - A_i y_N and D = D_i:
//   dD      = a~^T dSigma~ a~
//   d(A y_N) = a~^T dSigma~ b~
//   dNLL_i  = c1 a~^T dSigma~ a~ - c2 a~^T dSigma~ b~,
//   c1 = (1/D - r^2/D^2) / 2,  c2 = r / D,
// i.e. dNLL_i = sum_{p,q} W_pq dSigma~_pq with the symmetric adjoint weight
// W = c1 a~ a~^T - c2 (a~ b~^T + b~ a~^T) / 2: one pass over the pairs, O(m^2)
// per row, no stored factor.
//
// Mixed precision (T = float): covariance and Cholesky in FP32; one step of
// iterative refinement of A_i whose residual k - K_N A_i is accumulated in
// double-float arithmetic; D_i and r_i are formed in double-float; every sum
// over rows is FP64.  Rows whose Cholesky fails in FP32, or whose condition
// estimate (max_j L_jj / min_j L_jj)^2 exceeds tau, are flagged and redone by
// the FP64 instantiation.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace vst {

enum RowMode { kModeNll = 0, kModeNllGrad = 1, kModeFactor = 2 };

struct RowArgs {
  const double* xy;
  const double* t;
  const double* y;
  const int32_t* nn;
  const int32_t* nn_cnt;
  int64_t n;
  int m;
  DevTheta th;
  const LagD* lagd;
  const LagF* lagf;
  double* A;          // factor outputs
  double* D;
  double* partial;    // [total warps][8]: nll, grad[5]
  uint8_t* flag;      // [n] rows redone in FP64 (mixed writes, FP64 fallback reads)
  WsHeader* hdr;
  float tau;          // condition threshold of the mixed form
  int fallback_only;  // FP64 kernel: only rows with flag[i] != 0
  // batched form: dataset of each row range (nullptr for a single dataset)
  const int64_t* offsets;     // [nsets + 1] row offsets
  const DevTheta* thetas;     // [nsets]
  const LagD* lagd_sets;      // [nsets][kLagTab]
  const LagF* lagf_sets;
  int nsets;
  double* row_out;            // batched: per-row [6] (nll term, grad[5])
};

template <typename T, int PM>
struct WarpSm {
  T K[PM][PM + 1];                       // local covariance (FP64: reused for L)
  T Ls[std::is_same<T, float>::value ? PM : 1][PM + 1];  // mixed: factor L
  alignas(16) T col[PM];                 // column broadcast during Cholesky
  alignas(16) T v0[PM];                  // a (and a~)
  alignas(16) T v1[PM];                  // b~
  T ox[PM], oy[PM];                      // offsets from row i
  double tt[PM];                         // times (non-integer lag fallback)
  int td[PM];                            // integer days
  int valid[PM];
};

template <typename T>
__device__ __forceinline__ void lag_lookup(const RowArgs& g, const DevTheta& th, const LagD* lagd,
                                           const LagF* lagf, bool allint, int tdr, int tdc,
                                           double ttr, double ttc, T& P, T& G, T& Qa, T& L) {
  const int lag = abs(tdr - tdc);
  if (allint && lag < kLagTab) {
    if constexpr (std::is_same<T, float>::value) {
      const float4 f = __ldg(reinterpret_cast<const float4*>(lagf) + lag);
      P = f.x; G = f.y; Qa = f.z; L = f.w;
    } else {
      const double2 a = __ldg(reinterpret_cast<const double2*>(lagd) + 2 * lag);
      const double2 b = __ldg(reinterpret_cast<const double2*>(lagd) + 2 * lag + 1);
      P = a.x; G = a.y; Qa = b.x; L = b.y;
    }
  } else {
    const LagD f = lag_factors(th, ttr - ttc);
    P = (T)f.P; G = (T)f.G; Qa = (T)f.Qa; L = (T)f.L;
  }
}

// Process one row; all 32 lanes call it together.  Returns false if the row
// was skipped (error, or flagged for the FP64 fallback).
template <typename T, int NU, int PM, int MODE>
__device__ __forceinline__ void row_body(const RowArgs& g, const DevTheta& th, const LagD* lagd,
                                         const LagF* lagf, WarpSm<T, PM>& s, int64_t i, int64_t row0,
                                         int lane, double& acc_nll, double (&acc_g)[5]) {
  constexpr bool MIXED = std::is_same<T, float>::value;
  constexpr int LAST = PM - 1;
  const int m = g.m;
  const int64_t gi = row0 + i;  // global row (batched form); nn indices are local
  const int cnt = g.nn_cnt[gi];
  if (cnt < 0 || cnt > m || cnt > LAST || (int64_t)cnt > i) {
    if (lane == 0) report_error(g.hdr, VST_EINVAL, gi);
    return;
  }
  int idx = -1;
  bool bad = false;
  if (lane < cnt) {
    idx = g.nn[gi * m + lane];
    bad = (idx < 0) || ((int64_t)idx >= i);
  }
  if (__any_sync(kFull, bad)) {
    if (lane == 0) report_error(g.hdr, VST_EINVAL, gi);
    return;
  }
  if (lane == LAST) idx = (int)i;
  const bool valid = idx >= 0;
  const double* xy = g.xy + 2 * row0;
  const double* tv = g.t + row0;
  const double xi = xy[2 * i], yi = xy[2 * i + 1];
  double xj = xi, yj = yi, tj = tv[i], rj = 0.0;
  if (valid) {
    xj = xy[2 * (int64_t)idx];
    yj = xy[2 * (int64_t)idx + 1];
    tj = tv[idx];
    if (MODE != kModeFactor) rj = g.y[row0 + idx];
  }
  const bool tint = (tj == floor(tj)) && fabs(tj) < 1.0e9;
  const bool allint = __all_sync(kFull, tint);
  if (lane < PM) {
    s.ox[lane] = (T)(xj - xi);
    s.oy[lane] = (T)(yj - yi);
    s.tt[lane] = tj;
    s.td[lane] = allint ? (int)tj : 0;
    s.valid[lane] = valid;
  }
  __syncwarp();

  // ---- 2. local covariance, lower triangle distributed over the lanes
  constexpr int NPAIR = PM * (PM + 1) / 2;
  const T diag = (T)(th.sigma1sq + th.nugget);
  for (int e = lane; e < NPAIR; e += 32) {
    const int pr = e / (PM + 1), off = e - pr * (PM + 1);
    int r, c;
    if (off <= pr) { r = pr; c = off; } else { r = PM - 1 - pr; c = off - pr - 1; }
    T v;
    const bool vr = s.valid[r], vc = s.valid[c];
    if (r == c) {
      v = vr ? diag : T(1);
    } else if (!vr || !vc) {
      v = T(0);
    } else {
      const T dx = s.ox[r] - s.ox[c], dy = s.oy[r] - s.oy[c];
      const T h = dsqrt<T>(dx * dx + dy * dy);
      T P, G, Qa, L;
      lag_lookup<T>(g, th, lagd, lagf, allint, s.td[r], s.td[c], s.tt[r], s.tt[c], P, G, Qa, L);
      const T x = G * h;
      v = P * matern_M<NU, T>(x, dexp<T>(-x));
    }
    s.K[r][c] = v;
    s.K[c][r] = v;
  }
  __syncwarp();

  // ---- 3. Cholesky, row `lane` in registers
  const int lj = lane < PM ? lane : PM - 1;
  T a[PM];
#pragma unroll
  for (int l = 0; l < PM; ++l) a[l] = s.K[l][lj];
  bool ok = true;
  T dinv = T(1);
#pragma unroll
  for (int k = 0; k < PM; ++k) {
    const T piv = __shfl_sync(kFull, a[k], k);
    ok = ok && (piv > T(0));
    const T rs = drsqrt<T>(piv > T(0) ? piv : T(1));
    if (lane == k) dinv = rs;
    const bool act = (lane >= k) && (lane < PM);
    const T v = act ? a[k] * rs : T(0);
    if (act) a[k] = v;
    if (lane < PM) s.col[lane] = v;
    __syncwarp();
#pragma unroll
    for (int l = k + 1; l < PM; ++l) a[l] = fma(-v, s.col[l], a[l]);
    __syncwarp();
  }

  bool fallback = false;
  if constexpr (MIXED) {
    // condition estimate from the pivots of the used positions
    const float Ljj = (lane < PM && valid) ? 1.0f / dinv : 1.0f;
    float mx = (lane < PM && valid) ? Ljj : 0.0f;
    float mn = (lane < PM && valid) ? Ljj : 3.0e38f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
      mn = fminf(mn, __shfl_xor_sync(kFull, mn, o));
    }
    const float ratio = mx / mn;
    fallback = !ok || !(ratio * ratio <= g.tau);
    if (fallback) {
      if (lane == 0) {
        g.flag[gi] = 1;
        atomicAdd(&g.hdr->n_fallback, 1ull);
      }
      return;
    }
  } else {
    if (!ok) {
      if (lane == 0) report_error(g.hdr, VST_ENOTSPD, gi);
      return;
    }
  }

  // ---- factor rows to shared memory (row-major) for the transposed solves
  T(*Lsm)[PM + 1] = MIXED ? reinterpret_cast<T(*)[PM + 1]>(&s.Ls[0][0]) : s.K;
  __syncwarp();
  if (lane < PM) {
#pragma unroll
    for (int l = 0; l < PM; ++l) Lsm[lane][l] = a[l];
  }
  __syncwarp();
  const T Llast = (T)1 / __shfl_sync(kFull, dinv, LAST);
  const T wj = (lane < LAST) ? Lsm[LAST][lane] : T(0);  // last row: L_N^{-1} k

  // forward solve z = L^{-1} y_local (needed for the NLL of the FP64 form and for b)
  T zj = T(0);
  if ((!MIXED && MODE != kModeFactor) || MODE == kModeNllGrad) {
    T acc = (lane < PM) ? (T)rj : T(0);
#pragma unroll
    for (int k = 0; k < PM; ++k) {
      const T zk = __shfl_sync(kFull, acc * dinv, k);
      if (lane == k) zj = zk;
      if (lane > k) acc = fma(-a[k], zk, acc);
    }
  }

  // backward solves with L_N^T: aj = (L_N^{-T} w)_j, bj = (L_N^{-T} z_N)_j
  const bool need_b = (MODE == kModeNllGrad);
  const bool need_a = MIXED || MODE != kModeNll;
  T aj = T(0), bj = T(0);
  if (need_a) {
    T acc_a = wj, acc_b = (lane < LAST) ? zj : T(0);
#pragma unroll
    for (int k = LAST - 1; k >= 0; --k) {
      const T ak = __shfl_sync(kFull, acc_a * dinv, k);
      T bk = T(0);
      if (need_b) bk = __shfl_sync(kFull, acc_b * dinv, k);
      if (lane == k) { aj = ak; bj = bk; }
      if (lane < k) {
        const T lkj = Lsm[k][lane];
        acc_a = fma(-lkj, ak, acc_a);
        if (need_b) acc_b = fma(-lkj, bk, acc_b);
      }
    }
  }

  // ---- 4. D_i, r_i and the NLL term
  double Dd, rd;      // FP64 values of D_i and r_i
  T Dt, rt;           // the same in T for the adjoint weights
  df a_ref = {0.f, 0.f};  // mixed: refined A_i entry of this lane
  if constexpr (MIXED) {
    // one refinement step: res = k - K_N a (double-float), a += K_N^{-1} res
    if (lane < PM) s.v0[lane] = (lane < LAST) ? aj : 0.0f;
    __syncwarp();
    // The FP32 diagonal is sigma1^2 + nugget rounded once, the same way for
    // every row; the residual and D use the double-float value so that this
    // rounding does not bias every D_i in the same direction.
    const df dg = df_split(th.sigma1sq + th.nugget);
    df res = {(lane < LAST) ? s.K[lj][LAST] : 0.0f, 0.0f};
    if (lane < LAST) {
#pragma unroll
      for (int l = 0; l < LAST; ++l) df_fma_acc(res, -s.K[lane][l], df{s.v0[l], 0.0f});
      if (valid) res.lo = fmaf(-dg.lo, aj, res.lo);
    }
    const float rf = res.hi + res.lo;
    float acc = (lane < LAST) ? rf : 0.0f, dz = 0.0f;
#pragma unroll
    for (int k = 0; k < LAST; ++k) {
      const float zk = __shfl_sync(kFull, acc * dinv, k);
      if (lane == k) dz = zk;
      if (lane > k) acc = fmaf(-a[k], zk, acc);
    }
    float acc2 = (lane < LAST) ? dz : 0.0f, da = 0.0f;
#pragma unroll
    for (int k = LAST - 1; k >= 0; --k) {
      const float dk = __shfl_sync(kFull, acc2 * dinv, k);
      if (lane == k) da = dk;
      if (lane < k) acc2 = fmaf(-Lsm[k][lane], dk, acc2);
    }
    a_ref = (lane < LAST) ? df{aj, da} : df{0.0f, 0.0f};
    // D = K_ii - k . a   and   r = y_i - y_N . a   in double-float
    df Ds = (lane == LAST) ? dg : df{0.0f, 0.0f};
    df rs = (lane == LAST) ? df_split(rj) : df{0.0f, 0.0f};
    if (lane < LAST) {
      df_fma_acc(Ds, -s.K[lane][LAST], a_ref);
      const df yl = df_split(rj);
      df_fma_acc(rs, -yl.hi, a_ref);
      rs.lo = fmaf(-yl.lo, a_ref.hi, rs.lo);
    }
    Ds = df_warp_sum(Ds);
    rs = df_warp_sum(rs);
    Dd = df_to_double(Ds);
    rd = df_to_double(rs);
    Dt = (float)Dd;
    rt = (float)rd;
    if (!(Dd > 0.0) || !(rd == rd)) {  // lost to FP32 rounding: redo in FP64
      if (lane == 0) {
        g.flag[gi] = 1;
        atomicAdd(&g.hdr->n_fallback, 1ull);
      }
      return;
    }
    if (MODE != kModeFactor && lane == 0) {
      const float Df = Ds.hi + Ds.lo, rf2 = rs.hi + rs.lo;
      const float logD = logf(Ds.hi) + Ds.lo / Ds.hi;
      acc_nll += 0.5 * (double)logD + 0.5 * (double)(rf2 * rf2 / Df);
    }
  } else {
    const double Ll = (double)Llast;
    const double zl = __shfl_sync(kFull, (double)zj, LAST);
    Dd = Ll * Ll;
    rd = zl * Ll;
    Dt = (T)Dd;
    rt = (T)rd;
    if (!(Dd > 0.0)) {
      if (lane == 0) report_error(g.hdr, VST_ENOTSPD, gi);
      return;
    }
    if (MODE != kModeFactor && lane == 0) acc_nll += log(Ll) + 0.5 * zl * zl;
  }

  if (MODE == kModeFactor) {
    if (lane < m) {
      double v = 0.0;
      if (lane < cnt) v = MIXED ? df_to_double(a_ref) : (double)aj;
      g.A[gi * m + lane] = v;
    }
    if (lane == 0) g.D[gi] = Dd;
    return;
  }

  // ---- 5. adjoint: sum over pairs of W_pq dSigma~_pq / dtheta
  if (MODE == kModeNllGrad) {
    const T c2 = rt / Dt;
    const T c1 = T(0.5) * (T(1) / Dt - c2 * c2);
    __syncwarp();
    if (lane < PM) {
      const T at = (lane < cnt) ? -aj : (lane == LAST ? T(1) : T(0));
      const T bt = (lane < cnt) ? bj : T(0);
      s.v0[lane] = at;
      s.v1[lane] = bt;
    }
    __syncwarp();
    T g0 = 0, g1 = 0, g2 = 0, g3 = 0, g4 = 0;
    const T inv_s1 = T(1.0 / th.sigma1sq), inv_c = T(1.0 / th.c);
    const T pexp = (T)th.p, hg = (T)(0.5 * th.gamma);
    for (int e = lane; e < NPAIR; e += 32) {
      const int pr = e / (PM + 1), off = e - pr * (PM + 1);
      int r, c;
      if (off <= pr) { r = pr; c = off; } else { r = PM - 1 - pr; c = off - pr - 1; }
      if (!s.valid[r] || !s.valid[c]) continue;
      const T ar = s.v0[r], ac = s.v0[c], br = s.v1[r], bc = s.v1[c];
      T w = c1 * ar * ac - c2 * T(0.5) * (ar * bc + br * ac);
      if (r == c) {
        g0 += w;  // dC(0,0)/dsigma1^2 = 1
        g4 += w;  // nugget
      } else {
        w *= T(2);
        const T dx = s.ox[r] - s.ox[c], dy = s.oy[r] - s.oy[c];
        const T h = dsqrt<T>(dx * dx + dy * dy);
        T P, G, Qa, L;
        lag_lookup<T>(g, th, lagd, lagf, allint, s.td[r], s.td[c], s.tt[r], s.tt[c], P, G, Qa, L);
        const T x = G * h;
        const T E = dexp<T>(-x);
        const T M = matern_M<NU, T>(x, E), xM = matern_xdM<NU, T>(x, E);
        const T wP = w * P;
        g0 = fma(wP * M, inv_s1, g0);
        g1 = fma(wP * xM, inv_c, g1);
        g2 = fma(wP * Qa, -pexp * M - hg * xM, g2);
        g3 = fma(-wP * L, M + T(0.5) * xM, g3);
      }
    }
    acc_g[0] += (double)g0;
    acc_g[1] += (double)g1;
    acc_g[2] += (double)g2;
    acc_g[3] += (double)g3;
    acc_g[4] += (double)g4;
  }
}

template <typename T, int NU, int PM, int MODE, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) rows_kernel(RowArgs g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WarpSm<T, PM>* sm = reinterpret_cast<WarpSm<T, PM>*>(smem_raw);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpSm<T, PM>& s = sm[wib];
  const int64_t warp = (int64_t)blockIdx.x * WARPS + wib;
  const int64_t total = (int64_t)gridDim.x * WARPS;
  double acc_nll = 0.0, acc_g[5] = {0, 0, 0, 0, 0};

  if (g.offsets == nullptr) {
    const int64_t n = g.n;
    bool any = true;
    if (g.fallback_only) any = g.hdr->n_fallback != 0ull;
    if (any) {
      for (int64_t i = warp; i < n; i += total) {
        if (g.fallback_only && g.flag[i] == 0) continue;
        row_body<T, NU, PM, MODE>(g, g.th, g.lagd, g.lagf, s, i, 0, lane, acc_nll, acc_g);
      }
    }
    // fixed-order reduction of this warp's partial sums
    double v[6] = {acc_nll, acc_g[0], acc_g[1], acc_g[2], acc_g[3], acc_g[4]};
#pragma unroll
    for (int q = 0; q < 6; ++q) v[q] = warp_sum(v[q]);
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < 6; ++q) g.partial[warp * 8 + q] = v[q];
    }
  } else {
    // batched form: global rows across datasets, per-row outputs
    const int64_t n = g.offsets[g.nsets];
    int set = 0;
    for (int64_t gi = warp; gi < n; gi += total) {
      if (g.fallback_only && g.flag[gi] == 0) continue;
      while (set + 1 < g.nsets && g.offsets[set + 1] <= gi) ++set;
      const int64_t row0 = g.offsets[set];
      acc_nll = 0.0;
      acc_g[0] = acc_g[1] = acc_g[2] = acc_g[3] = acc_g[4] = 0.0;
      row_body<T, NU, PM, MODE>(g, g.thetas[set], g.lagd_sets + (int64_t)set * kLagTab,
                                g.lagf_sets + (int64_t)set * kLagTab, s, gi - row0, row0, lane, acc_nll,
                                acc_g);
      double v[6] = {acc_nll, acc_g[0], acc_g[1], acc_g[2], acc_g[3], acc_g[4]};
#pragma unroll
      for (int q = 0; q < 6; ++q) v[q] = warp_sum(v[q]);
      if (lane == 0 && !(g.flag != nullptr && !g.fallback_only && g.flag[gi])) {
#pragma unroll
        for (int q = 0; q < 6; ++q) g.row_out[gi * 6 + q] = v[q];
      }
    }
  }
}

}  // namespace vst
