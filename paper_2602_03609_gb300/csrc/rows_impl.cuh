// Fused per-row Vecchia kernel: for each row i (one warp per row),
//   1. gather the |N(i)| <= m neighbours and row i itself (position PM-1),
//   2. evaluate the local (m+1) x (m+1) response covariance Sigma~ (Eq. (2)
//      plus the nugget on the diagonal, Sect. 3.1),
//   3. Cholesky-factor it with row j of the factor held in lane j's registers,
//   4. solve for A_i = Sigma~_{i,N} Sigma~_N^{-1} and D_i (Sect. 4.1) and the
//      whitened residual, giving the NLL term 1/2 log D_i + 1/2 r_i^2 / D_i,
//   5. (gradient) contract the adjoint weights dNLL_i/dSigma~ with the
//      covariance derivatives dSigma~/dtheta, pair by pair.
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
// iterative refinement whose residual k - K_N A_i is accumulated in
// double-float arithmetic; D_i and r_i are formed in double-float; per-warp
// sums over rows are double-float, combined in FP64 at the end.  The FP64
// pipe of this part runs at 1/64 of the FP32 rate, so the mixed form has no
// FP64 arithmetic per row: coordinates, response and day come from per-point
// records written once per call (PrepPt).  Rows whose Cholesky fails in FP32,
// whose D_i is not positive, or whose condition estimate
// (max_j L_jj / min_j L_jj)^2 exceeds tau are flagged and redone by the FP64
// instantiation.
#pragma once

#include <climits>
#include <type_traits>

#include "common.cuh"
#include "dfmath.cuh"

namespace vst {

// kModeVifAdj: the VIF gradient's pass over the residual blocks (FP64, or mixed),
// with the per-row adjoints of A_i and D_i given (abar, dbar)
enum RowMode { kModeNll = 0, kModeNllGrad = 1, kModeFactor = 2, kModeVifAdj = 3 };

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
  int row_chunk;              // consecutive rows per warp assignment (>= 1)
  int blocks_per_sm;          // launch shape: resident blocks per SM (0 = as many as fit)
  // VIF: per-row Gram U_p . U_q of the local block (packed pair order),
  // subtracted from the covariance; at most one of the two is set
  const double* gram_d;
  const float* gram_f;
  // VIF, mixed form: per integer lag, the amplitude P and scale G of Eq. (2)
  // as double-floats {P_hi, P_lo, G_hi, G_lo}
  const float4* lagdf;
  // mixed form: per-point records (row0-relative like xy, t, y); required
  const PrepPt* prep;
  // kModeVifAdj: adjoints dNLL/dA_i [n][m] and dNLL/dD_i [n]; out:
  // b~_i = K_N^{-1} Abar_i [n][m] (0 beyond nn_cnt[i])
  const double* abar;
  const double* dbar;
  double* btil;
  // single-dataset form: rows out0..n-1 are processed and their per-row
  // arrays (nn, nn_cnt, flag, A, D) hold row i at index i - out0 (0: all rows)
  int64_t out0;
};

// Per-position record of the local block: offsets from row i, integer day
// (valid when all times of the block are integers), used flag.
template <typename T> struct alignas(16) Pos { T ox, oy; int td, valid; };

template <typename T, int PM>
struct WarpSm {
  static constexpr int KS = PM + 16 / (int)sizeof(T);   // row stride: rows 16-byte aligned
  static constexpr int NPAIR = PM * (PM + 1) / 2;
  static constexpr bool MIXED = std::is_same<T, float>::value;
  alignas(16) T K[PM][KS];                          // local covariance (FP64: reused for L)
  alignas(16) T Ls[MIXED ? PM : 1][KS];             // mixed: factor L
  alignas(16) T col[PM];                            // column broadcast during Cholesky
  alignas(16) T v0[PM];                             // a (refinement)
  alignas(16) T ab[PM][2];                          // (a~, b~) per position (adjoint)
  alignas(16) Pos<T> pos[PM];
  alignas(16) float q1[MIXED ? NPAIR : 1];          // mixed: P x M'(x) per pair
  alignas(16) double xe[MIXED ? 1 : NPAIR][2];      // FP64: (x, e^-x) per pair
  // tiled pair loops: P x M'(x) of the diagonal-block pairs (FP64: then their
  // covariance, the FP64 factor overwrites K)
  alignas(16) T qd[(MIXED ? 2 : 4) * PM];
  double tt[PM];                                    // times (non-integer lag path)
};

// Block-wide tables shared by the warps: the off-diagonal position pairs
// (r, c) a local block can use, as r | c << 8 | e << 16 with e the packed
// lower-triangle index (positions 0..m-1 and the row's own position PM-1;
// positions m..PM-2 are padding for every row and never enter the pair
// loops), and the first kLagSmem lags of the lag table.
constexpr int kLagSmem = 128;
template <typename T, int PM>
struct BlockSm {
  uint32_t pairs[PM * (PM + 1) / 2];
  int npairs;
  // tiled pair loops: the pairs r > c inside the 8 diagonal blocks of size
  // PM / 8 (as r | c << 8 | q << 16, q = the slot of their P x M'(x))
  uint32_t dpairs[2 * PM];
  int ndpairs;
  alignas(16) typename std::conditional<std::is_same<T, float>::value, LagF, LagD>::type lag[kLagSmem];
};

// Per-lane accumulators of the NLL and gradient sums over the rows a warp
// processes: FP64 for the FP64 form, double-float for the mixed form.
template <typename T> struct RowAcc;
template <> struct RowAcc<double> {
  double v[6];
  __device__ void zero() {
#pragma unroll
    for (int q = 0; q < 6; ++q) v[q] = 0.0;
  }
  __device__ void add(int q, double x) { v[q] += x; }
  __device__ double get(int q) const { return v[q]; }
};
template <> struct RowAcc<float> {
  df v[6];
  __device__ void zero() {
#pragma unroll
    for (int q = 0; q < 6; ++q) v[q] = df{0.f, 0.f};
  }
  __device__ void add(int q, float x) {
    const df t = df_two_sum(v[q].hi, x);
    v[q].hi = t.hi;
    v[q].lo += t.lo;
  }
  __device__ double get(int q) const { return df_to_double(v[q]); }
};

template <typename T, typename LagS>
__device__ __forceinline__ void lag_lookup(const DevTheta& th, const LagD* lagd, const LagF* lagf,
                                           const LagS* lags, bool allint, int tdr, int tdc, double ttr,
                                           double ttc, T& P, T& G, T& Qa, T& L) {
  const int lag = abs(tdr - tdc);
  if (allint && lag < kLagSmem && lags != nullptr) {
    if constexpr (std::is_same<T, float>::value) {
      const float4 f = *reinterpret_cast<const float4*>(&lags[lag]);
      P = f.x; G = f.y; Qa = f.z; L = f.w;
    } else {
      const double2 a = reinterpret_cast<const double2*>(&lags[lag])[0];
      const double2 b = reinterpret_cast<const double2*>(&lags[lag])[1];
      P = a.x; G = a.y; Qa = b.x; L = b.y;
    }
  } else if (allint && lag < kLagTab) {
    if constexpr (std::is_same<T, float>::value) {
      const float4 f = __ldg(reinterpret_cast<const float4*>(lagf) + lag);
      P = f.x; G = f.y; Qa = f.z; L = f.w;
    } else {
      const double2 a = __ldg(reinterpret_cast<const double2*>(lagd) + 2 * lag);
      const double2 b = __ldg(reinterpret_cast<const double2*>(lagd) + 2 * lag + 1);
      P = a.x; G = a.y; Qa = b.x; L = b.y;
    }
  } else {
    // integer days beyond the table: the lag itself (exact); the mixed form
    // stores the times of a block only when some are not integer days
    const LagD f = lag_factors(th, allint ? (double)lag : ttr - ttc);
    P = (T)f.P; G = (T)f.G; Qa = (T)f.Qa; L = (T)f.L;
  }
}

template <int PM>
__device__ __forceinline__ void pair_of(int e, int& r, int& c) {
  const int pr = e / (PM + 1), off = e - pr * (PM + 1);
  if (off <= pr) { r = pr; c = off; } else { r = PM - 1 - pr; c = off - pr - 1; }
}
// packed index of the pair (r, c), r >= c (the inverse of pair_of)
template <int PM>
__device__ __forceinline__ int pair_e(int r, int c) {
  if (r < PM / 2) return r * (PM + 1) + c;
  const int pr = PM - 1 - r;
  return pr * (PM + 1) + pr + 1 + c;
}

// 16-byte vector load / store of 16 / sizeof(T) consecutive shared elements
template <typename T, int VEC>
__device__ __forceinline__ void ld16(T (&v)[VEC], const T* p) {
  if constexpr (std::is_same<T, float>::value) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
    const double2 q = *reinterpret_cast<const double2*>(p);
    v[0] = q.x; v[1] = q.y;
  }
}
template <typename T, int VEC>
__device__ __forceinline__ void st16(T* p, const T (&v)[VEC]) {
  if constexpr (std::is_same<T, float>::value) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
}

// ---------------------------------------------------------------------------
// Tiled pair loops of the NLL and plain-gradient instantiations.  The strict
// lower triangle of the PM x PM block is cut into 8 x 8 blocks of TS = PM / 8
// positions.  Lane l < 28 owns the off-diagonal block (R, C), R > C,
// l = R (R - 1) / 2 + C: it holds the TS + TS positions in registers,
// evaluates the TS x TS pairs without any table decode or validity branch
// (a pair with an unused position gets 0) and stores row and column vectors
// of K.  Its TS^2 values P x M'(x) (FP64: and the covariance) stay in the
// warp's scratch at [u][lane] for the adjoint pass, which reads them back in
// the same order.  The pairs inside the 8 diagonal blocks (TS (TS - 1) / 2
// each) go through a small table, at most two per lane.
template <int PM> struct TileShape {
  static constexpr int TS = PM / 8;
  static constexpr int NT = TS * TS;       // pairs per off-diagonal block
  static constexpr int ND = 8 * TS * (TS - 1) / 2;  // diagonal-block pairs
};

__device__ __forceinline__ void tile_of_lane(int lane, int& R, int& C) {
  int r = 1;
  while ((r + 1) * r / 2 <= lane) ++r;
  R = r;
  C = lane - r * (r - 1) / 2;
}

// TS consecutive elements, vectorised where the width allows
template <typename T, int TS>
__device__ __forceinline__ void st_row(T* p, const T (&v)[TS]) {
  if constexpr (sizeof(T) * TS == 16) {
    st16<T, 16 / (int)sizeof(T)>(p, v);
  } else if constexpr (sizeof(T) * TS == 32) {
    T a[TS / 2], b[TS / 2];
#pragma unroll
    for (int u = 0; u < TS / 2; ++u) { a[u] = v[u]; b[u] = v[u + TS / 2]; }
    st16<T, TS / 2>(p, a);
    st16<T, TS / 2>(p + TS / 2, b);
  } else if constexpr (std::is_same<T, float>::value && TS == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else {
#pragma unroll
    for (int u = 0; u < TS; ++u) p[u] = v[u];
  }
}
template <typename T, int TS>
__device__ __forceinline__ void ld_row(T (&v)[TS], const T* p) {
  if constexpr (sizeof(T) * TS == 16) {
    ld16<T, 16 / (int)sizeof(T)>(v, p);
  } else if constexpr (sizeof(T) * TS == 32) {
    T a[TS / 2], b[TS / 2];
    ld16<T, TS / 2>(a, p);
    ld16<T, TS / 2>(b, p + TS / 2);
#pragma unroll
    for (int u = 0; u < TS / 2; ++u) { v[u] = a[u]; v[u + TS / 2] = b[u]; }
  } else if constexpr (std::is_same<T, float>::value && TS == 2) {
    const float2 q = *reinterpret_cast<const float2*>(p);
    v[0] = q.x;
    v[1] = q.y;
  } else {
#pragma unroll
    for (int u = 0; u < TS; ++u) v[u] = p[u];
  }
}

// covariance and P x M'(x) of one pair (mixed: FP32 with the exp2 unit; FP64)
template <typename T, int NU>
__device__ __forceinline__ void pair_cov(T dx, T dy, T P, T G, T& v, T& q) {
  const T d2 = dx * dx + dy * dy;
  if constexpr (std::is_same<T, float>::value) {
    const float h = d2 >= kFltMinNormal ? d2 * rsqrt_ftz(d2) : 0.f;
    const float x = G * h;
    const float E = __expf(-x);
    v = P * matern_M<NU, float>(x, E);
    q = P * matern_xdM<NU, float>(x, E);
  } else {
    const double x = G * sqrt(d2);
    const double E = exp(-x);
    v = P * matern_M<NU, double>(x, E);
    q = P * matern_xdM<NU, double>(x, E);
  }
}

// covariance and P x M'(x) of two pairs at once on packed FP32 pairs (mixed
// form, per-pair lag factors and distances as float2); Pm is P already
// multiplied by the pairs' validity (0 or 1)
template <int NU>
__device__ __forceinline__ void pair_cov2(float2 dx, float2 dy, float2 Pm, float2 G, float2& v, float2& q) {
  const float2 d2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
  const float2 hh = __fmul2_rn(d2, make_float2(rsqrt_ftz(d2.x), rsqrt_ftz(d2.y)));
  const float2 h = make_float2(d2.x >= kFltMinNormal ? hh.x : 0.f, d2.y >= kFltMinNormal ? hh.y : 0.f);
  const float2 x = __fmul2_rn(G, h);
  const float2 E = make_float2(__expf(-x.x), __expf(-x.y));
  float2 M, xdM;
  if constexpr (NU == 0) {
    M = E;
    xdM = __fmul2_rn(x, make_float2(-E.x, -E.y));
  } else if constexpr (NU == 1) {
    M = __ffma2_rn(x, E, E);  // (1 + x) e^-x
    xdM = __fmul2_rn(__fmul2_rn(x, x), make_float2(-E.x, -E.y));
  } else {
    const float2 x23 = __fmul2_rn(__fmul2_rn(x, x), make_float2(1.0f / 3.0f, 1.0f / 3.0f));
    M = __fmul2_rn(__fadd2_rn(__fadd2_rn(make_float2(1.0f, 1.0f), x), x23), E);
    xdM = __fmul2_rn(__fmul2_rn(x23, __fadd2_rn(make_float2(1.0f, 1.0f), x)), make_float2(-E.x, -E.y));
  }
  v = __fmul2_rn(Pm, M);
  q = __fmul2_rn(Pm, xdM);
}

// lag factors of a pair: from the row's table when FAST (all times integer
// days and every lag of the block inside the table), else the general lookup
template <typename T, bool FAST, typename LagS>
__device__ __forceinline__ void pair_lag(const DevTheta& th, const LagD* lagd, const LagF* lagf, const LagS* tab,
                                         bool allint, int tdr, int tdc, double ttr, double ttc, T& P, T& G, T& Qa,
                                         T& L) {
  if constexpr (FAST) {
    const LagS f = tab[abs(tdr - tdc)];
    P = (T)f.P; G = (T)f.G; Qa = (T)f.Qa; L = (T)f.L;
  } else {
    lag_lookup<T>(th, lagd, lagf, tab, allint, tdr, tdc, ttr, ttc, P, G, Qa, L);
  }
}

template <typename T, int NU, int PM, bool FAST, typename LagS>
__device__ __forceinline__ void cov_tiled(const DevTheta& th, const LagD* lagd, const LagF* lagf, const LagS* tab,
                                          bool allint, const BlockSm<T, PM>* bs, WarpSm<T, PM>& s, int tR, int tC,
                                          int lane) {
  constexpr int TS = TileShape<PM>::TS;
  constexpr bool MIXED = std::is_same<T, float>::value;
  T* qt = MIXED ? reinterpret_cast<T*>(&s.q1[0]) : reinterpret_cast<T*>(&s.xe[0][0]);
  if constexpr (MIXED && TS % 2 == 0) {
    // the tile's column pairs (b, b + 1) on packed FP32 pairs; invalid
    // positions enter as a zero factor on P.  The lag factors come from the
    // row's table or the general lookup; the arithmetic is the same either
    // way, so a dataset gives the same bits in single and batched calls.
    constexpr int TH = TS / 2;
    if (lane < 28) {
      float2 ncx[TH], ncy[TH], cmask[TH];
      int ctd[TS];
#pragma unroll
      for (int u = 0; u < TH; ++u) {
        const Pos<T> p0 = s.pos[tC * TS + 2 * u], p1 = s.pos[tC * TS + 2 * u + 1];
        ncx[u] = make_float2(-p0.ox, -p1.ox);
        ncy[u] = make_float2(-p0.oy, -p1.oy);
        cmask[u] = make_float2(p0.valid ? 1.0f : 0.0f, p1.valid ? 1.0f : 0.0f);
        ctd[2 * u] = p0.td;
        ctd[2 * u + 1] = p1.td;
      }
      T kv[TS][TS];
#pragma unroll
      for (int a = 0; a < TS; ++a) {
        const Pos<T> pr = s.pos[tR * TS + a];
        const float rm = pr.valid ? 1.0f : 0.0f;
        const float2 rx = make_float2(pr.ox, pr.ox), ry = make_float2(pr.oy, pr.oy), rmm = make_float2(rm, rm);
#pragma unroll
        for (int u = 0; u < TH; ++u) {
          T P0, G0, Qa0, L0, P1, G1, Qa1, L1;
          pair_lag<T, FAST>(th, lagd, lagf, tab, allint, pr.td, ctd[2 * u], s.tt[tR * TS + a], s.tt[tC * TS + 2 * u], P0,
                            G0, Qa0, L0);
          pair_lag<T, FAST>(th, lagd, lagf, tab, allint, pr.td, ctd[2 * u + 1], s.tt[tR * TS + a],
                            s.tt[tC * TS + 2 * u + 1], P1, G1, Qa1, L1);
          const float2 Pm = __fmul2_rn(make_float2(P0, P1), __fmul2_rn(rmm, cmask[u]));
          float2 v, q;
          pair_cov2<NU>(__fadd2_rn(rx, ncx[u]), __fadd2_rn(ry, ncy[u]), Pm, make_float2(G0, G1), v, q);
          kv[a][2 * u] = v.x;
          kv[a][2 * u + 1] = v.y;
          qt[(a * TS + 2 * u) * 32 + lane] = q.x;
          qt[(a * TS + 2 * u + 1) * 32 + lane] = q.y;
        }
      }
#pragma unroll
      for (int a = 0; a < TS; ++a) st_row<T, TS>(&s.K[tR * TS + a][tC * TS], kv[a]);
#pragma unroll
      for (int b = 0; b < TS; ++b) {
        T col[TS];
#pragma unroll
        for (int a = 0; a < TS; ++a) col[a] = kv[a][b];
        st_row<T, TS>(&s.K[tC * TS + b][tR * TS], col);
      }
    }
  } else if (lane < 28) {
    Pos<T> pc[TS];
#pragma unroll
    for (int u = 0; u < TS; ++u) pc[u] = s.pos[tC * TS + u];
    T kv[TS][TS];
#pragma unroll
    for (int a = 0; a < TS; ++a) {
      const Pos<T> pr = s.pos[tR * TS + a];
#pragma unroll
      for (int b = 0; b < TS; ++b) {
        T P, G, Qa, L, v, q;
        pair_lag<T, FAST>(th, lagd, lagf, tab, allint, pr.td, pc[b].td, s.tt[tR * TS + a], s.tt[tC * TS + b], P, G,
                          Qa, L);
        pair_cov<T, NU>(pr.ox - pc[b].ox, pr.oy - pc[b].oy, P, G, v, q);
        const bool ok = (pr.valid & pc[b].valid) != 0;
        kv[a][b] = ok ? v : T(0);
        qt[(a * TS + b) * 32 + lane] = ok ? q : T(0);
        if constexpr (!MIXED) qt[(TS * TS + a * TS + b) * 32 + lane] = kv[a][b];
      }
    }
#pragma unroll
    for (int a = 0; a < TS; ++a) st_row<T, TS>(&s.K[tR * TS + a][tC * TS], kv[a]);
#pragma unroll
    for (int b = 0; b < TS; ++b) {
      T col[TS];
#pragma unroll
      for (int a = 0; a < TS; ++a) col[a] = kv[a][b];
      st_row<T, TS>(&s.K[tC * TS + b][tR * TS], col);
    }
  }
  if constexpr (MIXED && TS % 2 == 0) {
    // the diagonal-block pairs two per lane (their count 8 TS (TS - 1) / 2 is even)
    const int q0 = 2 * lane;
    if (q0 < bs->ndpairs) {
      const uint32_t rc0 = bs->dpairs[q0], rc1 = bs->dpairs[q0 + 1];
      const int pr_0 = rc0 & 0xff, pc_0 = (rc0 >> 8) & 0xff, pr_1 = rc1 & 0xff, pc_1 = (rc1 >> 8) & 0xff;
      const Pos<T> pr0 = s.pos[pr_0], pc0 = s.pos[pc_0], pr1 = s.pos[pr_1], pc1 = s.pos[pc_1];
      T P0, G0, Qa0, L0, P1, G1, Qa1, L1;
      pair_lag<T, FAST>(th, lagd, lagf, tab, allint, pr0.td, pc0.td, s.tt[pr_0], s.tt[pc_0], P0, G0, Qa0, L0);
      pair_lag<T, FAST>(th, lagd, lagf, tab, allint, pr1.td, pc1.td, s.tt[pr_1], s.tt[pc_1], P1, G1, Qa1, L1);
      const float2 Pm = make_float2((pr0.valid & pc0.valid) ? P0 : 0.0f, (pr1.valid & pc1.valid) ? P1 : 0.0f);
      float2 v, q;
      pair_cov2<NU>(make_float2(pr0.ox - pc0.ox, pr1.ox - pc1.ox), make_float2(pr0.oy - pc0.oy, pr1.oy - pc1.oy), Pm,
                    make_float2(G0, G1), v, q);
      s.K[pr_0][pc_0] = v.x;
      s.K[pc_0][pr_0] = v.x;
      s.K[pr_1][pc_1] = v.y;
      s.K[pc_1][pr_1] = v.y;
      *reinterpret_cast<float2*>(&s.qd[q0]) = q;
    }
  } else {
    for (int q = lane; q < bs->ndpairs; q += 32) {
      const uint32_t rc = bs->dpairs[q];
      const int r = rc & 0xff, c = (rc >> 8) & 0xff;
      const Pos<T> pr = s.pos[r], pc = s.pos[c];
      T P, G, Qa, L, v, qq;
      pair_lag<T, FAST>(th, lagd, lagf, tab, allint, pr.td, pc.td, s.tt[r], s.tt[c], P, G, Qa, L);
      pair_cov<T, NU>(pr.ox - pc.ox, pr.oy - pc.oy, P, G, v, qq);
      const bool ok = (pr.valid & pc.valid) != 0;
      v = ok ? v : T(0);
      s.K[r][c] = v;
      s.K[c][r] = v;
      s.qd[q] = ok ? qq : T(0);
      if constexpr (!MIXED) s.qd[2 * PM + q] = v;
    }
  }
}

// sum over the pairs of W_pq dSigma~_pq / dtheta, W = c1 a~ a~^T - c2 (a~ b~^T
// + b~ a~^T) / 2, for the off-diagonal pairs (the caller adds the diagonal)
template <typename T, int NU, int PM, bool FAST, typename LagS>
__device__ __forceinline__ void adj_tiled(const DevTheta& th, const LagD* lagd, const LagF* lagf, const LagS* tab,
                                          bool allint, const BlockSm<T, PM>* bs, WarpSm<T, PM>& s, int tR, int tC,
                                          int lane, T c1, T hc2, T pexp, T hg, T& g0, T& g1, T& g2, T& g3) {
  constexpr int TS = TileShape<PM>::TS;
  constexpr bool MIXED = std::is_same<T, float>::value;
  const T* qt = MIXED ? reinterpret_cast<const T*>(&s.q1[0]) : reinterpret_cast<const T*>(&s.xe[0][0]);
  if constexpr (MIXED && TS % 2 == 0) {
    // column pairs (b, b + 1) on packed FP32 pairs, even and odd columns in
    // separate partial sums; g2 and g3 accumulate with the sign taken out
    constexpr int TH = TS / 2;
    if (lane < 28) {
      float2 ac2[TH], bc2[TH];
      int tc[TS];
#pragma unroll
      for (int u = 0; u < TH; ++u) {
        ac2[u] = make_float2(s.ab[tC * TS + 2 * u][0], s.ab[tC * TS + 2 * u + 1][0]);
        bc2[u] = make_float2(s.ab[tC * TS + 2 * u][1], s.ab[tC * TS + 2 * u + 1][1]);
        tc[2 * u] = s.pos[tC * TS + 2 * u].td;
        tc[2 * u + 1] = s.pos[tC * TS + 2 * u + 1].td;
      }
      const float2 pe2 = make_float2(pexp, pexp), hg2 = make_float2(hg, hg), half2 = make_float2(0.5f, 0.5f);
      float2 G0 = make_float2(0.f, 0.f), G1 = G0, G2 = G0, G3 = G0;
#pragma unroll
      for (int a = 0; a < TS; ++a) {
        const T ara = s.ab[tR * TS + a][0], bra = s.ab[tR * TS + a][1];
        const int tra = s.pos[tR * TS + a].td;
        T kv[TS];
        ld_row<T, TS>(kv, &s.K[tR * TS + a][tC * TS]);
        const T ra = c1 * ara - hc2 * bra, rb = -hc2 * ara;
        const float2 ra2 = make_float2(ra, ra), rb2 = make_float2(rb, rb);
#pragma unroll
        for (int u = 0; u < TH; ++u) {
          T P0, G0_, Qa0, L0, P1, G1_, Qa1, L1;
          pair_lag<T, FAST>(th, lagd, lagf, tab, allint, tra, tc[2 * u], s.tt[tR * TS + a], s.tt[tC * TS + 2 * u], P0,
                            G0_, Qa0, L0);
          pair_lag<T, FAST>(th, lagd, lagf, tab, allint, tra, tc[2 * u + 1], s.tt[tR * TS + a],
                            s.tt[tC * TS + 2 * u + 1], P1, G1_, Qa1, L1);
          const float2 Kv = make_float2(kv[2 * u], kv[2 * u + 1]);
          const float2 Xv = make_float2(qt[(a * TS + 2 * u) * 32 + lane], qt[(a * TS + 2 * u + 1) * 32 + lane]);
          const float2 w = __ffma2_rn(ra2, ac2[u], __fmul2_rn(rb2, bc2[u]));
          const float2 w2 = __fadd2_rn(w, w);  // both (r, c) and (c, r)
          G0 = __ffma2_rn(w2, Kv, G0);
          G1 = __ffma2_rn(w2, Xv, G1);
          G2 = __ffma2_rn(__fmul2_rn(w2, make_float2(Qa0, Qa1)), __ffma2_rn(pe2, Kv, __fmul2_rn(hg2, Xv)), G2);
          G3 = __ffma2_rn(__fmul2_rn(w2, make_float2(L0, L1)), __ffma2_rn(half2, Xv, Kv), G3);
        }
      }
      g0 += G0.x + G0.y;
      g1 += G1.x + G1.y;
      g2 -= G2.x + G2.y;
      g3 -= G3.x + G3.y;
    }
  } else if (lane < 28) {
    T ac[TS], bc[TS];
    int tc[TS];
#pragma unroll
    for (int u = 0; u < TS; ++u) {
      ac[u] = s.ab[tC * TS + u][0];
      bc[u] = s.ab[tC * TS + u][1];
      tc[u] = s.pos[tC * TS + u].td;
    }
#pragma unroll
    for (int a = 0; a < TS; ++a) {
      const T ara = s.ab[tR * TS + a][0], bra = s.ab[tR * TS + a][1];
      const int tra = s.pos[tR * TS + a].td;
      T kv[TS];
      if constexpr (MIXED) {
        ld_row<T, TS>(kv, &s.K[tR * TS + a][tC * TS]);
      } else {
#pragma unroll
        for (int b = 0; b < TS; ++b) kv[b] = qt[(TS * TS + a * TS + b) * 32 + lane];
      }
      const T ra = c1 * ara - hc2 * bra, rb = -hc2 * ara;
#pragma unroll
      for (int b = 0; b < TS; ++b) {
        T P, G, Qa, L;
        pair_lag<T, FAST>(th, lagd, lagf, tab, allint, tra, tc[b], s.tt[tR * TS + a], s.tt[tC * TS + b], P, G, Qa,
                          L);
        const T Kv = kv[b], Xv = qt[(a * TS + b) * 32 + lane];
        // w = ar (c1 ac - hc2 bc) - hc2 br ac, doubled (both (r, c) and (c, r))
        const T w2 = T(2) * fma(ra, ac[b], rb * bc[b]);
        g0 = fma(w2, Kv, g0);
        g1 = fma(w2, Xv, g1);
        g2 = fma(w2 * Qa, -pexp * Kv - hg * Xv, g2);
        g3 = fma(-w2 * L, Kv + T(0.5) * Xv, g3);
      }
    }
  }
  if constexpr (MIXED && TS % 2 == 0) {
    // the diagonal-block pairs two per lane, as in cov_tiled
    const int q0 = 2 * lane;
    if (q0 < bs->ndpairs) {
      const uint32_t rc0 = bs->dpairs[q0], rc1 = bs->dpairs[q0 + 1];
      const int pr_0 = rc0 & 0xff, pc_0 = (rc0 >> 8) & 0xff, pr_1 = rc1 & 0xff, pc_1 = (rc1 >> 8) & 0xff;
      T P0, G0_, Qa0, L0, P1, G1_, Qa1, L1;
      pair_lag<T, FAST>(th, lagd, lagf, tab, allint, s.pos[pr_0].td, s.pos[pc_0].td, s.tt[pr_0], s.tt[pc_0], P0, G0_,
                        Qa0, L0);
      pair_lag<T, FAST>(th, lagd, lagf, tab, allint, s.pos[pr_1].td, s.pos[pc_1].td, s.tt[pr_1], s.tt[pc_1], P1, G1_,
                        Qa1, L1);
      const float2 ar = make_float2(s.ab[pr_0][0], s.ab[pr_1][0]), br = make_float2(s.ab[pr_0][1], s.ab[pr_1][1]);
      const float2 ac = make_float2(s.ab[pc_0][0], s.ab[pc_1][0]), bc = make_float2(s.ab[pc_0][1], s.ab[pc_1][1]);
      const float2 Kv = make_float2(s.K[pr_0][pc_0], s.K[pr_1][pc_1]);
      const float2 Xv = *reinterpret_cast<const float2*>(&s.qd[q0]);
      // w = ar (c1 ac - hc2 bc) - hc2 br ac, doubled
      const float2 t = __ffma2_rn(make_float2(c1, c1), ac, __fmul2_rn(make_float2(-hc2, -hc2), bc));
      const float2 w = __ffma2_rn(ar, t, __fmul2_rn(__fmul2_rn(make_float2(-hc2, -hc2), br), ac));
      const float2 w2 = __fadd2_rn(w, w);
      const float2 G0 = __fmul2_rn(w2, Kv), G1 = __fmul2_rn(w2, Xv);
      const float2 G2 = __fmul2_rn(__fmul2_rn(w2, make_float2(Qa0, Qa1)),
                                   __ffma2_rn(make_float2(pexp, pexp), Kv, __fmul2_rn(make_float2(hg, hg), Xv)));
      const float2 G3 = __fmul2_rn(__fmul2_rn(w2, make_float2(L0, L1)), __ffma2_rn(make_float2(0.5f, 0.5f), Xv, Kv));
      g0 += G0.x + G0.y;
      g1 += G1.x + G1.y;
      g2 -= G2.x + G2.y;
      g3 -= G3.x + G3.y;
    }
  } else {
    for (int q = lane; q < bs->ndpairs; q += 32) {
      const uint32_t rc = bs->dpairs[q];
      const int r = rc & 0xff, c = (rc >> 8) & 0xff;
      T P, G, Qa, L;
      pair_lag<T, FAST>(th, lagd, lagf, tab, allint, s.pos[r].td, s.pos[c].td, s.tt[r], s.tt[c], P, G, Qa, L);
      const T ar = s.ab[r][0], br = s.ab[r][1], ac = s.ab[c][0], bc = s.ab[c][1];
      const T Kv = MIXED ? s.K[r][c] : s.qd[2 * PM + q], Xv = s.qd[q];
      const T w2 = T(2) * (ar * (c1 * ac - hc2 * bc) - hc2 * br * ac);
      g0 = fma(w2, Kv, g0);
      g1 = fma(w2, Xv, g1);
      g2 = fma(w2 * Qa, -pexp * Kv - hg * Xv, g2);
      g3 = fma(-w2 * L, Kv + T(0.5) * Xv, g3);
    }
  }
}

// Process one row; all 32 lanes call it together.
template <typename T, int NU, int PM, int MODE>
__device__ __forceinline__ void row_body(const RowArgs& g, const DevTheta& th, const LagD* lagd,
                                         const LagF* lagf, const BlockSm<T, PM>* bs, bool lag_smem,
                                         WarpSm<T, PM>& s, int64_t i, int64_t row0, int lane,
                                         RowAcc<T>& acc, int tR, int tC) {
  // the NLL and plain-gradient instantiations use the tiled pair loops
  constexpr bool TILED = (MODE == kModeNll || MODE == kModeNllGrad);
  constexpr bool MIXED = std::is_same<T, float>::value;
  constexpr int LAST = PM - 1;
  constexpr int VEC = 16 / (int)sizeof(T);
  constexpr int NPAIR = WarpSm<T, PM>::NPAIR;
  const int m = g.m;
  const int64_t gi = row0 + i;  // global row (batched form); nn indices are local
  const int64_t ri = gi - g.out0;  // index into the per-row arrays
  const int cnt = g.nn_cnt[ri];
  if (cnt < 0 || cnt > m || cnt > LAST || (int64_t)cnt > i) {
    if (lane == 0) report_error(g.hdr, VST_EINVAL, gi);
    return;
  }
  int idx = -1;
  bool bad = false;
  if (lane < cnt) {
    idx = g.nn[ri * m + lane];
    bad = (idx < 0) || ((int64_t)idx >= i);
  }
  if (__any_sync(kFull, bad)) {
    if (lane == 0) report_error(g.hdr, VST_EINVAL, gi);
    return;
  }
  if (lane == LAST) idx = (int)i;
  const bool valid = idx >= 0;
  bool allint;
  double rj = 0.0;         // FP64 form: y at this position (0 if unused)
  df yl = {0.0f, 0.0f};    // mixed form: the same as a double-float
  if constexpr (MIXED) {
    // per-point records: FP32 offsets from double-float coordinates; unused
    // positions read row i's record (zero offsets, its day)
    const PrepPt* pp = g.prep + row0;
    const int64_t src = valid ? (int64_t)idx : i;
    const float4 ci = __ldg(reinterpret_cast<const float4*>(pp + i));
    const float4 cj = __ldg(reinterpret_cast<const float4*>(pp + src));
    const float4 qj = __ldg(reinterpret_cast<const float4*>(pp + src) + 1);
    const int tdj = __float_as_int(qj.z);
    allint = __all_sync(kFull, __float_as_int(qj.w) != 0);
    if (MODE == kModeVifAdj) yl = (lane < cnt) ? df_split(g.abar[ri * m + lane]) : df{0.0f, 0.0f};
    else if (MODE != kModeFactor && valid) yl = df{qj.x, qj.y};
    if (lane < PM) {
      Pos<T> p;
      p.ox = df_diff(cj.x, cj.y, ci.x, ci.y);
      p.oy = df_diff(cj.z, cj.w, ci.z, ci.w);
      p.td = allint ? tdj : 0;
      p.valid = valid;
      s.pos[lane] = p;
      if (!allint) s.tt[lane] = g.t[row0 + src];
    }
  } else {
    const double* xy = g.xy + 2 * row0;
    const double* tv = g.t + row0;
    const double xi = xy[2 * i], yi = xy[2 * i + 1];
    double xj = xi, yj = yi, tj = tv[i];
    if (valid) {
      xj = xy[2 * (int64_t)idx];
      yj = xy[2 * (int64_t)idx + 1];
      tj = tv[idx];
      if (MODE == kModeVifAdj) rj = (lane < cnt) ? g.abar[ri * m + lane] : 0.0;
      else if (MODE != kModeFactor) rj = g.y[row0 + idx];
    }
    const bool tint = (tj == floor(tj)) && fabs(tj) < 1.0e9;
    allint = __all_sync(kFull, tint);
    if (lane < PM) {
      Pos<T> p;
      p.ox = (T)(xj - xi);
      p.oy = (T)(yj - yi);
      p.td = allint ? (int)tj : 0;
      p.valid = valid;
      s.pos[lane] = p;
      s.tt[lane] = tj;
    }
  }
  const T yv = MIXED ? (T)yl.hi : (T)rj;  // y in T (solves)
  // tiled loops: every lag of the block inside the shared lag table
  bool fast = false;
  if constexpr (TILED) {
    const int td = s.pos[lane < PM ? lane : 0].td;  // this lane's own record (written above)
    int tmx = (lane < PM && valid) ? td : INT_MIN, tmn = (lane < PM && valid) ? td : INT_MAX;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      tmx = max(tmx, __shfl_xor_sync(kFull, tmx, o));
      tmn = min(tmn, __shfl_xor_sync(kFull, tmn, o));
    }
    fast = lag_smem && allint && (int64_t)tmx - (int64_t)tmn < kLagSmem;
  }
  __syncwarp();

  // ---- 2. local covariance, lower triangle distributed over the lanes
  const T diag = MIXED ? (T)th.dg_hi : (T)(th.sigma1sq + th.nugget);
  // a Gram (VIF) is only ever passed to the factor mode; the NLL and
  // gradient instantiations compile without the VIF code
  constexpr bool CAN_VIF = (MODE == kModeFactor || MODE == kModeVifAdj);
  const bool vif = CAN_VIF && (g.gram_d != nullptr || g.gram_f != nullptr);
  (void)vif;
  const auto* lags = lag_smem ? bs->lag : nullptr;
  const int npairs = bs->npairs;
  if constexpr (TILED) {
    if (fast) cov_tiled<T, NU, PM, true>(th, lagd, lagf, bs->lag, allint, bs, s, tR, tC, lane);
    else cov_tiled<T, NU, PM, false>(th, lagd, lagf, lags, allint, bs, s, tR, tC, lane);
  }
#pragma unroll 2
  for (int q = lane; q < (TILED ? 0 : npairs); q += 32) {
    const uint32_t rce = bs->pairs[q];
    const int r = rce & 0xff, c = (rce >> 8) & 0xff, e = (int)(rce >> 16);
    T v;
    float q1 = 0.f;
    T xv = T(0), ev = T(1);
    const Pos<T> pr = s.pos[r], pc = s.pos[c];
    if (!pr.valid || !pc.valid) {
      v = T(0);
    } else {
      const T dx = pr.ox - pc.ox, dy = pr.oy - pc.oy;
      const T d2 = dx * dx + dy * dy;
      T P, G, Qa, L;
      lag_lookup<T>(th, lagd, lagf, lags, allint, pr.td, pc.td, s.tt[r], s.tt[c], P, G, Qa, L);
      if constexpr (MIXED) {
        // FP32: h = d2 * rsqrt(d2), e^-x via the exp2 unit (relative errors
        // of a few 1e-7, inside the mixed form's covariance error budget)
        const float h = d2 >= kFltMinNormal ? d2 * rsqrt_ftz(d2) : 0.f;
        if (CAN_VIF && vif) {
          // VIF: the residual C - U U^T is a small difference, which
          // amplifies any systematic FP32 error in C (a rounded lag factor,
          // an approximate exp): C is evaluated in double-float arithmetic
          // (~48 bits, FP32 pipe) and C - G rounded once
          df P2, G2;
          const int lag = abs(pr.td - pc.td);
          if (allint && lag < kLagTab && g.lagdf != nullptr) {
            const float4 f = __ldg(g.lagdf + lag);
            P2 = df{f.x, f.y};
            G2 = df{f.z, f.w};
          } else {
            const LagD f = lag_factors(th, allint ? (double)lag : s.tt[r] - s.tt[c]);
            P2 = df_split(f.P);
            G2 = df_split(f.G);
          }
          const df dx = df_two_sum(pr.ox, -pc.ox), dy = df_two_sum(pr.oy, -pc.oy);
          const df xx = dfm_mul(G2, dfm_sqrt(dfm_add(dfm_mul(dx, dx), dfm_mul(dy, dy))));
          const df ee = dfm_exp_neg(xx);
          const df cc = dfm_mul(P2, dfm_matern<NU>(xx, ee));
          if (MODE == kModeVifAdj) q1 = P2.hi * matern_xdM<NU, float>(xx.hi, ee.hi);  // P x M'(x)
          const float gv = g.gram_f ? g.gram_f[gi * NPAIR + e] : 0.f;
          const df t = df_two_sum(cc.hi, -gv);
          v = t.hi + (t.lo + cc.lo);
        } else {
          const float x = G * h;
          const float E = __expf(-x);
          v = P * matern_M<NU, float>(x, E);
          q1 = P * matern_xdM<NU, float>(x, E);
        }
      } else {
        xv = G * sqrt(d2);
        ev = exp(-xv);
        v = P * matern_M<NU, T>(xv, ev);
      }
    }
    if (CAN_VIF && vif && pr.valid && pc.valid) {
      if (g.gram_d) {
        v -= (T)g.gram_d[gi * NPAIR + e];
      } else if (g.gram_f && !MIXED) {
        v -= (T)g.gram_f[gi * NPAIR + e];
      }
    }
    s.K[r][c] = v;
    s.K[c][r] = v;
    if (MODE == kModeNllGrad || MODE == kModeVifAdj) {
      if constexpr (MIXED) {
        s.q1[e] = q1;
      } else {
        s.xe[e][0] = xv;
        s.xe[e][1] = ev;
      }
    }
  }
  // diagonal (unused positions: 1), and the padding positions m..PM-2, which
  // the pair loop skips: identity rows and columns
  if (lane < PM) {
    const bool vj = s.pos[lane].valid;
    T v = vj ? diag : T(1);
    if (CAN_VIF && vif && vj) {
      const int ed = pair_e<PM>(lane, lane);
      if (g.gram_d) v -= (T)g.gram_d[gi * NPAIR + ed];
      else if (g.gram_f) v = (T)((th.sigma1sq + th.nugget) - (double)g.gram_f[gi * NPAIR + ed]);
    }
    s.K[lane][lane] = v;
    for (int j = m; j < LAST; ++j) {
      if (lane != j) {
        s.K[j][lane] = T(0);
        s.K[lane][j] = T(0);
      }
    }
  }
  __syncwarp();

  // ---- 3. Cholesky, row `lane` in registers (row reads are 16-byte vectors)
  const int lj = lane < PM ? lane : PM - 1;
  T a[PM];
#pragma unroll
  for (int q = 0; q < PM; q += VEC) {
    T tmp[VEC];
    ld16<T, VEC>(tmp, &s.K[lj][q]);
#pragma unroll
    for (int u = 0; u < VEC; ++u) a[q + u] = tmp[u];
  }
  // Each lane keeps its own pivot (checked once after the loop) and 1/L_jj.
  // Entries above the diagonal (a[k] of lanes j < k) are updated like the
  // others but never read: the solves read the lower triangle only, and a
  // step reads the broadcast column only below its pivot.
  T dinv = T(1), mypiv = T(1);
#pragma unroll
  for (int k = 0; k < PM; ++k) {
    if (!MIXED && k >= m && k < LAST) continue;  // FP64: skip padding positions (identity rows and columns)
    const T piv = __shfl_sync(kFull, a[k], k);
    const T rs = drsqrt<T>(piv);  // NaN or inf for a pivot <= 0: the row fails the check below
    if (lane == k) {
      dinv = rs;
      mypiv = piv;
    }
    const T v = a[k] * rs;
    a[k] = v;
    if (lane < PM) s.col[lane] = v;
    __syncwarp();
#pragma unroll
    for (int q = ((k + 1) / VEC) * VEC; q < PM; q += VEC) {
      T cv[VEC];
      ld16<T, VEC>(cv, &s.col[q]);
      if constexpr (MIXED) {
        // packed FP32 pairs (q + u, q + u + 1): one instruction updates both
#pragma unroll
        for (int u = 0; u < VEC; u += 2) {
          if (q + u > k) {
            const float2 r = __ffma2_rn(make_float2(-v, -v), make_float2(cv[u], cv[u + 1]),
                                        make_float2(a[q + u], a[q + u + 1]));
            a[q + u] = r.x;
            a[q + u + 1] = r.y;
          } else if (q + u + 1 > k) {
            a[q + u + 1] = fma(-v, cv[u + 1], a[q + u + 1]);
          }
        }
      } else {
#pragma unroll
        for (int u = 0; u < VEC; ++u)
          if (q + u > k) a[q + u] = fma(-v, cv[u], a[q + u]);
      }
    }
    __syncwarp();
  }
  const bool ok = __all_sync(kFull, mypiv > T(0));

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
    if (!ok || !(ratio * ratio <= g.tau)) {
      if (lane == 0) {
        g.flag[ri] = 1;
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
  T(*Lsm)[WarpSm<T, PM>::KS] = MIXED ? reinterpret_cast<T(*)[WarpSm<T, PM>::KS]>(&s.Ls[0][0]) : s.K;
  __syncwarp();
  if (lane < PM) {
#pragma unroll
    for (int q = 0; q < PM; q += VEC) {
      T tmp[VEC];
#pragma unroll
      for (int u = 0; u < VEC; ++u) tmp[u] = a[q + u];
      st16<T, VEC>(&Lsm[lane][q], tmp);
    }
  }
  __syncwarp();
  const T Llast = (T)1 / __shfl_sync(kFull, dinv, LAST);
  const T wj = (lane < LAST) ? Lsm[LAST][lane] : T(0);  // last row: L_N^{-1} k

  // forward solve z = L^{-1} y_local (NLL of the FP64 form; b for the gradient)
  T zj = T(0);
  if ((!MIXED && MODE != kModeFactor) || MODE == kModeNllGrad || MODE == kModeVifAdj) {
    T accz = (lane < PM) ? yv : T(0);
#pragma unroll
    for (int k = 0; k < PM; ++k) {
      if (!MIXED && k >= m && k < LAST) continue;  // FP64: skip padding positions (identity rows and columns)
      const T zk = __shfl_sync(kFull, accz * dinv, k);
      if (lane == k) zj = zk;
      accz = fma(-a[k], zk, accz);  // lanes <= k: their z is taken already
    }
  }

  // backward solves with L_N^T: aj = (L_N^{-T} w)_j, bj = (L_N^{-T} z_N)_j
  const bool need_b = (MODE == kModeNllGrad) || (MODE == kModeVifAdj);
  const bool need_a = MIXED || MODE != kModeNll;
  T aj = T(0), bj = T(0);
  if (need_a) {
    T acc_a = wj, acc_b = (lane < LAST) ? zj : T(0);
#pragma unroll
    for (int k = LAST - 1; k >= 0; --k) {
      if (!MIXED && k >= m && k < LAST) continue;  // FP64: skip padding positions (identity rows and columns)
      T ak, bk = T(0);
      if constexpr (MIXED) {
        if (need_b) {
          const float2 sab = __fmul2_rn(make_float2(acc_a, acc_b), make_float2(dinv, dinv));
          ak = __shfl_sync(kFull, sab.x, k);
          bk = __shfl_sync(kFull, sab.y, k);
        } else {
          ak = __shfl_sync(kFull, acc_a * dinv, k);
        }
      } else {
        ak = __shfl_sync(kFull, acc_a * dinv, k);
        if (need_b) bk = __shfl_sync(kFull, acc_b * dinv, k);
      }
      if (lane == k) { aj = ak; bj = bk; }
      {
        // lanes >= k read entries on or above the diagonal and update sums
        // whose values are taken already
        const T lkj = Lsm[k][lane < PM ? lane : 0];
        if constexpr (MIXED) {
          if (need_b) {
            const float2 r = __ffma2_rn(make_float2(-lkj, -lkj), make_float2(ak, bk), make_float2(acc_a, acc_b));
            acc_a = r.x;
            acc_b = r.y;
          } else {
            acc_a = fma(-lkj, ak, acc_a);
          }
        } else {
          acc_a = fma(-lkj, ak, acc_a);
          if (need_b) acc_b = fma(-lkj, bk, acc_b);
        }
      }
    }
  }

  // ---- 4. D_i, r_i and the NLL term
  double Dd = 0.0;    // FP64 value of D_i (factor output)
  T Dt, rt;           // D_i and r_i in T for the adjoint weights
  df a_ref = {0.f, 0.f};  // mixed: refined A_i entry of this lane
  if constexpr (MIXED && MODE == kModeVifAdj) {
    // the adjoint pass needs neither D_i nor r_i (Dbar is given): no refinement
    Dt = T(1);
    rt = T(0);
  } else if constexpr (MIXED) {
    // One refinement step: res = k - K_N a (double-float), a += K_N^{-1} res.
    // The FP32 diagonal is sigma1^2 + nugget rounded once, the same way for
    // every row; the residual and D use its double-float value (dg_hi, dg_lo)
    // so that this rounding does not bias every D_i in the same direction.
    if (lane < PM) s.v0[lane] = (lane < LAST) ? aj : 0.0f;
    __syncwarp();
    df res = {0.0f, 0.0f};
    if (lane < LAST) {
      // two interleaved double-float sums (even and odd q) on packed FP32
      // pairs; v0[LAST] = 0, so the last pair's second term is exactly 0
      float2 hi = make_float2(s.K[lane][LAST], 0.0f), lo = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int q = 0; q < PM; q += 4) {
        float kv[4], av[4];
        ld16<float, 4>(kv, &s.K[lane][q]);
        ld16<float, 4>(av, &s.v0[q]);
        df2_dot_sub(hi, lo, make_float2(kv[0], kv[1]), make_float2(av[0], av[1]));
        df2_dot_sub(hi, lo, make_float2(kv[2], kv[3]), make_float2(av[2], av[3]));
      }
      res = df_two_sum(hi.x, hi.y);
      res.lo += lo.x + lo.y;
      if (valid && !vif) res.lo = fmaf(-th.dg_lo, aj, res.lo);
    }
    // with a Gram (VIF) every entry of K, the diagonal included, is the FP64
    // value rounded once, and K itself is the matrix the refinement solves with
    df Ds = (lane == LAST) ? (vif ? df{s.K[LAST][LAST], 0.0f} : df{th.dg_hi, th.dg_lo}) : df{0.0f, 0.0f};
    df rs = (lane == LAST) ? yl : df{0.0f, 0.0f};
    if (MODE != kModeNllGrad) {
      // explicit step a += K_N^{-1} res, then D = K_ii - k.a, r = y_i - y_N.a
      const float rf = res.hi + res.lo;
      float accr = (lane < LAST) ? rf : 0.0f, dz = 0.0f;
#pragma unroll
      for (int k = 0; k < LAST; ++k) {
        if (!MIXED && k >= m && k < LAST) continue;  // FP64: skip padding positions (identity rows and columns)
        const float zk = __shfl_sync(kFull, accr * dinv, k);
        if (lane == k) dz = zk;
        if (lane > k) accr = fmaf(-a[k], zk, accr);
      }
      float acc2 = (lane < LAST) ? dz : 0.0f, da = 0.0f;
#pragma unroll
      for (int k = LAST - 1; k >= 0; --k) {
        if (!MIXED && k >= m && k < LAST) continue;  // FP64: skip padding positions (identity rows and columns)
        const float dk = __shfl_sync(kFull, acc2 * dinv, k);
        if (lane == k) da = dk;
        if (lane < k) acc2 = fmaf(-Lsm[k][lane], dk, acc2);
      }
      a_ref = (lane < LAST) ? df{aj, da} : df{0.0f, 0.0f};
      if (lane < LAST) {
        df_fma_acc(Ds, -s.K[LAST][lane], a_ref);
        df_fma_acc(rs, -yl.hi, a_ref);
        rs.lo = fmaf(-yl.lo, a_ref.hi, rs.lo);
      }
    } else if (lane < LAST) {
      // the same step without the correction solves: with a* = a + K_N^{-1} res
      // and b = K_N^{-1} y_N (computed for the adjoint),
      //   D* = K_ii - k.a - a.res,   r* = y_i - y_N.a - b.res,
      // exact up to terms quadratic in the FP32 solve error
      // (the corrections are ~1e-7 of D and r: FP32 products suffice)
      const float rf = res.hi + res.lo;
      df_fma_acc(Ds, -s.K[LAST][lane], df{aj, 0.0f});
      Ds.lo = fmaf(-aj, rf, Ds.lo);
      df_fma_acc(rs, -yl.hi, df{aj, 0.0f});
      rs.lo = fmaf(-yl.lo, aj, fmaf(-bj, rf, rs.lo));
    }
    {
      // both double-float warp sums on packed FP32 pairs (the steps of df_warp_sum)
      const float2 m1 = make_float2(-1.0f, -1.0f);
      float2 hi = make_float2(Ds.hi, rs.hi), lo = make_float2(Ds.lo, rs.lo);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float2 oh = make_float2(__shfl_xor_sync(kFull, hi.x, o), __shfl_xor_sync(kFull, hi.y, o));
        const float2 ol = make_float2(__shfl_xor_sync(kFull, lo.x, o), __shfl_xor_sync(kFull, lo.y, o));
        const float2 sm = __fadd2_rn(hi, oh);
        const float2 bb = __ffma2_rn(hi, m1, sm);
        const float2 er = __fadd2_rn(__ffma2_rn(__ffma2_rn(bb, m1, sm), m1, hi), __ffma2_rn(bb, m1, oh));
        hi = sm;
        lo = __fadd2_rn(__fadd2_rn(lo, ol), er);
      }
      Ds = df{hi.x, lo.x};
      rs = df{hi.y, lo.y};
    }
    Dt = Ds.hi + Ds.lo;
    rt = rs.hi + rs.lo;
    if (!(Dt > 0.0f) || !(rt == rt)) {  // lost to FP32 rounding: redo in FP64
      if (lane == 0) {
        g.flag[ri] = 1;
        atomicAdd(&g.hdr->n_fallback, 1ull);
      }
      return;
    }
    if (MODE == kModeFactor) Dd = df_to_double(Ds);
    if (MODE != kModeFactor && lane == 0) {
      // log D = log(D_hi) + log(1 + D_lo / D_hi), the second term to first order
      const float logD = logf(Ds.hi) + Ds.lo / Ds.hi;
      acc.add(0, 0.5f * logD);
      acc.add(0, 0.5f * (rt * rt / Dt));
    }
  } else {
    const double Ll = (double)Llast;
    const double zl = __shfl_sync(kFull, (double)zj, LAST);
    Dd = Ll * Ll;
    Dt = (T)Dd;
    rt = (T)(zl * Ll);
    if (!(Dd > 0.0)) {
      if (lane == 0) report_error(g.hdr, VST_ENOTSPD, gi);
      return;
    }
    if (MODE != kModeFactor && MODE != kModeVifAdj && lane == 0) acc.add(0, log(Ll) + 0.5 * zl * zl);
  }

  if (MODE == kModeFactor) {
    if (lane < m) {
      double v = 0.0;
      if (lane < cnt) v = MIXED ? df_to_double(a_ref) : (double)aj;
      g.A[ri * m + lane] = v;
    }
    if (lane == 0) g.D[ri] = Dd;
    return;
  }

  // ---- 5. adjoint: sum over pairs of W_pq dSigma~_pq / dtheta
  // (kModeVifAdj: W = Dbar a~ a~^T + (a~ b~^T + b~ a~^T) / 2 with
  // b~ = (K_N^{-1} Abar, 0), i.e. c1 = Dbar, c2 = -1)
  if (MODE == kModeNllGrad || MODE == kModeVifAdj) {
    const T c2 = MODE == kModeVifAdj ? T(-1) : rt / Dt;
    const T c1 = MODE == kModeVifAdj ? (T)g.dbar[ri] : T(0.5) * (T(1) / Dt - c2 * c2);
    __syncwarp();
    if (lane < PM) {
      const T at = (lane < cnt) ? -aj : (lane == LAST ? T(1) : T(0));
      const T bt = (lane < cnt) ? bj : T(0);
      s.ab[lane][0] = at;
      s.ab[lane][1] = bt;
    }
    if (MODE == kModeVifAdj && lane < m) g.btil[ri * m + lane] = (lane < cnt) ? (double)bj : 0.0;
    __syncwarp();
    // off-diagonal sums of w K and w X are scaled by 1/sigma1^2 and 1/c at the end
    T gd = 0, g0 = 0, g1 = 0, g2 = 0, g3 = 0;
    const T pexp = MIXED ? (T)th.pf : (T)th.p, hg = MIXED ? (T)th.hgf : (T)(0.5 * th.gamma);
    const T hc2 = T(0.5) * c2;
    if constexpr (TILED) {
      if (fast) adj_tiled<T, NU, PM, true>(th, lagd, lagf, bs->lag, allint, bs, s, tR, tC, lane, c1, hc2, pexp, hg, g0,
                                           g1, g2, g3);
      else adj_tiled<T, NU, PM, false>(th, lagd, lagf, lags, allint, bs, s, tR, tC, lane, c1, hc2, pexp, hg, g0, g1,
                                       g2, g3);
    }
#pragma unroll 2
    for (int q = lane; q < (TILED ? 0 : npairs); q += 32) {
      const uint32_t rce = bs->pairs[q];
      const int r = rce & 0xff, c = (rce >> 8) & 0xff, e = (int)(rce >> 16);
      const Pos<T> pr = s.pos[r], pc = s.pos[c];
      if (!pr.valid || !pc.valid) {
        continue;
      }
      const T ar = s.ab[r][0], br = s.ab[r][1], ac = s.ab[c][0], bc = s.ab[c][1];
      const T w = ar * (c1 * ac - hc2 * bc) - hc2 * br * ac;
      {
        T P, G, Qa, L;
        lag_lookup<T>(th, lagd, lagf, lags, allint, pr.td, pc.td, s.tt[r], s.tt[c], P, G, Qa, L);
        T Kv, Xv;  // P M(x) and P x M'(x)
        if constexpr (MIXED) {
          Kv = s.K[r][c];
          // VIF: K holds the residual C - G; the derivative is that of C
          if (MODE == kModeVifAdj && vif) Kv += g.gram_f[gi * NPAIR + e];
          Xv = s.q1[e];
        } else {
          const T x = s.xe[e][0], E = s.xe[e][1];
          Kv = P * matern_M<NU, T>(x, E);
          Xv = P * matern_xdM<NU, T>(x, E);
        }
        const T w2 = w + w;
        g0 = fma(w2, Kv, g0);
        g1 = fma(w2, Xv, g1);
        g2 = fma(w2 * Qa, -pexp * Kv - hg * Xv, g2);
        g3 = fma(-w2 * L, Kv + T(0.5) * Xv, g3);
      }
    }
    // diagonal pairs: dC(0,0)/dsigma1^2 = 1 and d/dnugget = 1
    if (lane < PM) {
      const T at = s.ab[lane][0], bt = s.ab[lane][1];
      const T w = at * (c1 * at - hc2 * bt) - hc2 * bt * at;
      const bool vj = s.pos[lane].valid;
      if (vj) gd += w;
    }
    const T inv_s1 = MIXED ? (T)th.inv_s1f : T(1.0 / th.sigma1sq);
    const T inv_c = MIXED ? (T)th.inv_cf : T(1.0 / th.c);
    acc.add(1, fma(g0, inv_s1, gd));
    acc.add(2, g1 * inv_c);
    acc.add(3, g2);
    acc.add(4, g3);
    acc.add(5, gd);
  }
}

template <typename T, int PM>
__host__ __device__ constexpr size_t block_sm_bytes() {
  return (sizeof(BlockSm<T, PM>) + 15) / 16 * 16;
}

template <typename T, int PM, int WARPS>
__host__ __device__ constexpr size_t rows_smem_bytes() {
  return block_sm_bytes<T, PM>() + sizeof(WarpSm<T, PM>) * WARPS;
}

template <typename T, int NU, int PM, int MODE, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 16 / WARPS) rows_kernel(RowArgs g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BlockSm<T, PM>* bs = reinterpret_cast<BlockSm<T, PM>*>(smem_raw);
  WarpSm<T, PM>* sm = reinterpret_cast<WarpSm<T, PM>*>(smem_raw + block_sm_bytes<T, PM>());
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpSm<T, PM>& s = sm[wib];
  if (wib == 0) {
    // the off-diagonal pairs among positions 0..m-1 and PM-1, in packed order
    constexpr int NP = WarpSm<T, PM>::NPAIR;
    const int m = g.m;
    int count = 0;
    for (int base = 0; base < NP; base += 32) {
      const int e = base + lane;
      int r = 0, c = 0;
      bool keep = false;
      if (e < NP) {
        pair_of<PM>(e, r, c);
        keep = r != c && (r < m || r == PM - 1) && (c < m || c == PM - 1);
      }
      const unsigned mask = __ballot_sync(kFull, keep);
      if (keep) bs->pairs[count + __popc(mask & ((1u << lane) - 1u))] = (uint32_t)(r | (c << 8) | (e << 16));
      count += __popc(mask);
    }
    if (lane == 0) bs->npairs = count;
    // pairs r > c inside the 8 diagonal blocks of TS = PM / 8 positions
    if (lane == 0) {
      constexpr int TS = TileShape<PM>::TS;
      int nd = 0;
      for (int b = 0; b < 8; ++b)
        for (int r = 1; r < TS; ++r)
          for (int c = 0; c < r; ++c) bs->dpairs[nd++] = (uint32_t)((b * TS + r) | ((b * TS + c) << 8));
      bs->ndpairs = nd;
    }
  }
  if (g.offsets == nullptr) {
    for (int u = threadIdx.x; u < kLagSmem; u += WARPS * 32) {
      if constexpr (std::is_same<T, float>::value) bs->lag[u] = g.lagf[u];
      else bs->lag[u] = g.lagd[u];
    }
  }
  __syncthreads();
  const BlockSm<T, PM>* bsc = bs;
  int tR = 0, tC = 0;
  tile_of_lane(lane, tR, tC);
  const int64_t warp = (int64_t)blockIdx.x * WARPS + wib;
  const int64_t total = (int64_t)gridDim.x * WARPS;
  RowAcc<T> acc;
  acc.zero();

  if (g.offsets == nullptr) {
    const int64_t n = g.n;
    bool any = true;
    if (g.fallback_only) any = g.hdr->n_fallback != 0ull;
    if (any) {
      const int64_t chunk = g.row_chunk > 0 ? g.row_chunk : 1;
      for (int64_t base = g.out0 + warp * chunk; base < n; base += total * chunk) {
        const int64_t end = base + chunk < n ? base + chunk : n;
        for (int64_t i = base; i < end; ++i) {
          if (g.fallback_only && g.flag[i - g.out0] == 0) continue;
          row_body<T, NU, PM, MODE>(g, g.th, g.lagd, g.lagf, bsc, true, s, i, 0, lane, acc, tR, tC);
        }
      }
    }
    // fixed-order reduction of this warp's partial sums (FP64)
    double v[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) v[q] = warp_sum(acc.get(q));
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < 6; ++q) g.partial[warp * 8 + q] = v[q];
    }
  } else {
    // batched form: global rows across datasets, per-row outputs; the lag
    // table differs per dataset, so only the pair table is shared
    // rows beyond the caller's n are never touched, whatever the offsets hold
    const int64_t n = g.offsets[g.nsets] < g.n ? g.offsets[g.nsets] : g.n;
    const int64_t chunk = g.row_chunk > 0 ? g.row_chunk : 1;
    int set = 0;
    for (int64_t base = warp * chunk; base < n; base += total * chunk) {
      const int64_t end = base + chunk < n ? base + chunk : n;
      for (int64_t gi = base; gi < end; ++gi) {
        if (g.fallback_only && g.flag[gi] == 0) continue;
        while (set + 1 < g.nsets && g.offsets[set + 1] <= gi) ++set;
        const int64_t row0 = g.offsets[set];
        acc.zero();
        row_body<T, NU, PM, MODE>(g, g.thetas[set], g.lagd_sets + (int64_t)set * kLagTab,
                                  g.lagf_sets + (int64_t)set * kLagTab, bsc, false, s, gi - row0, row0, lane,
                                  acc, tR, tC);
        // per-row results: FP64 rows as double[6]; mixed rows as double-float
        // pairs float2[6] (same 48 bytes), combined by the segmented reduction
        const bool skip = g.flag != nullptr && !g.fallback_only && g.flag[gi];
        if constexpr (std::is_same<T, float>::value) {
          df v[6];
#pragma unroll
          for (int q = 0; q < 6; ++q) v[q] = df_warp_sum(acc.v[q]);
          if (lane == 0 && !skip) {
            float2* o = reinterpret_cast<float2*>(g.row_out + gi * 6);
#pragma unroll
            for (int q = 0; q < 6; ++q) o[q] = make_float2(v[q].hi, v[q].lo);
          }
        } else {
          double v[6];
#pragma unroll
          for (int q = 0; q < 6; ++q) v[q] = warp_sum(acc.get(q));
          if (lane == 0 && !skip) {
#pragma unroll
            for (int q = 0; q < 6; ++q) g.row_out[gi * 6 + q] = v[q];
          }
        }
      }
    }
  }
}

}  // namespace vst
