// Residual-correlation neighbours of the VIF approximation (Sect. 4.3 with
// the correlation-based selection of Sect. 4.4.1 applied to the residual
// process): N(i) = the min(i, m) predecessors j < i with the largest
// |rho_ij| = |C_ij - U_i . U_j| / sqrt(r_i r_j), ties to the smaller index,
// exact in FP64.
//
// The search is exact but filtered:
//   1. a lower bound tau_i of the m-th largest |rho_ij|: the smallest |rho|
//      (FP64) over m actual predecessors, the plain-correlation neighbours;
//   2. a pass over all pairs j < i in 128 x 64 tiles, FP32 dot products and
//      covariance, that keeps every j whose |rho| can reach tau_i: the test
//      carries a rigorous bound on the FP32 error (accumulation of k
//      products, rounding of U, the covariance functions and the coordinate
//      offsets), so every j with |rho_ij| >= tau_i (1 - 2e-12) is kept;
//   3. the kept candidates ranked in FP64, the top m + 1 kept in order.
// A row whose candidates overflow the kVifCand slots takes the m-th best of
// the stored ones (exact, so still a lower bound) as its threshold and is
// screened again over all predecessors, lane by lane (FP32 with the same
// bound, FP64 for the survivors); a row whose residual variance is below
// 1e-12 sigma1^2 goes there with every j kept.  The workspace header's
// n_fallback counts the rows of this second pass.
// The m-th / (m+1)-th comparison for the tie list is exact as well: a
// dropped j has |rho_ij| < tau_i (1 - 2e-12) <= the m-th value (1 - 2e-12).
#include <algorithm>
#include <climits>

#include "kernels.h"
#include "profile.h"
#include "vif.h"
#include "workspace.h"

namespace vst {

vst_status fail(vst_status s, const char* fmt, ...);
vst_status cuda_fail(cudaError_t e, const char* where);
vst_status plain_knn(const double* xy, const double* t, int64_t n, const vst_theta* theta, int m, int32_t* nn,
                     int32_t* nn_cnt, int64_t* tie_rows, int64_t tie_cap, char* base, const WsLayout& L,
                     WsHeader* hdr, int64_t n_cand, int64_t row0, cudaStream_t st);

namespace {

constexpr float kU = 5.9604645e-8f;  // 2^-24

struct KnnArgsV {
  const double* xy;
  const double* t;
  int64_t n;
  int m;
  int k;
  DevTheta th;
  const double* U;   // FP64 [n][k]
  const float* Uf;   // FP32 copy [n][k]
  const double* r;   // [n]
  float4* rowinfo;   // per row: (threshold tau_i s_i, s_i = sqrt(r_i), |U_i|, 0)
  int32_t* cand;     // [n][kVifCand]
  int32_t* ccount;   // [n]
  int32_t* fbrows;   // rows for the second pass
  unsigned long long* fbcount;
  int32_t* nn;       // in: plain neighbours (stage 1); out: residual neighbours
  int32_t* nn_cnt;
  int64_t* tie_rows;
  int64_t tie_cap;
  WsHeader* hdr;
};

// FP64 |rho_ij| of row i (U_i in shared memory) for up to 32 predecessors,
// one per lane (j < 0: none).  The covariance is evaluated by each lane for
// its own j; the dot products U_i . U_j are taken one j at a time by the
// whole warp (coalesced reads of U_j, lanes over the k columns).
template <int NU>
__device__ __forceinline__ double rho64_group(const KnnArgsV& A, const double* ui, double xi, double yi, double ti,
                                              double ri, int64_t j, int lane) {
  const double tiny = 1e-12 * A.th.sigma1sq;
  double C = 0.0, rj = 0.0;
  if (j >= 0) {
    C = cov64<NU>(A.th, xi - A.xy[2 * j], yi - A.xy[2 * j + 1], ti - A.t[j]);
    rj = A.r[j];
  }
  double mydot = 0.0;
  unsigned act = __ballot_sync(kFull, j >= 0);
  while (act) {
    const int q = __ffs(act) - 1;
    act &= act - 1;
    const int64_t jq = __shfl_sync(kFull, j, q);
    const double* uj = A.U + jq * A.k;
    double s = 0.0;
    for (int c = lane; c < A.k; c += 32) s = fma(ui[c], uj[c], s);
    s = warp_sum(s);
    if (lane == q) mydot = s;
  }
  if (j < 0) return -1.0e300;
  return (ri > tiny && rj > tiny) ? fabs(C - mydot) / sqrt(ri * rj) : 0.0;
}

// ---- stage 1: thresholds
template <int NU, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) tau_kernel(KnnArgsV A) {
  extern __shared__ double ui_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* ui = ui_raw + (int64_t)wib * A.k;
  const int64_t warp = (int64_t)blockIdx.x * WARPS + wib;
  const int64_t total = (int64_t)gridDim.x * WARPS;
  const double tiny = 1e-12 * A.th.sigma1sq;
  for (int64_t i = warp; i < A.n; i += total) {
    const double ri = A.r[i];
    const float si = (float)sqrt(fmax(ri, 0.0));
    const float nui = (float)sqrt(fmax(A.th.sigma1sq - ri, 0.0));
    if (i <= A.m) {  // all predecessors are neighbours: keep every j < i
      if (lane == 0) A.rowinfo[i] = make_float4(-1.0f, si, nui, 0.0f);
      continue;
    }
    if (!(ri > tiny)) {  // no residual correlation defined: every j to the exact pass
      if (lane == 0) {
        A.rowinfo[i] = make_float4(-1.0f, si, nui, 1.0f);
        A.fbrows[atomicAdd(A.fbcount, 1ull)] = (int32_t)i;
      }
      continue;
    }
    for (int c = lane; c < A.k; c += 32) ui[c] = A.U[i * A.k + c];
    __syncwarp();
    const double xi = A.xy[2 * i], yi = A.xy[2 * i + 1], ti = A.t[i];
    const int cnt = min(max(A.nn_cnt[i], 0), A.m);
    int64_t jn = -1;
    if (lane < cnt) {
      const int j = A.nn[i * A.m + lane];
      if (j >= 0 && j < i) jn = j;
    }
    const double rv = rho64_group<NU>(A, ui, xi, yi, ti, ri, jn, lane);
    double v = jn >= 0 ? rv : 1.0e300;
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(kFull, v, o));
    // tau (1 - 2e-12), times s_i, rounded down to FP32
    if (lane == 0) {
      float thr = -1.0f;
      if (cnt == A.m && v < 1.0e300) {
        const double tv = v * (1.0 - 2e-12) * (double)si;
        thr = __double2float_rd(tv);
      }
      A.rowinfo[i] = make_float4(thr, si, nui, 0.0f);
    }
    __syncwarp();
  }
}

__global__ void narrow_kernel(const double* U, int64_t count, float* Uf) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count; q += (int64_t)gridDim.x * blockDim.x)
    Uf[q] = (float)U[q];
}

// covariance of Eq. (2) in FP32 (the same steps as the mixed form's cov32)
// and a bound on its relative error in units of u = 2^-24, from the error
// bounds of the FP32 functions (log2f 2 ulp, exp2f / expf / rsqrtf 3 ulp,
// 1 ulp <= 2u) carried through each step: the lag powers (relative error of
// psi^-p grows with p |log2 psi| and the |2 alpha log2|u|| of the inner
// power), the Matern argument x = G h (its relative error enters C times x)
template <int NU>
__device__ __forceinline__ float cov32_err(const DevTheta& th, float dx, float dy, float u, float& rel) {
  const float au = fabsf(u);
  const float l2 = au > 0.f ? log2f(au) : 0.f;
  const float arg = 2.0f * (float)th.alpha * l2;
  const float psi = au > 0.f ? fmaf((float)th.a, exp2f(arg), 1.0f) : 1.0f;
  const float lp = log2f(psi);
  const float P = (float)th.sigma1sq * exp2f(-(float)th.p * lp);
  const float G = (float)th.c * exp2f(-0.5f * (float)th.gamma * lp);
  const float d2 = dx * dx + dy * dy;
  const float x = G * (d2 > 0.f ? d2 * rsqrtf(d2) : 0.f);
  const float C = P * matern_M<NU, float>(x, expf(-x));
  const float core = 4.3f * fabsf(arg) + 8.1f + 4.2f * fabsf(lp);
  const float relP = fabsf((float)th.p) * core + 8.0f;
  const float relx = 0.5f * fabsf((float)th.gamma) * core + 19.0f;
  rel = 1.25f * (relP + x * relx + 10.0f) + 16.0f;
  return C;
}

// ---- stage 2: candidates.  Tiles of 128 rows x 64 columns covering j < i
// (row tile ti, column tiles 0..2 ti + 1); 256 threads, 4 x 8 products per
// thread, K step 16.  Each 16-term chunk is summed in FP32 and added to a
// double-float accumulator, so the dot product's error is below
// 24 u |U_i| |U_j| (Cauchy-Schwarz on 18 u sum |U_ic U_jc|, plus the
// rounding of U to FP32 and of the final value).
template <int NU>
__global__ void __launch_bounds__(256) filter_kernel(KnnArgsV A, int64_t ntiles) {
  constexpr int BI = 128, BJ = 64, BK = 16;
  __shared__ __align__(16) float As[BK][BI + 4];
  __shared__ __align__(16) float Bs[BK][BJ + 4];
  __shared__ float rx[BI], ry[BI], rt[BI], cx[BJ], cy[BJ], ct[BJ];
  __shared__ float4 rinfo[BI];
  __shared__ float cs[BJ], cnu[BJ];
  const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
  const float sig = (float)A.th.sigma1sq, cpar = (float)A.th.c;
  const float dotc = 24.0f * 1.05f * kU;
  for (int64_t b = blockIdx.x; b < ntiles; b += gridDim.x) {
    // b = ti (ti + 1) + tj, 0 <= tj <= 2 ti + 1
    int64_t ti = (int64_t)((sqrt(4.0 * (double)b + 1.0) - 1.0) * 0.5);
    while (ti * (ti + 1) > b) --ti;
    while ((ti + 1) * (ti + 2) <= b) ++ti;
    const int64_t tj = b - ti * (ti + 1);
    const int64_t i0 = ti * BI, j0 = tj * BJ;
    __syncthreads();
    bool tok = true;
    if (tid < BI) {
      // coordinates and times as FP32 offsets from the tile's first row
      // (computed in FP64); the time offsets must be exact in FP32 (integer
      // days below 2^24), else the tile keeps every pair
      const double X0 = A.xy[2 * i0], Y0 = A.xy[2 * i0 + 1], T0 = A.t[i0];
      const int64_t i = i0 + tid;
      const bool vi = i < A.n;
      const double dti = vi ? A.t[i] - T0 : 0.0;
      tok = dti == floor(dti) && fabs(dti) < 16777216.0;
      rx[tid] = vi ? (float)(A.xy[2 * i] - X0) : 0.f;
      ry[tid] = vi ? (float)(A.xy[2 * i + 1] - Y0) : 0.f;
      rt[tid] = (float)dti;
      rinfo[tid] = vi ? A.rowinfo[i] : make_float4(3.0e38f, 0.f, 0.f, 0.f);
    } else if (tid < BI + BJ) {
      const double X0 = A.xy[2 * i0], Y0 = A.xy[2 * i0 + 1], T0 = A.t[i0];
      const int jl = tid - BI;
      const int64_t j = j0 + jl;
      const bool vj = j < A.n;
      const double dtj = vj ? A.t[j] - T0 : 0.0;
      tok = dtj == floor(dtj) && fabs(dtj) < 16777216.0;
      cx[jl] = vj ? (float)(A.xy[2 * j] - X0) : 0.f;
      cy[jl] = vj ? (float)(A.xy[2 * j + 1] - Y0) : 0.f;
      ct[jl] = (float)dtj;
      const float4 ci = vj ? A.rowinfo[j] : make_float4(0.f, 0.f, 0.f, 0.f);
      cs[jl] = ci.y;
      cnu[jl] = ci.z;
    }
    const int times_exact = __syncthreads_and(tok);
    float hi[4][8], lo[4][8];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 8; ++v) hi[u][v] = lo[u][v] = 0.f;
    for (int kb = 0; kb < A.k; kb += BK) {
      __syncthreads();
      for (int q = tid; q < BK * (BI + BJ); q += 256) {
        const int kk = q & (BK - 1), rr = q >> 4;
        if (rr < BI) {
          const int64_t i = i0 + rr;
          As[kk][rr] = (i < A.n && kb + kk < A.k) ? A.Uf[i * A.k + kb + kk] : 0.f;
        } else {
          const int64_t j = j0 + rr - BI;
          Bs[kk][rr - BI] = (j < A.n && kb + kk < A.k) ? A.Uf[j * A.k + kb + kk] : 0.f;
        }
      }
      __syncthreads();
      float acc[4][8];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
        const float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8]);
        const float4 b1 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8 + 4]);
        const float av[4] = {a0.x, a0.y, a0.z, a0.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          const df t = df_two_sum(hi[u][v], acc[u][v]);
          hi[u][v] = t.hi;
          lo[u][v] += t.lo;
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int il = ty * 4 + u;
      const int64_t i = i0 + il;
      if (i >= A.n) continue;
      const float4 ri = rinfo[il];
      if (ri.w != 0.0f) continue;  // searched by the second pass
      const float xi = rx[il], yi = ry[il], tiv = rt[il];
      const float offi = fabsf(xi) + fabsf(yi);
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        const int jl = tx * 8 + v;
        const int64_t j = j0 + jl;
        if (j >= i) continue;
        float rel;
        const float C = cov32_err<NU>(A.th, xi - cx[jl], yi - cy[jl], tiv - ct[jl], rel);
        const float R = fabsf(C - (hi[u][v] + lo[u][v]));
        // covariance: functions, and the coordinate offsets (|dC/dx| <= C,
        // G <= c, |dh| <= 2u (|x_i| + |y_i| + |x_j| + |y_j|)); dot product;
        // an underflow floor
        const float offs = offi + fabsf(cx[jl]) + fabsf(cy[jl]);
        const float bound = 1.1f * fabsf(C) * (rel * kU + cpar * 2.0f * kU * offs) + dotc * ri.z * cnu[jl] +
                            1.0e-33f * sig;
        const float rhs = ri.x * cs[jl];
        // keep if |R| + bound >= tau_i s_i s_j; the extra half bound and the
        // 4u terms cover the rounding of this test
        if (!times_exact || R + 1.5f * bound + 4.0f * kU * (R + fabsf(rhs)) >= rhs) {
          const int slot = atomicAdd(&A.ccount[i], 1);
          if (slot < kVifCand) A.cand[i * kVifCand + slot] = (int32_t)j;
        }
      }
    }
  }
}

// insert (cr, cj) into the warp's sorted top-K list (descending |rho|, ties to
// the smaller index); lanes < count hold the list
__device__ __forceinline__ void topk_insert(int lane, int K, double cr, int cj, double& lr, int& lid, int& count,
                                            double& thr) {
  if (count >= K && cr < thr) return;
  const bool better = lane < count && (lr > cr || (lr == cr && lid < cj));
  const int p = __popc(__ballot_sync(kFull, better));
  if (p >= K) return;
  const double ur = __shfl_up_sync(kFull, lr, 1);
  const int uid = __shfl_up_sync(kFull, lid, 1);
  if (lane > p) { lr = ur; lid = uid; }
  if (lane == p) { lr = cr; lid = cj; }
  count = min(count + 1, K);
  if (count >= K) thr = __shfl_sync(kFull, lr, K - 1);
}

__device__ __forceinline__ void write_row(const KnnArgsV& A, int lane, int64_t i, int count, double lr, int lid) {
  const int K = A.m + 1;
  const int cnt = min(count, A.m);
  if (lane < A.m) A.nn[i * A.m + lane] = lane < cnt ? lid : -1;
  if (lane == 0) A.nn_cnt[i] = cnt;
  if (count == K && A.m > 0) {
    const double rm = __shfl_sync(kFull, lr, A.m - 1);
    const double rm1 = __shfl_sync(kFull, lr, A.m);
    if (lane == 0 && (rm - rm1) <= 1e-12 * fabs(rm)) {
      const unsigned long long slot = atomicAdd(&A.hdr->n_tie, 1ull);
      if (A.tie_rows && (int64_t)slot < A.tie_cap) A.tie_rows[slot] = i;
    }
  }
}

// ---- stage 3: FP64 ranking of the candidates.  A row whose list overflowed
// takes the m-th best |rho| of its stored candidates (actual predecessors)
// as a tighter threshold and goes to the second pass.
template <int NU, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) rerank_kernel(KnnArgsV A) {
  extern __shared__ double ui_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* ui = ui_raw + (int64_t)wib * A.k;
  const int64_t warp = (int64_t)blockIdx.x * WARPS + wib;
  const int64_t total = (int64_t)gridDim.x * WARPS;
  const int K = A.m + 1;
  const double NEG = -1.0e300;
  for (int64_t i = warp; i < A.n; i += total) {
    const float4 info = A.rowinfo[i];
    if (info.w != 0.0f) continue;  // listed in stage 1
    const int nc_all = A.ccount[i];
    const int need = i < (int64_t)A.m ? (int)i : A.m;
    if (nc_all < need) {  // cannot happen when the bounds hold; searched exhaustively
      if (lane == 0) A.fbrows[atomicAdd(A.fbcount, 1ull)] = (int32_t)i;
      continue;
    }
    const int nc = min(nc_all, kVifCand);
    for (int c = lane; c < A.k; c += 32) ui[c] = A.U[i * A.k + c];
    __syncwarp();
    const double xi = A.xy[2 * i], yi = A.xy[2 * i + 1], ti = A.t[i], ri = A.r[i];
    double lr = NEG, thr = NEG;
    int lid = INT_MAX, count = 0;
    for (int b0 = 0; b0 < nc; b0 += 32) {
      const int q = b0 + lane;
      const int j = q < nc ? A.cand[i * kVifCand + q] : INT_MAX;
      const double rho = rho64_group<NU>(A, ui, xi, yi, ti, ri, q < nc ? (int64_t)j : -1, lane);
      unsigned mm = __ballot_sync(kFull, q < nc && (count < K || rho >= thr));
      while (mm) {
        const int src = __ffs(mm) - 1;
        mm &= mm - 1;
        const double cr = __shfl_sync(kFull, rho, src);
        const int cj = __shfl_sync(kFull, j, src);
        topk_insert(lane, K, cr, cj, lr, lid, count, thr);
      }
    }
    if (nc_all <= kVifCand) {
      write_row(A, lane, i, count, lr, lid);
    } else {
      const double tm = __shfl_sync(kFull, lr, A.m - 1);  // m-th best of the stored candidates
      if (lane == 0) {
        A.rowinfo[i] = make_float4(__double2float_rd(tm * (1.0 - 2e-12) * (double)info.y), info.y, info.z, 0.0f);
        A.fbrows[atomicAdd(A.fbcount, 1ull)] = (int32_t)i;
      }
    }
    __syncwarp();
  }
}

// ---- second pass over all predecessors of the listed rows: lane-local FP32
// screening with the same error bound as the tile pass (threshold from the
// row's record; -1 keeps every j), exact FP64 |rho| for the survivors.  One
// block of 8 warps per row: warp w takes the 32-wide j groups w, w + 8, ...
// into its own top-(m+1) list; warp 0 then merges the 8 lists (the merge
// keeps the same (|rho| desc, j asc) order, so the result does not depend
// on how j was split).
constexpr int kPass2Warps = 8;

template <int NU>
__global__ void __launch_bounds__(kPass2Warps * 32) pass2_kernel(KnnArgsV A) {
  extern __shared__ double ui_raw[];
  double* ui = ui_raw;
  float* uif = reinterpret_cast<float*>(ui_raw + A.k);
  __shared__ double mr[kPass2Warps][32];
  __shared__ int mid[kPass2Warps][32];
  __shared__ int mcnt[kPass2Warps];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int K = A.m + 1;
  const double NEG = -1.0e300;
  const double tiny = 1e-12 * A.th.sigma1sq;
  const float sig = (float)A.th.sigma1sq, cpar = (float)A.th.c;
  const float dotc = 24.0f * 1.05f * kU;
  const int64_t nrows = (int64_t)*A.fbcount;
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&A.hdr->n_fallback, (unsigned long long)nrows);
  for (int64_t w = blockIdx.x; w < nrows; w += gridDim.x) {
    const int64_t i = A.fbrows[w];
    __syncthreads();
    for (int c = threadIdx.x; c < A.k; c += kPass2Warps * 32) {
      ui[c] = A.U[i * A.k + c];
      uif[c] = A.Uf[i * A.k + c];
    }
    __syncthreads();
    const float4 info = A.rowinfo[i];
    const double xi = A.xy[2 * i], yi = A.xy[2 * i + 1], ti = A.t[i], ri = A.r[i];
    double lr = NEG, thr = NEG;
    int lid = INT_MAX, count = 0;
    for (int64_t j0 = (int64_t)wib * 32; j0 < i; j0 += kPass2Warps * 32) {
      const int64_t j = j0 + lane;
      double rho = NEG;
      if (j < i) {
        const double dxd = A.xy[2 * j] - xi, dyd = A.xy[2 * j + 1] - yi, dtd = A.t[j] - ti;
        bool pass = !(info.x > 0.0f) || !(dtd == floor(dtd) && fabs(dtd) < 16777216.0);
        if (!pass) {
          const float* uj = A.Uf + j * A.k;
          float hi = 0.f, lo = 0.f;
          for (int c0 = 0; c0 < A.k; c0 += 16) {
            float acc = 0.f;
            const int c1 = min(c0 + 16, A.k);
            for (int c = c0; c < c1; ++c) acc = fmaf(uif[c], uj[c], acc);
            const df t = df_two_sum(hi, acc);
            hi = t.hi;
            lo += t.lo;
          }
          const float dx = (float)dxd, dy = (float)dyd;
          float rel;
          const float C = cov32_err<NU>(A.th, dx, dy, (float)dtd, rel);
          const float R = fabsf(C - (hi + lo));
          const float4 cj = A.rowinfo[j];
          const float bound = 1.1f * fabsf(C) * (rel * kU + cpar * kU * (fabsf(dx) + fabsf(dy))) +
                              dotc * info.z * cj.z + 1.0e-33f * sig;
          const float rhs = info.x * cj.y;
          pass = R + 1.5f * bound + 4.0f * kU * (R + fabsf(rhs)) >= rhs;
        }
        if (pass) {
          const double* uj = A.U + j * A.k;
          double dot = 0.0;
          for (int c = 0; c < A.k; ++c) dot = fma(ui[c], uj[c], dot);
          const double Cd = cov64<NU>(A.th, -dxd, -dyd, -dtd);
          const double rj = A.r[j];
          rho = (ri > tiny && rj > tiny) ? fabs(Cd - dot) / sqrt(ri * rj) : 0.0;
        }
      }
      unsigned mm = __ballot_sync(kFull, rho > NEG && (count < K || rho >= thr));
      while (mm) {
        const int src = __ffs(mm) - 1;
        mm &= mm - 1;
        const double cr = __shfl_sync(kFull, rho, src);
        topk_insert(lane, K, cr, (int)(j0 + src), lr, lid, count, thr);
      }
    }
    mr[wib][lane] = lr;
    mid[wib][lane] = lid;
    if (lane == 0) mcnt[wib] = count;
    __syncthreads();
    if (wib == 0) {
      double fr = NEG, fthr = NEG;
      int fid = INT_MAX, fcount = 0;
      for (int q = 0; q < kPass2Warps; ++q) {
        const int cq = mcnt[q];
        for (int e = 0; e < cq; ++e) topk_insert(lane, K, mr[q][e], mid[q][e], fr, fid, fcount, fthr);
      }
      write_row(A, lane, i, fcount, fr, fid);
    }
  }
}

template <typename K>
void launch_rows_per_warp(K kern, const KnnArgsV& A, cudaStream_t st, size_t bytes_per_col = sizeof(double)) {
  constexpr int W = 4;
  const size_t smem = bytes_per_col * A.k * W;
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, W * 32, smem);
  kern<<<std::max(1, per) * sms, W * 32, smem, st>>>(A);
}

template <int NU>
vst_status knn_stages(const KnnArgsV& A, cudaStream_t st) {
  constexpr int W = 4;
  launch_rows_per_warp(tau_kernel<NU, W>, A, st);
  const int64_t T = (A.n + 127) / 128;
  const int64_t ntiles = T * (T + 1);  // 128-row tiles x 64-column tiles with j < i
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, filter_kernel<NU>, 256, 0);
  const int64_t grid = std::min<int64_t>(ntiles, (int64_t)std::max(1, per) * sms * 8);
  filter_kernel<NU><<<(unsigned)grid, 256, 0, st>>>(A, ntiles);
  launch_rows_per_warp(rerank_kernel<NU, W>, A, st);
  {
    const size_t smem = (sizeof(double) + sizeof(float)) * A.k;
    int dev = 0, sms2 = 0, per2 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms2, cudaDevAttrMultiProcessorCount, dev);
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(pass2_kernel<NU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, pass2_kernel<NU>, kPass2Warps * 32, smem);
    pass2_kernel<NU><<<std::max(1, per2) * sms2, kPass2Warps * 32, smem, st>>>(A);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VST_OK : cuda_fail(e, "VIF neighbour kernels");
}

}  // namespace

vst_status vif_knn(const vst_points* pts, const vst_theta* theta, int m, const vst_inducing* ind, int nu,
                   int32_t* nn, int32_t* nn_cnt, int64_t* tie_rows, int64_t tie_cap, char* base, WsHeader* hdr,
                   cudaStream_t st) {
  const int64_t n = pts->n;
  const int k = (int)ind->k;
  const WsLayout L0 = ws_layout(n, m, 0);
  const WsLayout L = ws_layout(n, m, k);
  char* vb = base + L.vif;
  const VifLayout V = vif_layout(n, m, k);
  // U (FP64) and r
  vst_status s = vif_lowrank(pts, theta, ind, nu, VST_FP64, vb, V, hdr, st);
  if (s != VST_OK) return s;
  // stage 1 input: the plain-correlation neighbours (their ties are not this search's)
  s = plain_knn(pts->xy, pts->t, n, theta, m, nn, nn_cnt, nullptr, 0, base, L0, hdr, n, 0, st);
  if (s != VST_OK) return s;
  cudaError_t e = cudaMemsetAsync(&hdr->n_tie, 0, sizeof(unsigned long long), st);
  KnnArgsV A{};
  A.xy = pts->xy;
  A.t = pts->t;
  A.n = n;
  A.m = m;
  A.k = k;
  A.th = dev_theta_vif(theta);
  A.U = reinterpret_cast<const double*>(vb + V.U);
  A.Uf = reinterpret_cast<const float*>(vb + V.Ap);
  A.r = reinterpret_cast<const double*>(vb + V.r);
  A.rowinfo = reinterpret_cast<float4*>(vb + V.tau);
  A.cand = reinterpret_cast<int32_t*>(vb + V.cand);
  A.ccount = reinterpret_cast<int32_t*>(vb + V.ccount);
  A.fbrows = reinterpret_cast<int32_t*>(vb + V.fbrows);
  A.fbcount = reinterpret_cast<unsigned long long*>(vb + V.fbcount);
  A.nn = nn;
  A.nn_cnt = nn_cnt;
  A.tie_rows = tie_rows;
  A.tie_cap = tie_rows ? tie_cap : 0;
  A.hdr = hdr;
  if (e == cudaSuccess) e = cudaMemsetAsync(A.ccount, 0, sizeof(int32_t) * (size_t)n, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(A.fbcount, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  narrow_kernel<<<(unsigned)std::min<int64_t>((n * k + 255) / 256, 65535), 256, 0, st>>>(A.U, n * k,
                                                                                         const_cast<float*>(A.Uf));
  ProfileScope ps(kProfKnn, st);
  return nu == 0 ? knn_stages<0>(A, st) : nu == 1 ? knn_stages<1>(A, st) : knn_stages<2>(A, st);
}

}  // namespace vst
