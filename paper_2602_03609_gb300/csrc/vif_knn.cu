// Residual-correlation neighbours of the VIF approximation (Sect. 4.3 with
// the correlation-based selection of Sect. 4.4.1 applied to the residual
// process): N(i) = the min(i, m) predecessors j < i with the largest
// |rho_ij| = |C_ij - U_i . U_j| / sqrt(r_i r_j), ties to the smaller index,
// exact in FP64.
//
// The search is exact but filtered:
//   1. a lower bound tau_i of the m-th largest |rho_ij|: the smallest |rho|
//      (FP64) over m actual predecessors, the plain-correlation neighbours;
//   2. a pass over all pairs j < i on the tensor cores (U U^T in BF16 tiles
//      of 128 x 256, FP32 accumulation, rfilter_tc_kernel below) that keeps
//      every j whose |rho| can reach tau_i: the test carries a rigorous
//      bound on the error of the BF16 dot product, of the FP32 covariance
//      functions and of the coordinate offsets, so every j with |rho_ij| >=
//      tau_i (1 - 2e-12) is kept;
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
#include <cmath>

#include <cuda_bf16.h>

#include "kernels.h"
#include "profile.h"
#include "umma.cuh"
#include "vif.h"
#include "workspace.h"

namespace vst {

vst_status fail(vst_status s, const char* fmt, ...);
vst_status cuda_fail(cudaError_t e, const char* where);
void launch_lag_table(const DevTheta& th, LagD* d, LagF* f, cudaStream_t st);
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
  // rerank over a list of rows instead of all rows (nullptr: all)
  const int32_t* rlist;
  int64_t rlist_n;
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

// the FP32 parameters the covariance below uses
struct CovF {
  float alpha, a, p, s1, c, gamma;
};
__device__ __forceinline__ CovF cov_f(const DevTheta& th) {
  return CovF{(float)th.alpha, (float)th.a, (float)th.p, (float)th.sigma1sq, (float)th.c, (float)th.gamma};
}

// covariance of Eq. (2) in FP32 (the same steps as the mixed form's cov32)
// and a bound on its relative error in units of u = 2^-24, from the error
// bounds of the FP32 functions (log2f 2 ulp, exp2f / expf / the approximate
// reciprocal square root 3 ulp, 1 ulp <= 2u; a subnormal squared distance is
// taken as 0, which changes C by a relative O(1e-38)) carried through each step: the lag powers (relative error of
// psi^-p grows with p |log2 psi| and the |2 alpha log2|u|| of the inner
// power), the Matern argument x = G h (its relative error enters C times x)
template <int NU>
__device__ __forceinline__ float cov32_err(const CovF& th, float dx, float dy, float u, float& rel) {
  const float au = fabsf(u);
  const float l2 = au > 0.f ? log2f(au) : 0.f;
  const float arg = 2.0f * th.alpha * l2;
  const float psi = au > 0.f ? fmaf(th.a, exp2f(arg), 1.0f) : 1.0f;
  const float lp = log2f(psi);
  const float P = th.s1 * exp2f(-th.p * lp);
  const float G = th.c * exp2f(-0.5f * th.gamma * lp);
  const float d2 = dx * dx + dy * dy;
  const float x = G * (d2 >= kFltMinNormal ? d2 * rsqrt_ftz(d2) : 0.f);
  const float C = P * matern_M<NU, float>(x, expf(-x));
  const float core = 4.3f * fabsf(arg) + 8.1f + 4.2f * fabsf(lp);
  const float relP = fabsf(th.p) * core + 8.0f;
  const float relx = 0.5f * fabsf(th.gamma) * core + 19.0f;
  rel = 1.25f * (relP + x * relx + 10.0f) + 16.0f;
  return C;
}
template <int NU>
__device__ __forceinline__ float cov32_err(const DevTheta& th, float dx, float dy, float u, float& rel) {
  return cov32_err<NU>(cov_f(th), dx, dy, u, rel);
}

// ---- stage 2 on the tensor cores.  The dot products U_i . U_j of the pairs
// j < i are the lower triangle of U U^T, a dense contraction over the k
// inducing points: BF16 tcgen05 tiles of 128 rows i x 256 columns j, K = k
// padded to 64, FP32 accumulation in tensor memory, with the threshold test
// fused into the epilogue.  Error of the BF16 dot: each U entry is rounded
// once to BF16 (relative 2^-9), a product of two rounded entries is exact in
// FP32, so the rounding contributes at most (2^-8 + 2^-18) sum_c |U_ic U_jc|;
// the tensor core's FP32 accumulation adds at most k 2^-22 of the same sum
// (a few ulps per MMA step, counted per term), and sum |U_ic U_jc| <=
// |U_i| |U_j|.  A pair is then kept under the same rule as the FP32 tile pass
// with this dot bound.  Most pairs are dismissed by a cheap test first:
// |dot| + bound + Cmax < tau_i s_i s_j, with Cmax = sigma1^2 psi(u_min)^-(delta
// + gamma) >= C_ij over the tile (u_min the smallest lag between the tiles'
// time ranges, M_nu <= 1); the rest evaluate C_ij and its error bound.
//
// Work: row tiles I of 128 rows and column tiles J of 256 with 256 J <=
// 128 I (every tile holds pairs j < i), grouped by 16 row tiles; inside a
// group the column tiles in increasing order, for each the group's row tiles
// (I >= 2 J).  A persistent CTA per SM takes the items round-robin, so the
// CTAs at work share a group's A tiles and a few B tiles in L2.
// Roles (320 threads): warp 0 issues the TMA loads (4-stage ring of 64-wide K
// blocks, 48 KiB each), warp 1 the MMAs (M = 128, N = 256, K = 16) into two
// TMEM accumulators of 256 columns (tile t in buffer t % 2), warps 2-9 the
// epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (= tile rows) and
// columns 128 ((w - 2) / 4) .. + 127, and the 256 epilogue threads load the
// tile's column records into shared memory (double-buffered by tile) first.
constexpr int kRfBM = kKnnTileRows, kRfBN = kKnnTileCols, kRfBK = 64, kRfStages = 4, kRfGroup = kKnnGroup;
constexpr int kRfThreads = 320;
constexpr uint64_t kRfWaitNs = 2000000000ull;  // 2 s per wait
constexpr int kRfBins = 256;                    // |rho| histogram of the later rounds
struct RfShape {
  static constexpr int A_BYTES = kRfBM * kRfBK * 2;
  static constexpr int B_BYTES = kRfBN * kRfBK * 2;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int COL_BYTES = 2 * kRfBN * (8 + 16);  // per column (s, nu) and (x, y, t, s), 2 buffers
  static constexpr int BAR_BYTES = 256;
  static constexpr int SMEM = kRfStages * STAGE + COL_BYTES + BAR_BYTES + 1024;
  static_assert(STAGE % 1024 == 0, "stage alignment");
  static_assert(SMEM <= 232448, "shared memory");
};

struct RfArgs {
  int64_t n;
  int k, kb;            // inducing points, 64-wide K blocks
  int T;                // row tiles
  int ngroups;
  const int64_t* gcum;  // [ngroups + 1] items before each group
  const double2* tb128; // per row tile: (t_min, t_max)
  const double2* tb256; // per column tile
  const int* times_exact;
  const LagF* lagf;     // FP32 lag table (P = sigma1^2 psi^-(delta+gamma))
  float epsd;           // relative bound of the BF16 dot product
  // gathered mode (rows != nullptr): the A operand holds the U rows of the
  // listed rows (nrows of them, tile I = list entries 128 I ..); items are
  // (I, J) for I < nt and J < nj, J from the last column tile down
  const int32_t* rows;
  int64_t nrows;
  int nt, nj;
  int* hist;  // [nrows][kRfBins] counts of the approximate |rho| of each row's candidates
  int* dmax;  // [nrows] largest approximation error (float bits)
  const double2* tbg;   // per gathered row tile: (t_min, t_max)
};

__device__ __forceinline__ void rf_item(const RfArgs& R, int64_t w, int& I, int& J) {
  if (R.rows) {
    // the latest columns first: a row's most correlated predecessors tend to
    // be recent (time-stratified order), and the candidates that fit in the
    // row's slots give the next round its threshold
    I = (int)(w % R.nt);
    J = R.nj - 1 - (int)(w / R.nt);
    return;
  }
  int lo = 0, hi = R.ngroups;  // largest G with gcum[G] <= w
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (R.gcum[mid] <= w) lo = mid; else hi = mid;
  }
  const int G = lo;
  int64_t r = w - R.gcum[G];
  const int I0 = G * kRfGroup, I1 = min(I0 + kRfGroup, R.T);
  const int F = I1 - I0, Jf = I0 / 2;
  if (r < (int64_t)(Jf + 1) * F) {
    J = (int)(r / F);
    I = I0 + (int)(r % F);
    return;
  }
  r -= (int64_t)(Jf + 1) * F;
  int j = Jf + 1;
  for (;;) {
    const int c = I1 - 2 * j;
    if (r < c) break;
    r -= c;
    ++j;
  }
  J = j;
  I = 2 * j + (int)r;
}

// Exact test of one pair that passed the cheap test: FP32 covariance with its
// error bound, the BF16 dot's bound, and the same keep rule as the FP32
// passes; appends j to row i's candidates.  Not inlined: one copy of the code
// serves the 32 columns of a chunk.
template <int NU>
__device__ __noinline__ void rf_exact(CovF cf, float dot, float4 cm, float nuj, float xi, float yi, float ti,
                                      float offi, float thr, float si, float eu, int texact, int64_t i, int j,
                                      int32_t* ccount, int32_t* cand, int* hist, int* dmax) {
  const float rhs = thr * cm.w;
  const float db = eu * nuj;
  bool keep = !texact;
  float Rv = 0.f, bound = 0.f;
  if (!keep) {
    float rel;
    const float C = cov32_err<NU>(cf, xi - cm.x, yi - cm.y, ti - cm.z, rel);
    Rv = fabsf(C - dot);
    const float offs = offi + fabsf(cm.x) + fabsf(cm.y);
    bound = 1.1f * fabsf(C) * (rel * kU + cf.c * 2.0f * kU * offs) + db + 1.0e-33f * cf.s1;
    keep = Rv + 1.5f * bound + 4.0f * kU * (Rv + fabsf(rhs)) >= rhs;
  }
  if (keep) {
    const int slot = atomicAdd(&ccount[i], 1);
    if (slot < kVifCand) cand[i * kVifCand + slot] = (int32_t)j;
    if (hist && texact) {
      // later rounds: the approximate |rho| of the candidate in one of
      // kRfBins bins over [0, 1], and the largest error of such an
      // approximation for the row (|rho - rho^| <= (1.5 bound + rounding) / (s_i s_j))
      const float ss = si * cm.w;
      if (ss > 0.f) {
        const float rh = Rv / ss;
        const float dl = (1.5f * bound + 8.0f * kU * (Rv + rhs)) / ss * 1.01f;
        const int bin = min(kRfBins - 1, max(0, (int)(rh * (float)kRfBins)));
        atomicAdd(&hist[bin], 1);
        atomicMax(dmax, __float_as_int(dl));
      }
    }
  }
}

template <int NU>
__global__ void __launch_bounds__(kRfThreads, 1)
    rfilter_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, KnnArgsV A,
                      RfArgs R) {
  extern __shared__ unsigned char rf_smem[];
  const uint32_t raw = umma::smem_u32(rf_smem);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = rf_smem + (base - raw);
  float4* colX = reinterpret_cast<float4*>(gbase + kRfStages * RfShape::STAGE);  // [2][256] (x, y, t, s)
  float2* colS = reinterpret_cast<float2*>(colX + 2 * kRfBN);                  // [2][256] (s, nu)
  uint64_t* full = reinterpret_cast<uint64_t*>(gbase + kRfStages * RfShape::STAGE + RfShape::COL_BYTES);
  uint64_t* empty = full + kRfStages;
  uint64_t* accf = empty + kRfStages;  // [2] accumulator filled
  uint64_t* acce = accf + 2;           // [2] accumulator drained (8 epilogue warps)
  uint64_t* done = acce + 2;           // every MMA of this CTA finished
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile uint32_t* epi_fail = tslot + 1;  // an epilogue warp's wait ran out

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t items = R.rows ? (int64_t)R.nt * R.nj : R.gcum[R.ngroups];
  if (threadIdx.x == 0) {
    for (int s = 0; s < kRfStages; ++s) {
      umma::mbar_init(&full[s], 1);
      umma::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      umma::mbar_init(&accf[b], 1);
      umma::mbar_init(&acce[b], 8);
    }
    umma::mbar_init(done, 1);
    *epi_fail = 0u;
    umma::fence_mbar_init();
  }
  if (warp == 0) {
    umma::tmem_alloc(umma::smem_u32(tslot), 512);
    umma::tmem_relinquish();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *tslot;
  bool ok = true;
  auto warp_wait = [&](uint64_t* bar, uint32_t parity) {
    bool d = true;
    if (lane == 0) d = umma::mbar_wait(bar, parity, kRfWaitNs);
    return __shfl_sync(0xffffffffu, d ? 1 : 0, 0) != 0;
  };

  if (warp == 0) {
    // producer
    int64_t cnt = 0;
    for (int64_t w = blockIdx.x; w < items && ok; w += gridDim.x) {
      int I, J;
      rf_item(R, w, I, J);
      for (int kb = 0; kb < R.kb; ++kb, ++cnt) {
        const int s = (int)(cnt % kRfStages);
        const uint32_t use = (uint32_t)(cnt / kRfStages);
        if (use > 0 && !warp_wait(&empty[s], (use - 1) & 1u)) {
          ok = false;
          break;
        }
        if (lane == 0) {
          umma::mbar_arrive_expect_tx(&full[s], RfShape::STAGE);
          const uint32_t sa = base + s * RfShape::STAGE, sb = sa + RfShape::A_BYTES;
          umma::tma_load_2d(sa, &tmA, kb * kRfBK, I * kRfBM, &full[s]);
          umma::tma_load_2d(sb, &tmB, kb * kRfBK, J * kRfBN, &full[s]);
        }
        __syncwarp();
      }
    }
    if (!ok) {
      // let the loads still in flight land before the CTA's shared memory goes
      for (int64_t c = cnt - kRfStages < 0 ? 0 : cnt - kRfStages; c < cnt; ++c)
        warp_wait(&full[c % kRfStages], (uint32_t)(c / kRfStages) & 1u);
    }
  } else if (warp == 1) {
    // MMA issuer
    constexpr uint32_t idesc = umma::idesc_bf16_f32(kRfBM, kRfBN);
    int64_t cnt = 0, it = 0;
    for (int64_t w = blockIdx.x; w < items && ok; w += gridDim.x, ++it) {
      const int b = (int)(it & 1);
      if (it >= 2 && !warp_wait(&acce[b], (uint32_t)((it >> 1) - 1) & 1u)) {
        ok = false;
        break;
      }
      umma::fence_after_sync();
      const uint32_t tb = tmem + (uint32_t)(b * kRfBN);
      for (int kb = 0; kb < R.kb; ++kb, ++cnt) {
        const int s = (int)(cnt % kRfStages);
        if (!warp_wait(&full[s], (uint32_t)(cnt / kRfStages) & 1u)) {
          ok = false;
          break;
        }
        umma::fence_after_sync();
        if (lane == 0) {
          const uint32_t sa = base + s * RfShape::STAGE, sb = sa + RfShape::A_BYTES;
#pragma unroll
          for (int kk = 0; kk < kRfBK / 16; ++kk)
            umma::mma_bf16(tb, umma::desc_kmajor_sw128(sa + kk * 32), umma::desc_kmajor_sw128(sb + kk * 32), idesc,
                           (kb | kk) != 0 ? 1u : 0u);
          umma::mma_commit(&empty[s]);
        }
        __syncwarp();
      }
      if (!ok) break;
      if (lane == 0) umma::mma_commit(&accf[b]);
      __syncwarp();
    }
    // every MMA this thread issued has finished before the tensor memory is freed
    if (lane == 0) umma::mma_commit(done);
    __syncwarp();
    if (!warp_wait(done, 0)) ok = false;
  } else {
    // epilogue: 8 warps, 256 threads
    const int et = threadIdx.x - 64;
    const int q4 = warp & 3, half = (warp - 2) >> 2;
    const int r = q4 * 32 + lane;
    const float sig = (float)A.th.sigma1sq;
    const CovF cf = cov_f(A.th);
    const int texact = *R.times_exact;
    int64_t it = 0;
    for (int64_t w = blockIdx.x; w < items; w += gridDim.x, ++it) {
      int I, J;
      rf_item(R, w, I, J);
      const int b = (int)(it & 1);
      const int64_t i0 = R.rows ? (int64_t)R.rows[(int64_t)I * kRfBM] : (int64_t)I * kRfBM, j0 = (int64_t)J * kRfBN;
      const double X0 = A.xy[2 * i0], Y0 = A.xy[2 * i0 + 1];
      // this thread's column record: offsets from the row tile's first point
      {
        const int64_t j = j0 + et;
        float4 ca = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 cs = make_float2(0.f, 0.f);
        if (j < A.n) {
          const float4 ij = A.rowinfo[j];
          ca = make_float4((float)(A.xy[2 * j] - X0), (float)(A.xy[2 * j + 1] - Y0), (float)A.t[j], ij.y);
          cs = make_float2(ij.y, ij.z);
        }
        colX[b * kRfBN + et] = ca;
        colS[b * kRfBN + et] = cs;
      }
      // bound of C over the tile pair from the two time ranges
      float cmax = sig;
      if (texact) {
        const double2 ti = R.rows ? R.tbg[I] : R.tb128[I], tj = R.tb256[J];
        const double u = fmax(0.0, fmax(ti.x - tj.y, tj.x - ti.y));
        const int lag = (int)fmin(u, (double)(kLagTab - 1));
        cmax = R.lagf[lag].P * (1.0f + 1.0e-5f) + 1.0e-30f;
      }
      const int64_t gi = (int64_t)I * kRfBM + r;  // gathered mode: list entry
      const int64_t i = R.rows ? (gi < R.nrows ? (int64_t)R.rows[gi] : A.n) : i0 + r;
      float4 ri = make_float4(0.f, 0.f, 0.f, 1.f);
      float xi = 0.f, yi = 0.f, tiv = 0.f;
      if (i < A.n) {
        ri = A.rowinfo[i];
        xi = (float)(A.xy[2 * i] - X0);
        yi = (float)(A.xy[2 * i + 1] - Y0);
        tiv = (float)A.t[i];
      }
      const bool rowon = i < A.n && ri.w == 0.0f;
      const float offi = fabsf(xi) + fabsf(yi);
      const float eu = R.epsd * ri.z;
      const int climit = (int)(i - j0);  // columns c < climit have j < i
      int* hrow = (R.rows && gi < R.nrows) ? R.hist + gi * kRfBins : nullptr;
      int* drow = hrow ? R.dmax + gi : nullptr;
      // the eight warps pass the same barriers: a warp whose wait ran out
      // says so here, and all of them stop together after the barrier
      if (!ok && lane == 0) *epi_fail = 1u;
      asm volatile("bar.sync 1, 256;" ::: "memory");  // column records written
      if (*epi_fail != 0u) break;
      if (!warp_wait(&accf[b], (uint32_t)(it >> 1) & 1u)) {
        ok = false;
        continue;
      }
      umma::fence_after_sync();
      const uint32_t ta = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(b * kRfBN + half * 128);
#pragma unroll 1
      for (int ch = 0; ch < 4; ++ch) {
        uint32_t v[32];
        __syncwarp();
        umma::tmem_ld_32x32b_x32(ta + ch * 32, v);
        umma::tmem_wait_ld();
        if (ch == 3) {
          // the buffer is free for the MMAs once its last columns are read
          umma::fence_before_sync();
          __syncwarp();
          if (lane == 0) umma::mbar_arrive(&acce[b]);
        }
        // cheap test for the 32 columns, a bit per column that may qualify
        const int cb0 = half * 128 + ch * 32;
        uint32_t mask = 0u;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const float2 sn = colS[b * kRfBN + cb0 + q];
          const float rhs = ri.x * sn.x;
          const float ub = fabsf(__uint_as_float(v[q])) + fmaf(eu, sn.y, cmax);
          mask |= (ub * (1.0f + 16.0f * kU) >= rhs && cb0 + q < climit) ? (1u << q) : 0u;
        }
        if (!rowon) mask = 0u;
        if (__any_sync(kFull, mask != 0u)) {
#pragma unroll
          for (int q = 0; q < 32; ++q)
            if (mask & (1u << q))
              rf_exact<NU>(cf, __uint_as_float(v[q]), colX[b * kRfBN + cb0 + q], colS[b * kRfBN + cb0 + q].y, xi, yi,
                           tiv, offi, ri.x, ri.y, eu, texact, i, (int)j0 + cb0 + q, A.ccount, A.cand, hrow, drow);
        }
      }
    }
  }
  if (!ok) report_error(A.hdr, VST_ETIMEOUT, (int64_t)blockIdx.x);
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tmem, 512);
}

// items before each group of kRfGroup row tiles (one thread)
__global__ void rf_groups_kernel(int T, int ngroups, int64_t* gcum) {
  int64_t acc = 0;
  for (int G = 0; G < ngroups; ++G) {
    gcum[G] = acc;
    const int I0 = G * kRfGroup, I1 = min(I0 + kRfGroup, T);
    for (int I = I0; I < I1; ++I) acc += I / 2 + 1;
  }
  gcum[ngroups] = acc;
}

// per tile of `rows` consecutive points: (t_min, t_max); one warp per tile
__global__ void tile_times_kernel(const double* t, int64_t n, int rows, int64_t ntiles, double2* out) {
  const int lane = threadIdx.x & 31;
  const int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (tile >= ntiles) return;
  double mn = 1.0e300, mx = -1.0e300;
  for (int64_t q = tile * rows + lane; q < min(n, (tile + 1) * rows); q += 32) {
    mn = fmin(mn, t[q]);
    mx = fmax(mx, t[q]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mn = fmin(mn, __shfl_xor_sync(kFull, mn, o));
    mx = fmax(mx, __shfl_xor_sync(kFull, mx, o));
  }
  if (lane == 0) out[tile] = make_double2(mn, mx);
}

// (t_min, t_max) of each tile of 128 listed rows; one warp per tile
__global__ void tile_times_list_kernel(const double* t, const int32_t* rows, int64_t nrows, int64_t ntiles,
                                       double2* out) {
  const int lane = threadIdx.x & 31;
  const int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (tile >= ntiles) return;
  double mn = 1.0e300, mx = -1.0e300;
  for (int64_t q = tile * kRfBM + lane; q < min(nrows, (tile + 1) * kRfBM); q += 32) {
    const double v = t[rows[q]];
    mn = fmin(mn, v);
    mx = fmax(mx, v);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mn = fmin(mn, __shfl_xor_sync(kFull, mn, o));
    mx = fmax(mx, __shfl_xor_sync(kFull, mx, o));
  }
  if (lane == 0) out[tile] = make_double2(mn, mx);
}

// Rows of a list of the previous round: those without a defined residual
// correlation (w != 0) appended to zlist (cnt[4]); those whose candidates
// overflowed, now with a tighter threshold, to the gathered round's list, or
// after the last round appended to the exhaustive list; counts and the
// largest gathered row in cnt[0..2].  One block.
__global__ void fb_split_kernel(const int32_t* fb, const unsigned long long* fbcount, const float4* rowinfo,
                                int last, int32_t* glist, int32_t* xlist, int32_t* zlist, unsigned long long* cnt) {
  const int64_t nfb = (int64_t)*fbcount;
  for (int64_t q = threadIdx.x; q < nfb; q += blockDim.x) {
    const int32_t i = fb[q];
    if (rowinfo[i].w != 0.0f) {
      zlist[atomicAdd(&cnt[4], 1ull)] = i;
    } else if (!last) {
      glist[atomicAdd(&cnt[0], 1ull)] = i;
      atomicMax(&cnt[2], (unsigned long long)i);
    } else {
      xlist[atomicAdd(&cnt[1], 1ull)] = i;
    }
  }
}

// Rows without a defined residual correlation (r_i <= 1e-12 sigma1^2, an
// inducing point on top of the point): |rho_ij| = 0 for every j, so the
// neighbours are the min(i, m) smallest indices and the cut-off is a tie
// whenever i > m.  One thread per row.
__global__ void zero_corr_rows_kernel(KnnArgsV A, const int32_t* rows, const unsigned long long* count) {
  const int64_t nz = (int64_t)*count;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nz; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = rows[q];
    const int c = i < (int64_t)A.m ? (int)i : A.m;
    for (int p = 0; p < A.m; ++p) A.nn[i * A.m + p] = p < c ? p : -1;
    A.nn_cnt[i] = c;
    if (i > (int64_t)A.m && A.m > 0) {
      const unsigned long long slot = atomicAdd(&A.hdr->n_tie, 1ull);
      if (A.tie_rows && (int64_t)slot < A.tie_cap) A.tie_rows[slot] = i;
    }
  }
}

// Rows of a gathered round whose candidates overflowed their slots: the
// histogram of the approximate |rho| gives a threshold that m of them reach
// (the lower edge of the bin holding the m-th largest, less the largest
// approximation error), raised into the row's record if it is the larger.
// One warp per row.
__global__ void hist_threshold_kernel(const int32_t* rows, int64_t nrows, const int* hist, const int* dmax,
                                      const int32_t* ccount, int m, float4* rowinfo) {
  const int lane = threadIdx.x & 31;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= nrows) return;
  const int64_t i = rows[w];
  if (ccount[i] <= kVifCand || m <= 0) return;
  // bins 8 lane .. 8 lane + 7; the candidates in the bins of higher lanes
  int c[8], tot = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    c[u] = hist[w * kRfBins + lane * 8 + u];
    tot += c[u];
  }
  int incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_down_sync(kFull, incl, o);
    if (lane + o < 32) incl += v;
  }
  const int above = incl - tot;
  int bin = -1;
  int acc = above;
#pragma unroll
  for (int u = 7; u >= 0; --u) {
    acc += c[u];
    if (bin < 0 && acc >= m) bin = lane * 8 + u;
  }
  // the highest bin over the lanes where the count reaches m
  int best = bin;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(kFull, best, o));
  if (lane == 0 && best >= 0) {
    const float4 info = rowinfo[i];
    const float lo = (float)best / (float)kRfBins - __int_as_float(dmax[w]);
    if (lo > 0.f) {
      const float thr = __double2float_rd((double)lo * (1.0 - 2e-12) * (double)info.y * (1.0 - 1e-6));
      if (thr > info.x) rowinfo[i] = make_float4(thr, info.y, info.z, info.w);
    }
  }
}

// BF16 U rows of the listed rows [nrows][k64] (zero padded); candidate
// counts of those rows reset
__global__ void gather_bf16_kernel(const double* U, const int32_t* rows, int64_t nrows, int k, int k64,
                                   __nv_bfloat16* Ug, int32_t* ccount) {
  const int64_t total = nrows * (int64_t)k64;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = q / k64;
    const int c = (int)(q - e * k64);
    const int64_t i = rows[e];
    Ug[q] = c < k ? __double2bfloat16(U[i * k + c]) : __float2bfloat16(0.0f);
    if (c == 0) ccount[i] = 0;
  }
}

// 1 if every time is an integer day with |t| < 2^24 (exact in FP32)
__global__ void times_exact_kernel(const double* t, int64_t n, int* flag) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const double v = t[q];
    if (!(v == floor(v) && fabs(v) < 16777216.0)) atomicAnd(flag, 0);
  }
}

// U (FP64 [n][k]) -> BF16 [n][k64] (k64 = k rounded up to 64, zero padded)
__global__ void u_bf16_kernel(const double* U, int64_t n, int k, int k64, __nv_bfloat16* Ub) {
  const int64_t total = n * (int64_t)k64;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / k64;
    const int c = (int)(q - i * k64);
    Ub[q] = c < k ? __double2bfloat16(U[i * k + c]) : __float2bfloat16(0.0f);
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
  const int64_t nrows = A.rlist ? A.rlist_n : A.n;
  for (int64_t q = warp; q < nrows; q += total) {
    const int64_t i = A.rlist ? (int64_t)A.rlist[q] : q;
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
        const float thr = __double2float_rd(tm * (1.0 - 2e-12) * (double)info.y);
        A.rowinfo[i] = make_float4(fmaxf(thr, A.rowinfo[i].x), info.y, info.z, 0.0f);
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

// Scratch of stage 2 (its own workspace region, knn_scratch_bytes): item
// counts per group, per-tile time ranges, the times flag, the two row lists
// of the second round and their counters.
struct RfScratch {
  int64_t* gcum;
  double2 *tb128, *tb256, *tbg;
  int* texact;
  int32_t *glist, *xlist, *plist, *zlist;
  int *hist, *dmax;  // per gathered row: |rho| histogram and largest error
  // [0] gathered rows, [1] exhaustive rows, [2] largest gathered row,
  // [3] rows of plist, [4] rows without a defined residual correlation
  unsigned long long* cnt;
  int T, T2, ngroups;
};
static RfScratch rf_scratch(char* vb, const VifLayout& V, int64_t n) {
  RfScratch S{};
  S.T = (int)((n + kRfBM - 1) / kRfBM);
  S.T2 = (int)((n + kRfBN - 1) / kRfBN);
  S.ngroups = (S.T + kRfGroup - 1) / kRfGroup;
  size_t off = V.kscr;
  auto take = [&](size_t bytes) {
    char* p = vb + off;
    off += align256(bytes);
    return p;
  };
  S.gcum = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * (S.ngroups + 1)));
  S.tb128 = reinterpret_cast<double2*>(take(sizeof(double2) * S.T));
  S.tb256 = reinterpret_cast<double2*>(take(sizeof(double2) * S.T2));
  S.tbg = reinterpret_cast<double2*>(take(sizeof(double2) * (std::min<int64_t>(n, kVifGather) / kRfBM + 1)));
  S.texact = reinterpret_cast<int*>(take(sizeof(int)));
  S.cnt = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * 8));
  S.glist = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * n));
  S.xlist = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * n));
  S.plist = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * n));
  S.zlist = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * n));
  S.hist = reinterpret_cast<int*>(take(sizeof(int) * std::min<int64_t>(n, kVifGather) * kRfBins));
  S.dmax = reinterpret_cast<int*>(take(sizeof(int) * std::min<int64_t>(n, kVifGather)));
  return S;
}

static int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

template <int NU>
vst_status rf_launch(const KnnArgsV& A, const RfArgs& R, const void* Aop, int64_t arows, const void* Bop, int k64,
                     cudaStream_t st) {
  CUtensorMap ta, tb;
  if (!tc_make_map_bf16(&ta, Aop, (uint64_t)arows, (uint64_t)k64, kRfBM) ||
      !tc_make_map_bf16(&tb, Bop, (uint64_t)A.n, (uint64_t)k64, kRfBN))
    return fail(VST_ECUDA, "residual filter: tensor map encoding failed");
  auto kern = rfilter_tc_kernel<NU>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, RfShape::SMEM);
  if (e != cudaSuccess) return cuda_fail(e, "residual filter attributes");
  ProfileScope ps(kProfVifFilter, st);
  kern<<<sm_count(), kRfThreads, RfShape::SMEM, st>>>(ta, tb, A, R);
  e = cudaGetLastError();
  return e == cudaSuccess ? VST_OK : cuda_fail(e, "residual filter kernel");
}

// stage 2 on the tensor cores over the lower triangle (rfilter_tc_kernel),
// with its inputs: U in BF16 after the FP32 copy in the operand region,
// per-tile time ranges and item counts in the scratch
template <int NU>
vst_status tc_filter(const KnnArgsV& A, char* vb, const VifLayout& V, const LagF* lagf, const RfScratch& S,
                     RfArgs& R, __nv_bfloat16*& Ub, cudaStream_t st) {
  const int64_t n = A.n;
  const int k = A.k, k64 = (k + 63) / 64 * 64;
  Ub = reinterpret_cast<__nv_bfloat16*>(vb + V.Ap + align256(sizeof(float) * (size_t)n * k));
  const int sms = sm_count();
  cudaError_t e = cudaMemsetAsync(S.texact, 0xff, sizeof(int), st);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  times_exact_kernel<<<sms * 4, 256, 0, st>>>(A.t, n, S.texact);
  tile_times_kernel<<<(unsigned)((S.T * 32 + 255) / 256), 256, 0, st>>>(A.t, n, kRfBM, S.T, S.tb128);
  tile_times_kernel<<<(unsigned)((S.T2 * 32 + 255) / 256), 256, 0, st>>>(A.t, n, kRfBN, S.T2, S.tb256);
  rf_groups_kernel<<<1, 1, 0, st>>>(S.T, S.ngroups, S.gcum);
  u_bf16_kernel<<<sms * 8, 256, 0, st>>>(A.U, n, k, k64, Ub);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "filter set-up kernels");
  R = RfArgs{};
  R.n = n;
  R.k = k;
  R.kb = k64 / kRfBK;
  R.T = S.T;
  R.ngroups = S.ngroups;
  R.gcum = S.gcum;
  R.tb128 = S.tb128;
  R.tb256 = S.tb256;
  R.times_exact = S.texact;
  R.lagf = lagf;
  // BF16 rounding of both factors plus the FP32 accumulation, 5% margin
  R.epsd = (float)(1.05 * (std::ldexp(1.0, -8) + std::ldexp(1.0, -18) + (double)k64 * std::ldexp(1.0, -22)));
  return rf_launch<NU>(A, R, Ub, n, Ub, k64, st);
}

template <int NU>
vst_status knn_stages(KnnArgsV A, char* vb, const VifLayout& V, const LagF* lagf, cudaStream_t st) {
  constexpr int W = 4;
  const int64_t n = A.n;
  const int k64 = (A.k + 63) / 64 * 64;
  launch_rows_per_warp(tau_kernel<NU, W>, A, st);
  if (n <= 1) return VST_OK;
  const RfScratch S = rf_scratch(vb, V, n);
  RfArgs R;
  __nv_bfloat16* Ub = nullptr;
  vst_status s = tc_filter<NU>(A, vb, V, lagf, S, R, Ub, st);
  if (s != VST_OK) return s;
  launch_rows_per_warp(rerank_kernel<NU, W>, A, st);
  // later rounds: rows whose candidates overflowed, with the tighter
  // threshold rerank gave them (the m-th best of their stored candidates),
  // screened again on the tensor cores against all predecessors, in batches
  // of gathered rows; a round's overflow feeds the next, whose threshold is
  // the larger of the m-th best stored candidate and the bound from the
  // round's histogram of approximate |rho| (hist_threshold_kernel).
  // Rows without a defined residual correlation take the first predecessors
  // (every |rho| is 0); those still overflowing after the last round go to
  // the exhaustive pass.
  constexpr int kRounds = 8;
  KnnArgsV A2 = A;
  __nv_bfloat16* Ug = reinterpret_cast<__nv_bfloat16*>(vb + V.gath);
  const int sms = sm_count();
  int32_t* fb_in = A.fbrows;
  unsigned long long* fbc_in = A.fbcount;
  cudaError_t e = cudaMemsetAsync(S.cnt, 0, sizeof(unsigned long long) * 8, st);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  for (int round = 0; round <= kRounds; ++round) {
    const int last = round == kRounds;
    e = cudaMemsetAsync(S.cnt, 0, sizeof(unsigned long long), st);                // gathered rows
    if (e == cudaSuccess) e = cudaMemsetAsync(S.cnt + 2, 0, sizeof(unsigned long long), st);  // largest row
    if (e != cudaSuccess) return cuda_fail(e, "memset");
    fb_split_kernel<<<1, 1024, 0, st>>>(fb_in, fbc_in, A.rowinfo, last, S.glist, S.xlist, S.zlist, S.cnt);
    unsigned long long h[4] = {0, 0, 0, 0};
    e = cudaMemcpyAsync(h, S.cnt, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "second-round counts");
    const int64_t ng = (int64_t)h[0];
    if (ng == 0) break;
    // this round's overflow goes to the other list
    int32_t* fb_out = fb_in == A.fbrows ? S.plist : A.fbrows;
    unsigned long long* fbc_out = fb_in == A.fbrows ? S.cnt + 3 : A.fbcount;
    e = cudaMemsetAsync(fbc_out, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_fail(e, "memset");
    A2.fbrows = fb_out;
    A2.fbcount = fbc_out;
    for (int64_t b0 = 0; b0 < ng; b0 += kVifGather) {
      const int64_t nb = std::min<int64_t>(kVifGather, ng - b0);
      const int32_t* rows = S.glist + b0;
      gather_bf16_kernel<<<sms * 8, 256, 0, st>>>(A.U, rows, nb, A.k, k64, Ug, A.ccount);
      e = cudaMemsetAsync(S.hist, 0, sizeof(int) * nb * kRfBins, st);
      if (e == cudaSuccess) e = cudaMemsetAsync(S.dmax, 0, sizeof(int) * nb, st);
      if (e != cudaSuccess) return cuda_fail(e, "memset");
      const int nt = (int)((nb + kRfBM - 1) / kRfBM);
      tile_times_list_kernel<<<(unsigned)((nt * 32 + 255) / 256), 256, 0, st>>>(A.t, rows, nb, nt, S.tbg);
      e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e, "second-round set-up");
      RfArgs R2 = R;
      R2.rows = rows;
      R2.nrows = nb;
      R2.nt = nt;
      R2.nj = (int)(((int64_t)h[2] + kRfBN - 1) / kRfBN);  // columns j < the largest listed row
      R2.tbg = S.tbg;
      R2.hist = S.hist;
      R2.dmax = S.dmax;
      if (R2.nj > 0) {
        s = rf_launch<NU>(A, R2, Ug, nb, Ub, k64, st);
        if (s != VST_OK) return s;
      }
      hist_threshold_kernel<<<(unsigned)((nb * 32 + 255) / 256), 256, 0, st>>>(rows, nb, S.hist, S.dmax, A.ccount,
                                                                               A.m, A.rowinfo);
      A2.rlist = rows;
      A2.rlist_n = nb;
      launch_rows_per_warp(rerank_kernel<NU, W>, A2, st);
    }
    fb_in = fb_out;
    fbc_in = fbc_out;
  }
  zero_corr_rows_kernel<<<sms, 256, 0, st>>>(A, S.zlist, S.cnt + 4);
  A2.fbrows = S.xlist;
  A2.fbcount = S.cnt + 1;
  {
    A2.rlist = nullptr;
    A2.rlist_n = 0;
    const size_t smem = (sizeof(double) + sizeof(float)) * A.k;
    int per2 = 0;
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(pass2_kernel<NU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, pass2_kernel<NU>, kPass2Warps * 32, smem);
    pass2_kernel<NU><<<std::max(1, per2) * sms, kPass2Warps * 32, smem, st>>>(A2);
  }
  e = cudaGetLastError();
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
  // FP32 lag table (its amplitudes bound the covariance of a tile pair)
  LagD* lagd = reinterpret_cast<LagD*>(base + L.lagd);
  LagF* lagf = reinterpret_cast<LagF*>(base + L.lagf);
  launch_lag_table(A.th, lagd, lagf, st);
  ProfileScope ps(kProfKnn, st);
  return nu == 0   ? knn_stages<0>(A, vb, V, lagf, st)
         : nu == 1 ? knn_stages<1>(A, vb, V, lagf, st)
                   : knn_stages<2>(A, vb, V, lagf, st);
}

}  // namespace vst
