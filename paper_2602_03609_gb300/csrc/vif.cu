// VIF: the Vecchia-inducing-point full-scale approximation (Sect. 4.3).
//
//   Sigma~_VIF = U U^T + B^{-1} D B^{-T},  U = Sigma_nk L_kk^{-T},  L_kk L_kk^T = Sigma_kk,
//
// with (B, D) the Vecchia factor of the residual R + sigma^2 I,
// R = Sigma - U U^T, and neighbours chosen by the residual correlation
// |R_ij| / sqrt(R_ii R_jj).  The NLL uses the Sherman-Woodbury-Morrison
// identity (the complexity remark closing Sect. 4.3):
//   W = D^{-1/2} B U,  e = D^{-1/2} B y,  M = I + W^T W,
//   log det = sum_i log D_i + log det M,
//   quad    = e^T e - (W^T e)^T M^{-1} (W^T e).
//
// Kernels (T = double for the FP64 form, float for the mixed form):
//   kk_kernel            Sigma_kk in FP64
//   chol_diag/trsm/trail blocked FP64 Cholesky (in place, lower): 32 x 32 diagonal
//                        block in one warp, panel rows by forward substitution,
//                        tiled trailing update
//   trinv_kernel         L^{-1}, FP64, one warp per column
//   snk64_kernel, gemm_nt U = Sigma_nk L^{-T} (FP64: Sigma_nk once, then the dense tile GEMM)
//   rdiag_kernel<T>      r_i = sigma1^2 - ||U_i||^2
//   gram64_kernel        FP64: per-row U_p . U_q over the local block (fed to the row kernel)
//   gram_delta_kernel    mixed: per-row U_p . U_q, accumulated without cancellation
//                        (blocks of 8, 16, 24 positions; 32-position blocks go to the
//                        tensor-core kernel of vif_gram_tc.cu)
//   wvec_kernel<T>       rows of [W e] and sum log D_i
//   syrk_kernel<double>  partial [W e]^T [W e] over row chunks, then a fixed-order sum
//                        (FP64 form; the mixed form's is tc_syrk on the tensor cores)
//   final_kernel         M = I + G, FP64 Cholesky, z = L_M^{-1} W^T e, the NLL
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>

#include "dgemm.cuh"
#include "kernels.h"
#include "profile.h"
#include "vif.h"
#include "workspace.h"

namespace vst {

vst_status fail(vst_status s, const char* fmt, ...);
vst_status cuda_fail(cudaError_t e, const char* where);
void launch_init_header(WsHeader* h, cudaStream_t st);
void launch_lag_table(const DevTheta& th, LagD* d, LagF* f, cudaStream_t st);
void apply_launch_shape(RowArgs& g, int batched, int precision, int nu, int pm);

// 16-byte read-only vector load of VEC consecutive values
template <typename T, int VEC>
__device__ __forceinline__ void ldg_vec(T (&v)[VEC], const T* p) {
  if constexpr (sizeof(T) == 4) {
    const float4 f = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
  } else {
    const double2 d = __ldg(reinterpret_cast<const double2*>(p));
    v[0] = d.x; v[1] = d.y;
  }
}

// integer-day range of the data times: info[0] = min day, info[1] = number of
// days, info[2] = 1 if every time is an integer and the span is tabulable.
// Two stages: per-block (min, max, all-integer) partials, then one block.
__global__ void day_partial_kernel(const double* t, int64_t n, double* part) {
  __shared__ double smin[256], smax[256];
  __shared__ int sint[256];
  double lo = DBL_MAX, hi = -DBL_MAX;
  int allint = 1;
  for (int64_t i = blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    const double v = t[i];
    lo = fmin(lo, v);
    hi = fmax(hi, v);
    allint &= (v == floor(v)) && fabs(v) < 1.0e9;
  }
  smin[threadIdx.x] = lo;
  smax[threadIdx.x] = hi;
  sint[threadIdx.x] = allint;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + w]);
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + w]);
      sint[threadIdx.x] &= sint[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = smin[0];
    part[3 * blockIdx.x + 1] = smax[0];
    part[3 * blockIdx.x + 2] = sint[0];
  }
}
__global__ void day_range_kernel(const double* part, int nparts, int64_t n, int64_t* info) {
  __shared__ double smin[256], smax[256];
  __shared__ int sint[256];
  double lo = DBL_MAX, hi = -DBL_MAX;
  int allint = 1;
  for (int b = threadIdx.x; b < nparts; b += 256) {
    lo = fmin(lo, part[3 * b]);
    hi = fmax(hi, part[3 * b + 1]);
    allint &= part[3 * b + 2] != 0.0;
  }
  smin[threadIdx.x] = lo;
  smax[threadIdx.x] = hi;
  sint[threadIdx.x] = allint;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + w]);
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + w]);
      sint[threadIdx.x] &= sint[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const bool ok = n > 0 && sint[0] && (smax[0] - smin[0]) < (double)kVifMaxDays;
    info[0] = ok ? (int64_t)smin[0] : 0;
    info[1] = ok ? (int64_t)(smax[0] - smin[0]) + 1 : 0;
    info[2] = ok ? 1 : 0;
  }
}

// per (data day d, inducing point p): amplitude and Matern scale of the lag
// |dmin + d - t_p|, evaluated in FP64 and rounded once to FP32
__global__ void day_lag_kernel(const double* tk, int k, DevTheta th, const int64_t* info, float2* tab) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (info[2] == 0) return;
  const int64_t nd = info[1];
  if (id >= nd * k) return;
  const int64_t d = id / k;
  const int p = (int)(id % k);
  const LagD f = lag_factors(th, (double)(info[0] + d) - tk[p]);
  tab[id] = make_float2((float)f.P, (float)f.G);
}

// per integer lag u < kLagTab: P and G of Eq. (2) as double-floats
__global__ void lag_df_kernel(DevTheta th, float4* out) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= kLagTab) return;
  const LagD f = lag_factors(th, (double)u);
  const float ph = (float)f.P, gh = (float)f.G;
  out[u] = make_float4(ph, (float)(f.P - (double)ph), gh, (float)(f.G - (double)gh));
}

template <int NU>
__global__ void kk_kernel(const double* xyk, const double* tk, int k, DevTheta th, double* S) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= (int64_t)k * k) return;
  const int r = (int)(id / k), c = (int)(id % k);
  S[id] = cov64<NU>(th, xyk[2 * r] - xyk[2 * c], xyk[2 * r + 1] - xyk[2 * c + 1], tk[r] - tk[c]);
}

// ---------------------------------------------------------------------------
// blocked Cholesky, FP64, lower, in place (A row-major k x k)
constexpr int kPanel = 32;

// diagonal block of the panel, jb x jb (jb <= 32), factored by one warp with
// lane r holding row r in registers (the block staged through shared memory
// for coalesced loads and stores); a non-positive pivot is reported and
// replaced by 1 so that the factorisation finishes
__global__ void chol_diag_kernel(double* A, int k, int j0, int jb, WsHeader* hdr, int err_code) {
  __shared__ double st[32][33];
  __shared__ double col[32];
  const int lane = threadIdx.x;
  for (int r = 0; r < 32; ++r) st[r][lane] = (r < jb && lane < jb) ? A[(int64_t)(j0 + r) * k + j0 + lane] : 0.0;
  __syncwarp();
  double a[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) a[q] = st[lane][q];
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    if (c >= jb) break;
    double d = __shfl_sync(0xffffffffu, a[c], c);
    if (!(d > 0.0)) {
      if (lane == 0) report_error(hdr, err_code, j0 + c);
      d = 1.0;
    }
    d = sqrt(d);
    if (lane == c) a[c] = d;
    if (lane > c) a[c] /= d;
    col[lane] = a[c];
    __syncwarp();
#pragma unroll
    for (int q = c + 1; q < 32; ++q) a[q] = fma(-a[c], col[q], a[q]);
    __syncwarp();
  }
#pragma unroll
  for (int q = 0; q < 32; ++q) st[lane][q] = a[q];
  __syncwarp();
  for (int r = 0; r < jb; ++r)
    if (lane <= r) A[(int64_t)(j0 + r) * k + j0 + lane] = st[r][lane];
}

// panel rows below the diagonal block: L21 = A21 L11^{-T}, one thread per row
// (forward substitution with the factored block in shared memory)
__global__ void chol_trsm_kernel(double* A, int k, int j0, int jb) {
  __shared__ double l[32][33];
  for (int q = threadIdx.x; q < jb * jb; q += blockDim.x) {
    const int r = q / jb, c = q % jb;
    l[r][c] = (c <= r) ? A[(int64_t)(j0 + r) * k + j0 + c] : 0.0;
  }
  __syncthreads();
  const int r = j0 + jb + blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= k) return;
  double x[32];
  double* row = A + (int64_t)r * k + j0;
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    if (c < jb) {
      double v = row[c];
#pragma unroll
      for (int p = 0; p < c; ++p) v -= x[p] * l[c][p];
      x[c] = v / l[c][c];
      row[c] = x[c];
    }
  }
}

// trailing update A[r][c] -= sum_{p in panel} A[r][p] A[c][p], j0+jb <= c <= r < k
__global__ void chol_trail_kernel(double* A, int k, int j0, int jb) {
  __shared__ double Ar[32][kPanel + 1], Ac[32][kPanel + 1];
  const int t0 = j0 + jb;
  const int br = blockIdx.y, bc = blockIdx.x;
  if (bc > br) return;
  const int r0 = t0 + br * 32, c0 = t0 + bc * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int q = threadIdx.x; q < 32 * jb; q += blockDim.x) {
    const int rr = q / jb, pp = q % jb;
    Ar[rr][pp] = (r0 + rr < k) ? A[(int64_t)(r0 + rr) * k + j0 + pp] : 0.0;
    Ac[rr][pp] = (c0 + rr < k) ? A[(int64_t)(c0 + rr) * k + j0 + pp] : 0.0;
  }
  __syncthreads();
  for (int rr = ty; rr < 32; rr += 8) {
    const int r = r0 + rr, c = c0 + tx;
    if (r >= k || c >= k || c > r) continue;
    double s = 0.0;
    for (int p = 0; p < jb; ++p) s += Ar[rr][p] * Ac[tx][p];
    A[(int64_t)r * k + c] -= s;
  }
}

vst_status chol64(double* A, int k, WsHeader* hdr, int err_code, cudaStream_t st) {
  for (int j0 = 0; j0 < k; j0 += kPanel) {
    const int jb = std::min(kPanel, k - j0);
    chol_diag_kernel<<<1, 32, 0, st>>>(A, k, j0, jb, hdr, err_code);
    const int rest = k - (j0 + jb);
    if (rest > 0) {
      chol_trsm_kernel<<<(rest + 127) / 128, 128, 0, st>>>(A, k, j0, jb);
      const int nb = (rest + 31) / 32;
      chol_trail_kernel<<<dim3(nb, nb), 256, 0, st>>>(A, k, j0, jb);
    }
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VST_OK : cuda_fail(e, "cholesky");
}

// X = L^{-1} (lower); one warp per column j: forward substitution of L x = e_j
__global__ void trinv_kernel(const double* L, int k, double* X) {
  extern __shared__ double xs_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  double* x = xs_raw + (int64_t)wib * k;
  for (int j = blockIdx.x * wpb + wib; j < k; j += gridDim.x * wpb) {
    for (int r = lane; r < k; r += 32) x[r] = 0.0;
    __syncwarp();
    if (lane == 0) x[j] = 1.0 / L[(int64_t)j * k + j];
    __syncwarp();
    for (int r = j + 1; r < k; ++r) {
      // row segment L[r][j..r) read 8 loads per lane at a time (independent
      // loads in flight instead of one dependent load per step)
      double s = 0.0;
      const double* Lr = L + (int64_t)r * k;
      for (int p0 = j; p0 < r; p0 += 256) {
        double lv[8], xv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int p = p0 + u * 32 + lane;
          lv[u] = p < r ? Lr[p] : 0.0;
          xv[u] = p < r ? x[p] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) s = fma(lv[u], xv[u], s);
      }
      s = warp_sum(s);
      if (lane == 0) x[r] = -s / L[(int64_t)r * k + r];
      __syncwarp();
    }
    for (int r = lane; r < k; r += 32) X[(int64_t)r * k + j] = x[r];
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// FP64 form: Sigma_nk[i][p] = C(x_i, z_p), one thread per entry
template <int NU>
__global__ void snk64_kernel(const double* xy, const double* t, int64_t n, const double* xyk, const double* tk,
                             int k, DevTheta th, double* S) {
  const int64_t total = n * k;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / k;
    const int p = (int)(q - i * k);
    S[q] = cov64<NU>(th, xy[2 * i] - xyk[2 * p], xy[2 * i + 1] - xyk[2 * p + 1], t[i] - tk[p]);
  }
}

template <typename T>
__global__ void rdiag_kernel(const T* U, int64_t n, int k, double s1, double* r) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nw) {
    double s = 0.0;
    for (int c = lane; c < k; c += 32) {
      const double u = (double)U[i * k + c];
      s += u * u;
    }
    s = warp_sum(s);
    if (lane == 0) r[i] = s1 - s;
  }
}

// ---------------------------------------------------------------------------
// Local blocks of the row kernel: positions 0..cnt-1 are the neighbours of
// row i, position PM-1 is row i itself, the rest unused (index -1).
template <int PM>
__device__ __forceinline__ void block_indices(const int32_t* nn, const int32_t* nn_cnt, int64_t i, int m,
                                              int (&idx)[PM]) {
  const int cnt = min(max(nn_cnt[i], 0), min(m, PM - 1));
#pragma unroll
  for (int p = 0; p < PM; ++p) {
    int v = -1;
    if (p < cnt) v = nn[i * m + p];
    if (p == PM - 1) v = (int)i;
    idx[p] = (v >= 0 && v <= i) ? v : -1;
  }
}

// FP64 form: gram[i][e] = U_{pos r} . U_{pos c} over the pairs e of the local
// block in the packed order of the row kernel.  One warp per row.
template <int PM>
__global__ void __launch_bounds__(128) gram64_kernel(const int32_t* nn, const int32_t* nn_cnt, int64_t n, int m,
                                                     int k, const double* U, double* gram) {
  constexpr int NPAIR = PM * (PM + 1) / 2;
  constexpr int NPL = (NPAIR + 31) / 32;  // pairs per lane
  __shared__ double Us[4][PM][33];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t warp = (int64_t)blockIdx.x * 4 + wib;
  const int64_t total = (int64_t)gridDim.x * 4;
  int pr[NPL], pc[NPL];
#pragma unroll
  for (int q = 0; q < NPL; ++q) {
    const int e = lane + 32 * q;
    int r = 0, c = 0;
    if (e < NPAIR) pair_of<PM>(e, r, c);
    pr[q] = r;
    pc[q] = c;
  }
  for (int64_t i = warp; i < n; i += total) {
    int idx[PM];
    block_indices<PM>(nn, nn_cnt, i, m, idx);
    double acc[NPL];
#pragma unroll
    for (int q = 0; q < NPL; ++q) acc[q] = 0.0;
    for (int c0 = 0; c0 < k; c0 += 32) {
      const int c = c0 + lane;
#pragma unroll
      for (int p = 0; p < PM; ++p) Us[wib][p][lane] = (idx[p] >= 0 && c < k) ? U[(int64_t)idx[p] * k + c] : 0.0;
      __syncwarp();
#pragma unroll
      for (int q = 0; q < NPL; ++q) {
        const double* a = Us[wib][pr[q]];
        const double* b = Us[wib][pc[q]];
        double s = 0.0;
#pragma unroll 8
        for (int u = 0; u < 32; ++u) s = fma(a[u], b[u], s);
        acc[q] += s;
      }
      __syncwarp();
    }
#pragma unroll
    for (int q = 0; q < NPL; ++q) {
      const int e = lane + 32 * q;
      if (e < NPAIR) gram[i * NPAIR + e] = acc[q];
    }
  }
}

// Mixed form: gram[i][e] = U_p . U_q for the pairs e of the local block,
// accumulated without cancellation and rounded once to FP32.  With the row's
// own vector as the reference, V_p = U_p - U_i and w_p = U_i . V_p:
//   U_p . U_q = |U_i|^2 + w_p + w_q + V_p . V_q,   |U_i|^2 = sigma1^2 - r_i,
// (U_p . U_i = |U_i|^2 + w_p) where the sums over k are of terms that are
// small next to |U_i|^2 for the neighbours.  (Handing the row kernel
// U_p . U_q - sigma1^2 instead, a value with a finer FP32 rounding, measured a
// ~10x larger mixed-vs-FP64 NLL difference on the VIF benchmark rows, with D_i
// biased upward; the row kernel therefore forms C - G as before.)  The Gram of the vectors {V_0, .., V_{PM-2}, U_i} is a small SYRK:
// one warp per RW = 2 rows, the lower triangle in 4 x 4 tiles (NT per row),
// lane jobs (row slot, tile) in rounds where the 32 lanes of a round share the
// row slot, so that the 16-byte shared loads of a tile's four positions are
// broadcasts.  Columns are staged 32 at a time: lane p loads U_p, the shuffled
// U_i gives V_p, and the chunk is stored position-contiguous.  Each chunk's
// 32 products are summed in FP32 (exact products in the FMA, a short chain)
// and added to double-float running sums; a single FP32 sum over all k
// columns (k ~ 1e3) loses enough to bias the NLL by ~1e-6 per point, since
// the V_p are not small when k is large.
template <int PM>
struct GramTiles {
  static constexpr int B = PM / 4;              // 4-position blocks
  static constexpr int NT = B * (B + 1) / 2;    // lower-triangle tiles per row
  static constexpr int RW = 2;                  // rows per warp
  static constexpr int FULL = NT / 32;          // rounds with one row slot per round
  static constexpr int LEFT = NT - FULL * 32;   // tiles per row left over
  static constexpr int ROUNDS = FULL * RW + (LEFT * RW + 31) / 32;
  static constexpr int SLOT = 32 * PM + 4;      // floats per row slot (+1 chunk against bank conflicts)
};

template <int PM>
__global__ void __launch_bounds__(128) gram_delta_kernel(const int32_t* nn, const int32_t* nn_cnt, int64_t n,
                                                         int m, int k, const float* U, const double* r, double s1,
                                                         float* gram) {
  using GT = GramTiles<PM>;
  constexpr int NPAIR = PM * (PM + 1) / 2;
  constexpr int L = PM - 1;
  extern __shared__ __align__(16) float gsm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* Vs = gsm + (size_t)wib * GT::RW * GT::SLOT;
  const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  // this lane's jobs: row slot, and the tile's first rows (4 R) and columns (4 C)
  int jrs[GT::ROUNDS], jr[GT::ROUNDS], jc[GT::ROUNDS];
  bool jon[GT::ROUNDS];
#pragma unroll
  for (int q = 0; q < GT::ROUNDS; ++q) {
    int rs = 0, t = 0;
    bool on = true;
    constexpr int FD = GT::FULL > 0 ? GT::FULL : 1;  // (no full rounds when PM = 8)
    if (q < GT::FULL * GT::RW) {
      rs = q / FD;
      t = (q % FD) * 32 + lane;
    } else {
      const int j = (q - GT::FULL * GT::RW) * 32 + lane;
      on = j < GT::LEFT * GT::RW;
      rs = on ? j / GT::LEFT : 0;
      t = on ? GT::FULL * 32 + j % GT::LEFT : 0;
    }
    int R = 0;
    while ((R + 1) * (R + 2) / 2 <= t) ++R;
    jrs[q] = rs;
    jr[q] = 4 * R;
    jc[q] = 4 * (t - R * (R + 1) / 2);
    jon[q] = on;
  }
  const bool vec = (k & 3) == 0;
  for (int64_t i0 = warp * GT::RW; i0 < n; i0 += nwarps * GT::RW) {
    int idx[GT::RW];  // this lane's position in each row slot (-1: unused)
#pragma unroll
    for (int rs = 0; rs < GT::RW; ++rs) {
      const int64_t i = i0 + rs;
      int v = -1;
      if (i < n && lane < PM) {
        const int cnt = min(max(nn_cnt[i], 0), min(m, L));
        if (lane < cnt) v = nn[i * m + lane];
        if (lane == L) v = (int)i;
        if (v < 0 || v > i) v = -1;
      }
      idx[rs] = v;
    }
    float acc[GT::ROUNDS][16], accl[GT::ROUNDS][16];  // double-float running sums
#pragma unroll
    for (int q = 0; q < GT::ROUNDS; ++q)
#pragma unroll
      for (int z = 0; z < 16; ++z) acc[q][z] = accl[q][z] = 0.f;
    for (int c0 = 0; c0 < k; c0 += 32) {
      __syncwarp();
#pragma unroll
      for (int rs = 0; rs < GT::RW; ++rs) {
        float u[32];
        const int64_t row = idx[rs];
        if (row >= 0 && vec && c0 + 32 <= k) {
          const float4* src = reinterpret_cast<const float4*>(U + row * k + c0);
#pragma unroll
          for (int z = 0; z < 8; ++z) {
            const float4 f = __ldg(src + z);
            u[4 * z] = f.x; u[4 * z + 1] = f.y; u[4 * z + 2] = f.z; u[4 * z + 3] = f.w;
          }
        } else {
#pragma unroll
          for (int z = 0; z < 32; ++z) u[z] = (row >= 0 && c0 + z < k) ? __ldg(U + row * k + c0 + z) : 0.f;
        }
        float* dst = Vs + rs * GT::SLOT;
#pragma unroll
        for (int z = 0; z < 32; ++z) {
          const float ui = __shfl_sync(0xffffffffu, u[z], L);
          // V_p = U_p - U_i for the neighbours, U_i itself at position L
          const float v = lane == L ? ui : (idx[rs] >= 0 ? u[z] - ui : 0.f);
          if (lane < PM) dst[z * PM + lane] = v;
        }
      }
      __syncwarp();
      // each chunk's 32 products summed apart, then added to the running sums
      // (shorter FP32 accumulation chains than one sum over all k columns)
#pragma unroll
      for (int q = 0; q < GT::ROUNDS; ++q) {
        if (!jon[q]) continue;
        float part[16];
#pragma unroll
        for (int z = 0; z < 16; ++z) part[z] = 0.f;
        const float* col = Vs + jrs[q] * GT::SLOT;
#pragma unroll 4
        for (int z = 0; z < 32; ++z) {
          const float4 a = *reinterpret_cast<const float4*>(col + z * PM + jr[q]);
          const float4 b = *reinterpret_cast<const float4*>(col + z * PM + jc[q]);
          const float av[4] = {a.x, a.y, a.z, a.w};
          const float2 b01 = make_float2(b.x, b.y), b23 = make_float2(b.z, b.w);
#pragma unroll
          for (int x = 0; x < 4; ++x) {  // packed FP32 pairs: the same fmaf per product
            const float2 ax = make_float2(av[x], av[x]);
            const float2 p01 = __ffma2_rn(ax, b01, make_float2(part[4 * x], part[4 * x + 1]));
            const float2 p23 = __ffma2_rn(ax, b23, make_float2(part[4 * x + 2], part[4 * x + 3]));
            part[4 * x] = p01.x;
            part[4 * x + 1] = p01.y;
            part[4 * x + 2] = p23.x;
            part[4 * x + 3] = p23.y;
          }
        }
#pragma unroll
        for (int z = 0; z < 16; ++z) {
          const df t = df_two_sum(acc[q][z], part[z]);
          acc[q][z] = t.hi;
          accl[q][z] += t.lo;
        }
      }
    }
    // S (lower triangle, PM x PM per row slot) to shared memory, then E
    __syncwarp();
#pragma unroll
    for (int q = 0; q < GT::ROUNDS; ++q) {
      if (!jon[q]) continue;
      float* S = Vs + jrs[q] * GT::SLOT;
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) S[(jr[q] + x) * PM + jc[q] + y] = acc[q][4 * x + y] + accl[q][4 * x + y];
    }
    __syncwarp();
#pragma unroll
    for (int rs = 0; rs < GT::RW; ++rs) {
      const int64_t i = i0 + rs;
      if (i >= n) break;
      const float* S = Vs + rs * GT::SLOT;
      const df s1m = df_split(s1 - r[i]);  // |U_i|^2 = sigma1^2 - r_i
      for (int e = lane; e < NPAIR; e += 32) {
        int a, b;
        pair_of<PM>(e, a, b);  // a >= b
        // w_a + w_b + S_ab - r_i in double-float, rounded once
        df v = {0.f, 0.f};
        if (a != L) {
          v = df_two_sum(S[L * PM + a], S[L * PM + b]);
          const df t = df_two_sum(v.hi, S[a * PM + b]);
          v = df{t.hi, v.lo + t.lo};
        } else if (b != L) {
          v = df{S[L * PM + b], 0.f};
        }
        // G = sigma1^2 - r_i + (w_a + w_b + S_ab), rounded once
        const df t = df_two_sum(v.hi, s1m.hi);
        gram[i * NPAIR + e] = t.hi + (t.lo + (v.lo + s1m.lo));
      }
    }
  }
}

template <int PM>
constexpr size_t gram_delta_smem(int warps) {
  return sizeof(float) * (size_t)GramTiles<PM>::RW * GramTiles<PM>::SLOT * warps;
}

// rows of [W e]: W_i = (U_i - sum_q A_iq U_{nn(i,q)}) / sqrt(D_i), e_i likewise
// with y; writes WE[i][0..k) = W_i and WE[i][k] = e_i; per-warp partial sums
// of log D_i into part[warp].  One warp per row: the neighbours' indices and
// coefficients staged once in shared memory, U rows read 16 bytes per lane.
template <typename T>
__global__ void __launch_bounds__(256) wvec_kernel(const int32_t* nn, const int32_t* nn_cnt, int64_t n, int m,
                                                   int k, const T* U, const double* y, const double* A,
                                                   const double* D, T* WE, double* part) {
  constexpr int VEC = 16 / (int)sizeof(T);
  __shared__ int sj[8][32];
  __shared__ T sa[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const bool vec = (k % VEC) == 0;
  double slog = 0.0;
  for (int64_t i = warp; i < n; i += nw) {
    const int cnt0 = min(max(nn_cnt[i], 0), min(m, 32));
    const double Di = D[i];
    const double s = 1.0 / sqrt(Di);
    int myj = -1;
    double mya = 0.0;
    if (lane < cnt0) {
      myj = nn[i * m + lane];
      mya = A[i * m + lane];
      if (myj < 0 || myj >= i) { myj = -1; mya = 0.0; }
    }
    double ey = (myj >= 0) ? mya * y[myj] : 0.0;
    ey = warp_sum(ey);
    // compact the used neighbours (a skipped one has coefficient 0)
    __syncwarp();
    sj[wib][lane] = myj >= 0 ? myj : (int)i;
    sa[wib][lane] = (T)mya;
    __syncwarp();
    const int cnt = cnt0;
    const T sT = (T)s;
    const T* Ui = U + i * k;
    T* Wi = WE + i * (k + 1);
    if (vec) {
      for (int c = lane * VEC; c < k; c += 32 * VEC) {
        T v[VEC];
        ldg_vec<T, VEC>(v, Ui + c);
#pragma unroll 4
        for (int q = 0; q < cnt; ++q) {
          T u[VEC];
          ldg_vec<T, VEC>(u, U + (int64_t)sj[wib][q] * k + c);
          const T aq = sa[wib][q];
#pragma unroll
          for (int z = 0; z < VEC; ++z) v[z] = fma(-aq, u[z], v[z]);
        }
#pragma unroll
        for (int z = 0; z < VEC; ++z) Wi[c + z] = v[z] * sT;
      }
    } else {
      for (int c = lane; c < k; c += 32) {
        T v = Ui[c];
        for (int q = 0; q < cnt; ++q) v = fma(-sa[wib][q], U[(int64_t)sj[wib][q] * k + c], v);
        Wi[c] = v * sT;
      }
    }
    if (lane == 0) {
      Wi[k] = (T)((y[i] - ey) * s);
      slog += log(Di);
    }
  }
  slog = warp_sum(slog);
  if (lane == 0) part[warp] = slog;
}

// partial G = WE^T WE over a row chunk: 64 x 64 output tile of the (k+1)^2
// lower triangle per block (4 x 4 per thread), 16 rows per K step,
// blockIdx.z = row chunk.  Products accumulate in T over 256 rows and then
// in FP64; the chunks are summed in a fixed order by syrk_sum_kernel.
template <typename T>
__global__ void __launch_bounds__(256) syrk_kernel(const T* WE, int64_t n, int kk, int64_t chunk, double* part) {
  constexpr int BT = 64, BK = 16;
  __shared__ T As[BK][BT + 4], Bs[BK][BT + 4];
  const int br = blockIdx.y, bc = blockIdx.x;
  if (bc > br) return;
  const int r0 = br * BT, c0 = bc * BT;
  const int64_t n0 = (int64_t)blockIdx.z * chunk;
  const int64_t n1 = n < n0 + chunk ? n : n0 + chunk;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
  T part_acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      acc[a][b] = 0.0;
      part_acc[a][b] = T(0);
    }
  int steps = 0;
  for (int64_t b0 = n0; b0 < n1; b0 += BK) {
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + q * 256;
      const int kk2 = e >> 6, cc = e & (BT - 1);
      const int64_t srow = b0 + kk2;
      As[kk2][cc] = (srow < n1 && r0 + cc < kk) ? WE[srow * kk + r0 + cc] : T(0);
      Bs[kk2][cc] = (srow < n1 && c0 + cc < kk) ? WE[srow * kk + c0 + cc] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < BK; ++q) {
      T a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[q][ty * 4 + u];
        b[u] = Bs[q][tx * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) part_acc[u][v] = fma(a[u], b[v], part_acc[u][v]);
    }
    if (++steps == 16) {  // every 256 rows: fold into FP64
      steps = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          acc[u][v] += (double)part_acc[u][v];
          part_acc[u][v] = T(0);
        }
    }
  }
  const int64_t kk2 = (int64_t)kk * kk;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int r = r0 + ty * 4 + u, c = c0 + tx * 4 + v;
      if (r < kk && c < kk && c <= r)
        part[(int64_t)blockIdx.z * kk2 + (int64_t)r * kk + c] = acc[u][v] + (double)part_acc[u][v];
    }
}

__global__ void syrk_sum_kernel(const double* part, int nchunk, int kk, double* G) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t kk2 = (int64_t)kk * kk;
  if (id >= kk2) return;
  const int r = (int)(id / kk), c = (int)(id % kk);
  if (c > r) return;
  double s = 0.0;
  for (int q = 0; q < nchunk; ++q) s += part[q * kk2 + id];
  G[id] = s;
  G[(int64_t)c * kk + r] = s;
}

// M = I + G[0..k) (in place into Mout, k x k), v = G[0..k][k], ete = G[k][k]
__global__ void make_m_kernel(const double* G, int k, double* M, double* v, double* ete) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int kk = k + 1;
  if (id < (int64_t)k * k) {
    const int r = (int)(id / k), c = (int)(id % k);
    M[id] = G[(int64_t)r * kk + c] + (r == c ? 1.0 : 0.0);
  }
  if (id < k) v[id] = G[(int64_t)id * kk + k];
  if (id == 0) *ete = G[(int64_t)k * kk + k];
}

// z = L_M^{-1} v (one block of 1024 threads), then the NLL.  The forward
// substitution runs in blocks of 32 rows: the 32 warps each take one row's
// product with the solved part (lanes over the row, 8 loads in flight per
// lane), then warp 0 solves the 32 x 32 diagonal block by shuffles with the
// reciprocal diagonal computed up front.
__global__ void __launch_bounds__(1024) final_kernel(const double* Lm, int k, const double* v, const double* ete,
                                                     const double* logd_part, int64_t nparts, int64_t n, double* z,
                                                     double* nll) {
  __shared__ double sh[1024];
  __shared__ double rhs[32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // sum log D_i (fixed order) and log det M; reciprocal diagonal into z
  double s = 0.0;
  for (int64_t q = tid; q < nparts; q += 1024) s += logd_part[q];
  double ld = 0.0;
  for (int r = tid; r < k; r += 1024) {
    const double d = Lm[(int64_t)r * k + r];
    ld += 2.0 * log(d);
    z[r] = 1.0 / d;
  }
  sh[tid] = s + ld;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (tid < w) sh[tid] += sh[tid + w];
    __syncthreads();
  }
  const double logdet = sh[0];
  __syncthreads();
  for (int b0 = 0; b0 < k; b0 += 32) {
    const int R = min(32, k - b0);
    if (wid < R) {
      const int r = b0 + wid;
      const double* Lr = Lm + (int64_t)r * k;
      double d = 0.0;
      for (int p0 = 0; p0 < b0; p0 += 256) {
        double lv[8], zv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int p = p0 + u * 32 + lane;
          lv[u] = p < b0 ? Lr[p] : 0.0;
          zv[u] = p < b0 ? z[p] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) d = fma(lv[u], zv[u], d);
      }
      d = warp_sum(d);
      if (lane == 0) rhs[wid] = v[r] - d;
    }
    __syncthreads();
    if (wid == 0) {
      // lane i: row b0 + i of the diagonal block
      double acc = lane < R ? rhs[lane] : 0.0;
      const double rd = lane < R ? z[b0 + lane] : 0.0;  // 1 / L_ii
      double zi = 0.0;
      for (int c = 0; c < R; ++c) {
        const double zc = __shfl_sync(0xffffffffu, acc * rd, c);
        if (lane == c) zi = zc;
        if (lane > c && lane < R) acc = fma(-Lm[(int64_t)(b0 + lane) * k + b0 + c], zc, acc);
      }
      if (lane < R) z[b0 + lane] = zi;
    }
    __syncthreads();
  }
  double zz = 0.0;
  for (int r = tid; r < k; r += 1024) zz += z[r] * z[r];
  sh[tid] = zz;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (tid < w) sh[tid] += sh[tid + w];
    __syncthreads();
  }
  if (tid == 0) *nll = 0.5 * (double)n * log(2.0 * M_PI) + 0.5 * logdet + 0.5 * (*ete - sh[0]);
}

// ---------------------------------------------------------------------------
// host side

template <typename T>
static vst_status lowrank_T(const vst_points* pts, const vst_theta* theta, const vst_inducing* ind, int nu,
                            int split_terms, char* vbase, const VifLayout& V, WsHeader* hdr, cudaStream_t st) {
  const int64_t n = pts->n;
  const int k = (int)ind->k;
  const DevTheta th = dev_theta_vif(theta);
  double* S = reinterpret_cast<double*>(vbase + V.S);
  double* X = reinterpret_cast<double*>(vbase + V.X);
  T* U = reinterpret_cast<T*>(vbase + V.U);
  double* r = reinterpret_cast<double*>(vbase + V.r);
  const int64_t kk = (int64_t)k * k;
  const int gb = (int)((kk + 255) / 256);
  if (nu == 0) kk_kernel<0><<<gb, 256, 0, st>>>(ind->xy, ind->t, k, th, S);
  else if (nu == 1) kk_kernel<1><<<gb, 256, 0, st>>>(ind->xy, ind->t, k, th, S);
  else kk_kernel<2><<<gb, 256, 0, st>>>(ind->xy, ind->t, k, th, S);
  vst_status s = chol64(S, k, hdr, VST_ENOTSPD, st);
  if (s != VST_OK) return s;
  const int wpb = 4;
  const size_t smem = sizeof(double) * k * wpb;
  if (smem > 48 * 1024) cudaFuncSetAttribute(trinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  trinv_kernel<<<(k + wpb - 1) / wpb, 32 * wpb, smem, st>>>(S, k, X);
  if (n > 0) {
    int64_t* dinfo = reinterpret_cast<int64_t*>(vbase + V.dinfo);
    float2* dtab = reinterpret_cast<float2*>(vbase + V.dtab);
    double* dpart = reinterpret_cast<double*>(vbase + V.dpart);
    const int dblocks = (int)std::min<int64_t>(kVifDayBlocks, (n + 255) / 256);
    day_partial_kernel<<<dblocks, 256, 0, st>>>(pts->t, n, dpart);
    day_range_kernel<<<1, 256, 0, st>>>(dpart, dblocks, n, dinfo);
    day_lag_kernel<<<(int)((kVifMaxDays * (int64_t)k + 255) / 256), 256, 0, st>>>(ind->t, k, th, dinfo, dtab);
    if constexpr (std::is_same<T, double>::value) {
      // Sigma_nk once (into the [W e] buffer, unused until the Woodbury
      // step), then U = Sigma_nk X^T with X = L^{-1} lower triangular
      double* Snk = reinterpret_cast<double*>(vbase + V.WE);
      const unsigned gs = (unsigned)std::min<int64_t>((n * k + 255) / 256, 65535 * 16);
      if (nu == 0) snk64_kernel<0><<<gs, 256, 0, st>>>(pts->xy, pts->t, n, ind->xy, ind->t, k, th, Snk);
      else if (nu == 1) snk64_kernel<1><<<gs, 256, 0, st>>>(pts->xy, pts->t, n, ind->xy, ind->t, k, th, Snk);
      else snk64_kernel<2><<<gs, 256, 0, st>>>(pts->xy, pts->t, n, ind->xy, ind->t, k, th, Snk);
      ProfileScope ps(kProfVifGemm, st);
      gemm_nt(Snk, k, X, k, U, k, n, k, k, true, st);
    } else {
      (void)dtab;
      s = lowrank_tc(pts, theta, ind, nu, split_terms, vbase, V, hdr, st);
      if (s != VST_OK) return s;
    }
    // (the tensor-core path forms r from its GEMM epilogue)
    if constexpr (std::is_same<T, double>::value)
      rdiag_kernel<T><<<(int)std::min<int64_t>((n + 7) / 8, 65535), 256, 0, st>>>(U, n, k, theta->sigma1sq, r);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VST_OK : cuda_fail(e, "VIF low-rank kernels");
}

// U and r: FP64 SIMT GEMM (VST_FP64), or the split-BF16 tensor-core GEMM with
// 6 products (VST_MIXED) or 3 products (VST_MIXED_BF16X3)
vst_status vif_lowrank(const vst_points* pts, const vst_theta* theta, const vst_inducing* ind, int nu,
                       int precision, char* vbase, const VifLayout& V, WsHeader* hdr, cudaStream_t st) {
  if (precision == VST_FP64) return lowrank_T<double>(pts, theta, ind, nu, 0, vbase, V, hdr, st);
  return lowrank_T<float>(pts, theta, ind, nu, precision == VST_MIXED_BF16X3 ? 3 : 6, vbase, V, hdr, st);
}

// gram = U_p . U_q for the pairs of each local block (FP64; mixed: accumulated without
// cancellation and rounded once to FP32, see gram_delta_kernel)
static void launch_gram(int pm, const int32_t* nn, const int32_t* nn_cnt, int64_t n, int m, int k, const double* U,
                        const double* r, double s1, double* gram, cudaStream_t st) {
  (void)r;
  (void)s1;
  const int blocks = (int)std::min<int64_t>((n + 3) / 4, 152 * 16);
  switch (padded_pm(pm)) {
    case 8: gram64_kernel<8><<<blocks, 128, 0, st>>>(nn, nn_cnt, n, m, k, U, gram); break;
    case 16: gram64_kernel<16><<<blocks, 128, 0, st>>>(nn, nn_cnt, n, m, k, U, gram); break;
    case 24: gram64_kernel<24><<<blocks, 128, 0, st>>>(nn, nn_cnt, n, m, k, U, gram); break;
    default: gram64_kernel<32><<<blocks, 128, 0, st>>>(nn, nn_cnt, n, m, k, U, gram);
  }
}
static void launch_gram(int pm, const int32_t* nn, const int32_t* nn_cnt, int64_t n, int m, int k, const float* U,
                        const double* r, double s1, float* gram, cudaStream_t st) {
  auto go = [&](auto kern, size_t smem) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 128, smem);
    const int64_t need = (n + 4 * 2 - 1) / (4 * 2);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)std::max(per, 1) * sms));
    kern<<<blocks, 128, smem, st>>>(nn, nn_cnt, n, m, k, U, r, s1, gram);
  };
  // (blocks of 32 positions go to the tensor-core kernel, gram_tc_rows)
  switch (padded_pm(pm)) {
    case 8: go(gram_delta_kernel<8>, gram_delta_smem<8>(4)); break;
    case 16: go(gram_delta_kernel<16>, gram_delta_smem<16>(4)); break;
    default: go(gram_delta_kernel<24>, gram_delta_smem<24>(4));
  }
}

// factor of the residual (A, D) with the fused row kernel fed the Gram
template <typename T>
static vst_status vif_factor_T(const vst_points* pts, const vst_theta* theta, int m, const vst_inducing* ind, int nu,
                               const int32_t* nn, const int32_t* nn_cnt, int precision, double* Aout, double* Dout,
                               char* base, const WsLayout& L, char* vbase, const VifLayout& V, cudaStream_t st) {
  WsHeader* hdr = reinterpret_cast<WsHeader*>(base + L.hdr);
  vst_status s = vif_lowrank(pts, theta, ind, nu, precision, vbase, V, hdr, st);
  if (s != VST_OK) return s;
  const int64_t n = pts->n;
  const int k = (int)ind->k;
  T* U = reinterpret_cast<T*>(vbase + V.U);
  T* gram = reinterpret_cast<T*>(vbase + V.gram);
  if (n > 0) {
    ProfileScope ps(kProfVifGram, st);
    const double* rr = reinterpret_cast<const double*>(vbase + V.r);
    if constexpr (std::is_same<T, float>::value) {
      // blocks of 32 positions: the tensor-core kernel (vif_gram_tc.cu)
      if (padded_pm(m + 1) == 32) {
        // (the operand-part buffers of the low rank are free once U is formed)
        s = gram_tc_rows(nn, nn_cnt, n, m, k, U, reinterpret_cast<__nv_bfloat16*>(vbase + V.Ap),
                         reinterpret_cast<float*>(vbase + V.uscale), gram, hdr, st);
        if (s != VST_OK) return s;
      } else {
        launch_gram(m + 1, nn, nn_cnt, n, m, k, U, rr, theta->sigma1sq, gram, st);
      }
    } else {
      launch_gram(m + 1, nn, nn_cnt, n, m, k, U, rr, theta->sigma1sq, gram, st);
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "gram kernel");
  LagD* lagd = reinterpret_cast<LagD*>(base + L.lagd);
  LagF* lagf = reinterpret_cast<LagF*>(base + L.lagf);
  uint8_t* flag = reinterpret_cast<uint8_t*>(base + L.flag);
  const DevTheta th = dev_theta_vif(theta);
  launch_lag_table(th, lagd, lagf, st);
  float4* lagdf = reinterpret_cast<float4*>(vbase + V.lagdf);
  lag_df_kernel<<<(kLagTab + 127) / 128, 128, 0, st>>>(th, lagdf);
  const bool mixed = precision != VST_FP64;
  PrepPt* prep = reinterpret_cast<PrepPt*>(base + L.prep);
  if (mixed) launch_prep_points(n, pts->xy, pts->t, nullptr, prep, flag, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "prep kernel");
  RowArgs g{};
  g.xy = pts->xy;
  g.t = pts->t;
  g.nn = nn;
  g.nn_cnt = nn_cnt;
  g.n = n;
  g.m = m;
  g.th = th;
  g.lagd = lagd;
  g.lagf = lagf;
  g.A = Aout;
  g.D = Dout;
  g.flag = flag;
  g.hdr = hdr;
  g.tau = kDefaultTau;
  g.partial = reinterpret_cast<double*>(base + L.partial);
  g.prep = prep;
  g.lagdf = lagdf;
  if constexpr (std::is_same<T, double>::value) g.gram_d = gram;
  else g.gram_f = gram;
  apply_launch_shape(g, 0, precision, nu, m + 1);
  int64_t w = 0;
  if (n > 0) {
    {
      ProfileScope ps(kProfRows, st);
      e = launch_rows(mixed, nu, m + 1, kModeFactor, g, st, &w);
    }
    if (e != cudaSuccess) return cuda_fail(e, "VIF row kernel");
    if (mixed) {
      // FP64 redo of flagged rows: needs the FP64 Gram of those rows
      g.fallback_only = 1;
      e = launch_rows(false, nu, m + 1, kModeFactor, g, st, &w);
      if (e != cudaSuccess) return cuda_fail(e, "VIF fallback kernel");
    }
  }
  return VST_OK;
}

vst_status vif_factor(const vst_points* pts, const vst_theta* theta, int m, const vst_inducing* ind, int nu,
                      const int32_t* nn, const int32_t* nn_cnt, int precision, double* A, double* D, void* ws,
                      cudaStream_t st) {
  char* base = static_cast<char*>(ws);
  const WsLayout L = ws_layout(pts->n, m, ind->k);
  char* vbase = base + L.vif;
  const VifLayout V = vif_layout(pts->n, m, ind->k);
  return precision == VST_FP64 ? vif_factor_T<double>(pts, theta, m, ind, nu, nn, nn_cnt, precision, A, D, base, L,
                                                      vbase, V, st)
                               : vif_factor_T<float>(pts, theta, m, ind, nu, nn, nn_cnt, precision, A, D, base, L,
                                                     vbase, V, st);
}

template <typename T>
static vst_status vif_nll_T(const vst_points* pts, const vst_theta* theta, int m, const vst_inducing* ind, int nu,
                            const int32_t* nn, const int32_t* nn_cnt, const double* y, int precision, double* nll,
                            void* ws, cudaStream_t st) {
  char* base = static_cast<char*>(ws);
  const int64_t n = pts->n;
  const int k = (int)ind->k;
  const WsLayout L = ws_layout(n, m, k);
  char* vbase = base + L.vif;
  const VifLayout V = vif_layout(n, m, k);
  double* A = reinterpret_cast<double*>(base + L.sA);
  double* D = reinterpret_cast<double*>(base + L.sD);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(base + L.hdr);
  vst_status s = vif_factor_T<T>(pts, theta, m, ind, nu, nn, nn_cnt, precision, A, D, base, L, vbase, V, st);
  if (s != VST_OK) return s;
  T* U = reinterpret_cast<T*>(vbase + V.U);
  T* WE = reinterpret_cast<T*>(vbase + V.WE);
  double* logd = reinterpret_cast<double*>(vbase + V.logd);
  double* part = reinterpret_cast<double*>(vbase + V.syrk);
  double* G = reinterpret_cast<double*>(vbase + V.G);
  double* M = reinterpret_cast<double*>(vbase + V.M);
  double* v = reinterpret_cast<double*>(vbase + V.v);
  double* z = reinterpret_cast<double*>(vbase + V.z);
  const int wblocks = (int)std::min<int64_t>((n + 7) / 8, kVifMaxWarps / 8);
  int64_t nparts = 0;
  if (n > 0) {
    wvec_kernel<T><<<wblocks, 256, 0, st>>>(nn, nn_cnt, n, m, k, U, y, A, D, WE, logd);
    nparts = (int64_t)wblocks * 8;
  }
  const int kk = k + 1;
  const int64_t kk2 = (int64_t)kk * kk;
  if constexpr (std::is_same<T, float>::value) {
    // [W e]^T [W e] on the tensor cores with the fixed-point split (six
    // products in both mixed forms): the Woodbury quadratic form
    // e^T e - v^T M^{-1} v cancels two O(n) terms, so the summation must be
    // free of bias (a floating split's leading accumulator, not
    // round-to-nearest, left |dNLL|/n above 1e-6 at n = 30,000, k = 1000)
    ProfileScope ps(kProfVifSyrk, st);
    s = tc_syrk(WE, kk, n, kk, G, vbase + V.Ap, part, hdr, st);
    if (s != VST_OK) return s;
  } else {
    const int64_t chunk = std::max<int64_t>((n + kVifSyrkChunks - 1) / kVifSyrkChunks, 1);
    const int nchunk = (int)std::min<int64_t>(kVifSyrkChunks, (n + chunk - 1) / chunk);
    const int nb = (kk + 63) / 64;
    if (n > 0) {
      ProfileScope ps(kProfVifSyrk, st);
      syrk_kernel<T><<<dim3(nb, nb, nchunk), 256, 0, st>>>(WE, n, kk, chunk, part);
    }
    if (nchunk > 0) syrk_sum_kernel<<<(int)((kk2 + 255) / 256), 256, 0, st>>>(part, nchunk, kk, G);
    else cudaMemsetAsync(G, 0, sizeof(double) * kk2, st);
  }
  make_m_kernel<<<(int)(((int64_t)k * k + 255) / 256 + 1), 256, 0, st>>>(G, k, M, v, z + k);
  s = chol64(M, k, hdr, VST_ENOTSPD, st);
  if (s != VST_OK) return s;
  final_kernel<<<1, 1024, 0, st>>>(M, k, v, z + k, logd, nparts, n, z, nll);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VST_OK : cuda_fail(e, "VIF Woodbury kernels");
}

vst_status vif_nll(const vst_points* pts, const vst_theta* theta, int m, const vst_inducing* ind, int nu,
                   const int32_t* nn, const int32_t* nn_cnt, const double* y, int precision, double* nll, void* ws,
                   cudaStream_t st) {
  return precision == VST_FP64 ? vif_nll_T<double>(pts, theta, m, ind, nu, nn, nn_cnt, y, precision, nll, ws, st)
                               : vif_nll_T<float>(pts, theta, m, ind, nu, nn, nn_cnt, y, precision, nll, ws, st);
}

}  // namespace vst

namespace vst {
vst_status check_theta(const vst_theta* th);
vst_status check_inducing(const vst_inducing* ind);
int nu_code(double nu);

__global__ void widen_kernel(const float* src, int64_t count, double* dst) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count; q += (int64_t)gridDim.x * blockDim.x)
    dst[q] = (double)src[q];
}
}  // namespace vst

using namespace vst;

extern "C" vst_status vif_lowrank_u(const vst_points* pts, const vst_theta* theta, const vst_inducing* ind,
                                    int precision, double* U, double* r, void* ws, size_t ws_bytes, void* stream) {
  if (!pts) return fail(VST_EINVAL, "pts is NULL");
  const int64_t n = pts->n;
  if (n < 0 || n >= (int64_t(1) << 31)) return fail(VST_EINVAL, "n=%lld out of range", (long long)n);
  vst_status s = check_theta(theta);
  if (s != VST_OK) return s;
  if (!ind || ind->k <= 0) return fail(VST_EINVAL, "vif_lowrank_u needs k > 0 inducing points");
  s = check_inducing(ind);
  if (s != VST_OK) return s;
  if (!valid_precision(precision)) return fail(VST_EINVAL, "bad precision %d", precision);
  if (n > 0 && (!pts->xy || !pts->t || !U || !r)) return fail(VST_EINVAL, "NULL array");
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256) return fail(VST_EINVAL, "workspace NULL or not 256-byte aligned");
  const int64_t k = ind->k;
  const WsLayout L = ws_layout(n, 0, k);
  if (ws_bytes < L.total) return fail(VST_ENOMEM, "workspace has %zu bytes, %zu needed", ws_bytes, L.total);
  cudaStream_t st = (cudaStream_t)stream;
  char* base = static_cast<char*>(ws);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(base + L.hdr);
  char* vbase = base + L.vif;
  const VifLayout V = vif_layout(n, 0, k);
  launch_init_header(hdr, st);
  s = vif_lowrank(pts, theta, ind, nu_code(theta->nu), precision, vbase, V, hdr, st);
  if (s != VST_OK) return s;
  if (n == 0) return VST_OK;
  const int64_t count = n * k;
  cudaError_t e;
  if (precision == VST_FP64) {
    e = cudaMemcpyAsync(U, vbase + V.U, sizeof(double) * count, cudaMemcpyDeviceToDevice, st);
  } else {
    widen_kernel<<<(int)std::min<int64_t>((count + 255) / 256, 152 * 64), 256, 0, st>>>(
        reinterpret_cast<const float*>(vbase + V.U), count, U);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(r, vbase + V.r, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? VST_OK : cuda_fail(e, "vif_lowrank_u copies");
}
