// Correlation-based Vecchia neighbour selection (Sect. 4.4.1) on the GPU.
//
// For every row i the search returns the min(i, m) predecessors j < i with the
// largest correlation rho_ij = C(h_ij, u_ij) / sigma1^2 under Eq. (2), ranked
// in FP64 with ties broken by the smaller index.  The paper does this with a
// cover tree under d_c = sqrt(1 - |rho|) (Algorithms 1-2); here the points are
// bucketed on a regular space-time grid instead and the search is exact
// because each bucket is skipped only when a rigorous upper bound of rho over
// the bucket falls below the current (m+1)-th best correlation:
//
//   rho(h, u) <= psi(u_lo)^{-(delta+gamma)} * M_nu(c h_lo psi(u_hi)^{-gamma/2})
//
// for every h >= h_lo and u in [u_lo, u_hi]: psi^{-(delta+gamma)} decreases in
// u, M_nu decreases in its argument, and psi^{-gamma/2} decreases in u.  (The
// correlation itself is not monotone in the time lag for h > 0.)
//
// Kernels: bounding box -> bucket keys + per-time-bin minimum index ->
// exclusive scan -> scatter -> per-bucket sort by index (so that the
// predecessors of i in a bucket are a prefix) -> one warp per query.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>

#include "kernels.h"
#include "profile.h"
#include "vif.h"
#include "workspace.h"

namespace vst {

vst_status fail(vst_status s, const char* fmt, ...);
vst_status cuda_fail(cudaError_t e, const char* where);
vst_status check_theta(const vst_theta* th);
vst_status check_inducing(const vst_inducing* ind);
int nu_code(double nu);
void launch_lag_table(const DevTheta& th, LagD* d, LagF* f, cudaStream_t st);
void launch_init_header(WsHeader* h, cudaStream_t st);

struct Grid {
  double xmin, ymin, tmin, cs, tw;
  int ncx, ncy, nt, ncell;
  int int_times;
  float margin;  // absolute slack of the FP32 correlation filter
};

// ---------------------------------------------------------------------------
__global__ void bbox_partial_kernel(const double* xy, const double* t, int64_t n, double* part) {
  double v[6] = {DBL_MAX, -DBL_MAX, DBL_MAX, -DBL_MAX, DBL_MAX, -DBL_MAX};
  int allint = 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = xy[2 * i], y = xy[2 * i + 1], tt = t[i];
    v[0] = fmin(v[0], x); v[1] = fmax(v[1], x);
    v[2] = fmin(v[2], y); v[3] = fmax(v[3], y);
    v[4] = fmin(v[4], tt); v[5] = fmax(v[5], tt);
    allint &= (tt == floor(tt)) && fabs(tt) < 1.0e9;
  }
  __shared__ double sh[6][256];
  __shared__ int shi[256];
  for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] = v[q];
  shi[threadIdx.x] = allint;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      for (int q = 0; q < 6; q += 2) {
        sh[q][threadIdx.x] = fmin(sh[q][threadIdx.x], sh[q][threadIdx.x + s]);
        sh[q + 1][threadIdx.x] = fmax(sh[q + 1][threadIdx.x], sh[q + 1][threadIdx.x + s]);
      }
      shi[threadIdx.x] &= shi[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int q = 0; q < 6; ++q) part[blockIdx.x * 8 + q] = sh[q][0];
    part[blockIdx.x * 8 + 6] = shi[0];
  }
}

__global__ void bbox_final_kernel(const double* part, int nb, double* out) {
  if (threadIdx.x != 0) return;
  double v[7] = {DBL_MAX, -DBL_MAX, DBL_MAX, -DBL_MAX, DBL_MAX, -DBL_MAX, 1.0};
  for (int b = 0; b < nb; ++b) {
    for (int q = 0; q < 6; q += 2) {
      v[q] = fmin(v[q], part[b * 8 + q]);
      v[q + 1] = fmax(v[q + 1], part[b * 8 + q + 1]);
    }
    v[6] = fmin(v[6], part[b * 8 + 6]);
  }
  for (int q = 0; q < 7; ++q) out[q] = v[q];
}

__device__ __forceinline__ int time_bin(const Grid& g, double t) {
  int b = (int)floor((t - g.tmin) / g.tw);
  return min(max(b, 0), g.nt - 1);
}
__device__ __forceinline__ int cell_x(const Grid& g, double x) {
  int c = (int)floor((x - g.xmin) / g.cs);
  return min(max(c, 0), g.ncx - 1);
}
__device__ __forceinline__ int cell_y(const Grid& g, double y) {
  int c = (int)floor((y - g.ymin) / g.cs);
  return min(max(c, 0), g.ncy - 1);
}

__global__ void key_kernel(const double* xy, const double* t, int64_t n, Grid g, int32_t* pbucket,
                           int32_t* counts, int32_t* binmin) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int tb = time_bin(g, t[i]);
    const int b = tb * g.ncell + cell_y(g, xy[2 * i + 1]) * g.ncx + cell_x(g, xy[2 * i]);
    pbucket[i] = b;
    atomicAdd(&counts[b], 1);
    atomicMin(&binmin[tb], (int)i);
  }
}

// exclusive scan, three passes (block scan, scan of block sums, add)
__device__ __forceinline__ int block_excl_scan_1024(int v, int* sh, int* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = sh[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, s, o);
      if (lane >= o) s += y;
    }
    sh[lane] = s;
  }
  __syncthreads();
  const int before = (w > 0 ? sh[w - 1] : 0);
  *total = sh[31];
  return before + x - v;
}

__global__ void scan_blocks_kernel(const int32_t* in, int64_t nb, int32_t* out, int32_t* blocksums) {
  __shared__ int sh[32];
  const int64_t i = blockIdx.x * 1024ll + threadIdx.x;
  const int v = i < nb ? in[i] : 0;
  int total;
  const int ex = block_excl_scan_1024(v, sh, &total);
  if (i < nb) out[i] = ex;
  if (threadIdx.x == 0) blocksums[blockIdx.x] = total;
}

__global__ void scan_sums_kernel(int32_t* sums, int nblk) {
  __shared__ int sh[32];
  const int per = (nblk + 1023) / 1024;
  const int b0 = threadIdx.x * per;
  int s = 0;
  for (int q = 0; q < per; ++q)
    if (b0 + q < nblk) s += sums[b0 + q];
  int total;
  int ex = block_excl_scan_1024(s, sh, &total);
  for (int q = 0; q < per; ++q)
    if (b0 + q < nblk) {
      const int v = sums[b0 + q];
      sums[b0 + q] = ex;
      ex += v;
    }
}

__global__ void scan_add_kernel(int32_t* out, int64_t nb, const int32_t* sums, int32_t total_n) {
  const int64_t i = blockIdx.x * 1024ll + threadIdx.x;
  if (i < nb) out[i] += sums[blockIdx.x];
  if (i == 0) out[nb] = total_n;
}

__global__ void scatter_kernel(int64_t n, const int32_t* pbucket, const int32_t* offsets, int32_t* cursor,
                               int32_t* sidx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int b = pbucket[i];
    sidx[offsets[b] + atomicAdd(&cursor[b], 1)] = (int)i;
  }
}

// sort each bucket by point index (insertion sort; buckets are small) and
// write FP32 coordinates relative to the grid origin
__global__ void sort_buckets_kernel(int64_t nb, const int32_t* offsets, int32_t* sidx, const double* xy, Grid g,
                                    float* sx, float* sy) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
    const int s = offsets[b], e = offsets[b + 1];
    for (int q = s + 1; q < e; ++q) {
      const int v = sidx[q];
      int r = q - 1;
      while (r >= s && sidx[r] > v) {
        sidx[r + 1] = sidx[r];
        --r;
      }
      sidx[r + 1] = v;
    }
    for (int q = s; q < e; ++q) {
      const int j = sidx[q];
      sx[q] = (float)(xy[2 * (int64_t)j] - g.xmin);
      sy[q] = (float)(xy[2 * (int64_t)j + 1] - g.ymin);
    }
  }
}

// ---------------------------------------------------------------------------
struct KnnArgs {
  double inv_s1;  // 1 / sigma1^2 (correlation = covariance / sigma1^2)
  float inv_s1f;
  const double* xy;
  const double* t;
  int64_t n;
  int m;
  DevTheta th;
  const LagD* lagd;
  const LagF* lagf;
  Grid g;
  const int32_t* offsets;
  const int32_t* sidx;
  const float* sx;
  const float* sy;
  const int32_t* binmin;
  int32_t* nn;
  int32_t* nn_cnt;
  int64_t* tie_rows;
  int64_t tie_cap;
  WsHeader* hdr;
  // candidates of query row i are the rows j < min(i, n_cand); queries are the
  // rows row0..n-1, written to nn / nn_cnt at (i - row0)
  int64_t n_cand;
  int64_t row0;
};

template <int NU>
__device__ __forceinline__ float M32(float x) {
  return matern_M<NU, float>(x, __expf(-x) * (1.0f + 1e-6f));  // slightly high: used in upper bounds
}

// correlation amplitude/argument scale for a lag interval, FP64
__device__ __forceinline__ void lag_rho(const KnnArgs& A, double u, double& Prho, double& G) {
  const double ua = fabs(u);
  if (A.g.int_times && ua < kLagTab) {
    const LagD f = A.lagd[(int)ua];
    Prho = f.P * A.inv_s1;
    G = f.G;
  } else {
    const LagD f = lag_factors(A.th, ua);
    Prho = f.P * A.inv_s1;
    G = f.G;
  }
}

template <int NU, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) knn_kernel(KnnArgs A) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
  const int64_t total = (int64_t)gridDim.x * WARPS;
  const Grid& g = A.g;
  const int K = A.m + 1;  // keep m+1 to detect cut-off ties
  const double NEG = -1.0e300;

  __shared__ int sq_all[WARPS][64];
  int* sq = sq_all[threadIdx.x >> 5];
  for (int64_t i = A.row0 + warp; i < A.n; i += total) {
    const int64_t lim = i < A.n_cand ? i : A.n_cand;  // candidates j < lim
    const double xi = A.xy[2 * i], yi = A.xy[2 * i + 1], ti = A.t[i];
    const float xif = (float)(xi - g.xmin), yif = (float)(yi - g.ymin);
    const int qb = time_bin(g, ti), qcx = cell_x(g, xi), qcy = cell_y(g, yi);
    const int rmax = max(max(qcx, g.ncx - 1 - qcx), max(qcy, g.ncy - 1 - qcy));

    double lr = NEG;  // this lane's slot of the top-K list
    int lid = INT_MAX;
    int count = 0;
    double thr = NEG;  // K-th best correlation once the list is full
    float thr_lo = -FLT_MAX;  // thr rounded down to FP32 (for the FP32 filter and bounds)
    int qn = 0;        // queued candidates awaiting the FP64 ranking

    // exact FP64 correlation of the first nf queued candidates (one per lane),
    // merged into the sorted top-K list, then the queue is compacted
    auto flush = [&](int nf) {
      int j = -1;
      double rho64 = NEG;
      if (lane < nf) {
        j = sq[lane];
        const double dx = A.xy[2 * (int64_t)j] - xi, dy = A.xy[2 * (int64_t)j + 1] - yi;
        const double h = sqrt(dx * dx + dy * dy);
        double Pj, Gj;
        lag_rho(A, A.t[j] - ti, Pj, Gj);
        const double x = Gj * h;
        rho64 = Pj * matern_M<NU, double>(x, exp(-x));
      }
      unsigned mm = __ballot_sync(kFull, lane < nf);
      while (mm) {
        const int src = __ffs(mm) - 1;
        mm &= mm - 1;
        const double cr64 = __shfl_sync(kFull, rho64, src);
        const int cj = __shfl_sync(kFull, j, src);
        if (count >= K && cr64 < thr) continue;
        const bool better = lane < count && (lr > cr64 || (lr == cr64 && lid < cj));
        const int p = __popc(__ballot_sync(kFull, better));
        if (p >= K) continue;
        const double ur = __shfl_up_sync(kFull, lr, 1);
        const int uid = __shfl_up_sync(kFull, lid, 1);
        if (lane > p) { lr = ur; lid = uid; }
        if (lane == p) { lr = cr64; lid = cj; }
        count = min(count + 1, K);
        if (count >= K) {
          thr = __shfl_sync(kFull, lr, K - 1);
          thr_lo = __double2float_rd(thr);
        }
      }
      __syncwarp();
      const int rest = qn - nf;
      const int moved = (lane < rest) ? sq[nf + lane] : 0;
      __syncwarp();
      if (lane < rest) sq[lane] = moved;
      __syncwarp();
      qn = rest;
    };

    for (int w0 = 0;; w0 += 32) {
      // lane -> bin in order of increasing lag: offsets 0, -1, +1, -2, +2, ...
      const int seq = w0 + lane;
      const int off = (seq & 1) ? -((seq + 1) >> 1) : (seq >> 1);
      const int bin = qb + off;
      // stop once the smallest lag of this window cannot beat the threshold
      const int lag0 = w0 >> 1;
      if (lag0 > g.nt) break;
      if (count >= K && w0 > 0) {
        double Pl, Gl;
        const double ulo = g.int_times ? (double)lag0 : fmax(0.0, (lag0 - 1) * g.tw);
        lag_rho(A, ulo, Pl, Gl);
        if (Pl + (double)g.margin < thr) break;
      }
      bool vb = bin >= 0 && bin < g.nt && A.binmin[bin] < lim;
      double ulo = 0.0, uhi = 0.0;
      if (vb) {
        if (g.int_times) {
          ulo = uhi = fabs(ti - (g.tmin + (double)bin));
        } else {
          const double b0 = g.tmin + bin * g.tw, b1 = b0 + g.tw;
          ulo = fmax(0.0, fmax(b0 - ti, ti - b1)) * (1.0 - 1e-12);
          uhi = fmax(fabs(ti - b0), fabs(ti - b1)) * (1.0 + 1e-12);
        }
      }
      double Plo = 0.0, Ghi = 0.0;
      if (vb) {
        double t1;
        lag_rho(A, ulo, Plo, t1);
        lag_rho(A, uhi, t1, Ghi);
      }
      const float Plo_f = (float)Plo * (1.0f + 1e-6f), Ghi_f = (float)Ghi * (1.0f - 1e-6f);
      int ring = 0;
      float bound = vb ? Plo_f : -FLT_MAX;

      while (true) {
        // best-first: the (bin, ring) with the largest upper bound
        float bmax = bound;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bmax = fmaxf(bmax, __shfl_xor_sync(kFull, bmax, o));
        if (bmax == -FLT_MAX) break;
        if (count >= K && bmax + g.margin < thr_lo) break;
        const unsigned bm = __ballot_sync(kFull, bound == bmax);
        if (bm == 0u) break;  // defensive: a NaN bound must not stall the loop
        const int bl = __ffs(bm) - 1;
        const int cbin = __shfl_sync(kFull, bin, bl);
        const int cr = __shfl_sync(kFull, ring, bl);
        const float cP = __shfl_sync(kFull, Plo_f, bl), cG = __shfl_sync(kFull, Ghi_f, bl);
        const double cPd = __shfl_sync(kFull, Plo, bl);
        const double cu = __shfl_sync(kFull, ulo, bl);
        const bool exact_lag = g.int_times != 0;
        // per-bin FP32 correlation scale for the filter (exact lag) and FP64 for the rank
        double P64 = 0.0, G64 = 0.0;
        float P32 = 0.f, G32 = 0.f;  // FP32 filter's lag factors (exact integer lag)
        if (exact_lag) {
          const int lg = (int)fabsf((float)cu);
          if (lg < kLagTab) {
            const float4 f = __ldg(reinterpret_cast<const float4*>(A.lagf) + lg);
            P32 = f.x * A.inv_s1f;
            G32 = f.y;
          } else {
            lag_rho(A, cu, P64, G64);
            P32 = (float)P64;
            G32 = (float)G64;
          }
        }
        (void)cPd;

        // enumerate the cells of ring cr around (qcx, qcy), 32 at a time
        const int ncr = cr == 0 ? 1 : 8 * cr;
        for (int cb = 0; cb < ncr; cb += 32) {
          const int e = cb + lane;
          int s = 0, len = 0;
          if (e < ncr) {
            int cx, cy;
            if (cr == 0) {
              cx = qcx; cy = qcy;
            } else {
              const int side = e / (2 * cr), pos = e - side * 2 * cr;
              if (side == 0) { cx = qcx - cr + pos; cy = qcy - cr; }
              else if (side == 1) { cx = qcx + cr; cy = qcy - cr + pos; }
              else if (side == 2) { cx = qcx + cr - pos; cy = qcy + cr; }
              else { cx = qcx - cr; cy = qcy + cr - pos; }
            }
            if (cx >= 0 && cx < g.ncx && cy >= 0 && cy < g.ncy) {
              // exact distance from the query to the cell rectangle (slightly low)
              const float x0 = (float)(cx * g.cs), y0 = (float)(cy * g.cs), csf = (float)g.cs;
              const float ddx = fmaxf(0.0f, fmaxf(x0 - xif, xif - (x0 + csf)));
              const float ddy = fmaxf(0.0f, fmaxf(y0 - yif, yif - (y0 + csf)));
              const float hlo = fmaxf(0.0f, sqrtf(ddx * ddx + ddy * ddy) - 1e-6f * csf);
              const float cbound = cP * M32<NU>(cG * hlo);
              if (count < K || cbound + g.margin >= thr_lo) {
                const int b = cbin * g.ncell + cy * g.ncx + cx;
                s = A.offsets[b];
                int en = A.offsets[b + 1];
                if (en > s && A.sidx[en - 1] >= lim) {  // keep the candidates j < lim only
                  int lo = s, hi = en;
                  while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (A.sidx[mid] < lim) lo = mid + 1; else hi = mid;
                  }
                  en = lo;
                }
                len = en - s;
              }
            }
          }
          // flatten the candidate ranges of the 32 lanes
          int incl = len;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
          }
          const int tot = __shfl_sync(kFull, incl, 31);
          for (int base = 0; base < tot; base += 32) {
            const int c = base + lane;
            const bool act = c < tot;
            int lo = 0;
#pragma unroll
            for (int stp = 16; stp >= 1; stp >>= 1) {
              const int v = __shfl_sync(kFull, incl, lo + stp - 1);
              if (v <= c) lo += stp;
            }
            const int owner = min(lo, 31);
            const int os = __shfl_sync(kFull, s, owner);
            const int oincl = __shfl_sync(kFull, incl, owner);
            const int olen = __shfl_sync(kFull, len, owner);
            int j = -1;
            float rho32 = 0.0f;
            bool pass = false;
            if (act) {
              const int pos = os + (c - (oincl - olen));
              j = A.sidx[pos];
              if (exact_lag) {
                const float dx = A.sx[pos] - xif, dy = A.sy[pos] - yif;
                const float h = sqrtf(dx * dx + dy * dy);
                rho32 = P32 * matern_M<NU, float>(G32 * h, __expf(-G32 * h));
                pass = count < K || rho32 + g.margin + 1e-5f * thr_lo >= thr_lo;
              } else {
                pass = true;
              }
            }
            // queue the candidates that pass the FP32 filter; the exact FP64
            // ranking runs on 32 queued candidates at a time (full lanes)
            const unsigned passm = __ballot_sync(kFull, pass);
            if (passm == 0u) continue;
            if (pass) sq[qn + __popc(passm & ((1u << lane) - 1u))] = j;
            qn += __popc(passm);
            __syncwarp();
            if (qn >= 32) flush(32);
          }
        }
        // before the next pruning decision: rank what is queued once it is
        // worth a warp, or whenever the list is not full yet
        if (qn > 0 && (qn >= 16 || count < K)) flush(qn);
        // advance the chosen lane to its next ring
        if (lane == bl) {
          ring += 1;
          if (ring > rmax) {
            bound = -FLT_MAX;
          } else {
            const float hlb = (float)((ring - 1) * g.cs) * (1.0f - 1e-6f);
            bound = Plo_f * M32<NU>(Ghi_f * fmaxf(hlb, 0.0f));
          }
        }
      }
    }

    while (qn > 0) flush(qn < 32 ? qn : 32);
    // write the sorted neighbour list
    const int want = (int)(lim < (int64_t)A.m ? lim : (int64_t)A.m);
    const int cnt = min(count, A.m);
    const int64_t oi = i - A.row0;
    if (lane < A.m) A.nn[oi * A.m + lane] = lane < cnt ? lid : -1;
    if (lane == 0) {
      A.nn_cnt[oi] = cnt;
      if (cnt != want) report_error(A.hdr, VST_EINTERNAL, i);
    }
    if (count == K) {
      const double rm = __shfl_sync(kFull, lr, A.m - 1);
      const double rm1 = __shfl_sync(kFull, lr, A.m);
      if (lane == 0 && (rm - rm1) <= 1e-12 * fabs(rm)) {
        const unsigned long long slot = atomicAdd(&A.hdr->n_tie, 1ull);
        if (A.tie_rows && (int64_t)slot < A.tie_cap) A.tie_rows[slot] = oi;
      }
    }
  }
}

template <int NU>
static cudaError_t launch_knn(const KnnArgs& A, cudaStream_t st) {
  constexpr int W = 4;
  auto kern = knn_kernel<NU, W>;
  static int grid = 0;
  if (grid == 0) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, W * 32, 0);
    if (e != cudaSuccess) return e;
    grid = std::max(1, per) * sms;
  }
  kern<<<grid, W * 32, 0, st>>>(A);
  return cudaGetLastError();
}

// Bucket grid over the n points and the exact search for query rows
// row0..n-1 among the rows j < min(i, n_cand) (n_cand = n, row0 = 0: the
// Vecchia predecessors of every row).  Synchronises st once (bounding box).
vst_status plain_knn(const double* xy, const double* t, int64_t n, const vst_theta* theta, int m, int32_t* nn,
                     int32_t* nn_cnt, int64_t* tie_rows, int64_t tie_cap, char* base, const WsLayout& L,
                     WsHeader* hdr, int64_t n_cand, int64_t row0, cudaStream_t st) {
  const DevTheta th = dev_theta(theta);
  LagD* lagd = reinterpret_cast<LagD*>(base + L.lagd);
  LagF* lagf = reinterpret_cast<LagF*>(base + L.lagf);
  launch_lag_table(th, lagd, lagf, st);

  // bounding box (one synchronisation)
  double* bpart = reinterpret_cast<double*>(base + L.bbox_part);
  double* bbox = reinterpret_cast<double*>(base + L.bbox);
  const int nbb = (int)std::min<int64_t>(kBBoxBlocks, (n + 255) / 256);
  bbox_partial_kernel<<<nbb, 256, 0, st>>>(xy, t, n, bpart);
  bbox_final_kernel<<<1, 32, 0, st>>>(bpart, nbb, bbox);
  double hb[7];
  cudaError_t e = cudaMemcpyAsync(hb, bbox, sizeof(hb), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "bounding box");
  if (!std::isfinite(hb[0]) || !std::isfinite(hb[1]) || !std::isfinite(hb[2]) || !std::isfinite(hb[3]) ||
      !std::isfinite(hb[4]) || !std::isfinite(hb[5]))
    return fail(VST_EINVAL, "non-finite coordinates or times");

  // grid geometry: unit time bins when the span allows; square spatial cells
  // sized for a few points per (bin, cell) on average
  Grid g{};
  g.xmin = hb[0];
  g.ymin = hb[2];
  g.tmin = hb[4];
  const double wx = std::max(hb[1] - hb[0], 1e-12), wy = std::max(hb[3] - hb[2], 1e-12);
  const double span = hb[5] - hb[4];
  const int64_t nbmax = max_buckets(n);
  // at most nt_cap time bins, so that one spatial cell per bin always fits
  const int64_t nt_cap = std::min<int64_t>(kMaxTimeBins - 1, nbmax);
  const bool unit_bins = span < (double)(nt_cap - 1);
  g.int_times = hb[6] > 0.5 && unit_bins;
  if (unit_bins) {
    g.tw = 1.0;
    g.nt = (int)std::floor(span) + 1;
  } else {
    g.tw = span / (double)(nt_cap - 2);
    g.nt = (int)nt_cap - 1;
  }
  const double per_bin = (double)n / g.nt;
  const double occupancy = 3.0;
  double cs = std::sqrt(wx * wy * occupancy / std::max(per_bin, 1.0));
  g.ncx = g.ncy = 1;
  for (int it = 0; it < 200; ++it) {
    const int64_t ncx = (int64_t)std::floor(wx / cs) + 1, ncy = (int64_t)std::floor(wy / cs) + 1;
    if (ncx * ncy * g.nt <= nbmax && ncx < 65536 && ncy < 65536) {
      g.ncx = (int)ncx;
      g.ncy = (int)ncy;
      break;
    }
    cs *= 1.25;
  }
  cs = std::max(cs, std::max(wx, wy) / std::max(g.ncx, g.ncy) * (1.0 + 1e-12));
  if ((int64_t)g.ncx * g.ncy * g.nt > nbmax) return fail(VST_EINTERNAL, "bucket grid does not fit");
  g.cs = cs;
  g.ncell = g.ncx * g.ncy;
  // FP32 filter slack: coordinates relative to the grid origin carry an
  // absolute error <= (wx + wy) 2^-24 each; the correlation moves by at most
  // c * |dh| * max|M'| <= c * |dh| per unit of h.
  g.margin = (float)(4.0 * theta->c * (wx + wy) * 6.0e-8 + 2.0e-6);

  const int64_t nb = (int64_t)g.ncell * g.nt;
  int32_t* offsets = reinterpret_cast<int32_t*>(base + L.offsets);
  int32_t* cursor = reinterpret_cast<int32_t*>(base + L.cursor);
  int32_t* bsums = reinterpret_cast<int32_t*>(base + L.blocksums);
  int32_t* sidx = reinterpret_cast<int32_t*>(base + L.sidx);
  float* sx = reinterpret_cast<float*>(base + L.sx);
  float* sy = reinterpret_cast<float*>(base + L.sy);
  int32_t* pb = reinterpret_cast<int32_t*>(base + L.pbucket);
  int32_t* binmin = reinterpret_cast<int32_t*>(base + L.binmin);

  e = cudaMemsetAsync(cursor, 0, sizeof(int32_t) * nb, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(binmin, 0x7f, sizeof(int32_t) * g.nt, st);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  const int gridn = (int)std::min<int64_t>((n + 255) / 256, 4096);
  key_kernel<<<gridn, 256, 0, st>>>(xy, t, n, g, pb, cursor, binmin);
  const int nblk = (int)((nb + 1023) / 1024);
  scan_blocks_kernel<<<nblk, 1024, 0, st>>>(cursor, nb, offsets, bsums);
  scan_sums_kernel<<<1, 1024, 0, st>>>(bsums, nblk);
  scan_add_kernel<<<nblk, 1024, 0, st>>>(offsets, nb, bsums, (int32_t)n);
  e = cudaMemsetAsync(cursor, 0, sizeof(int32_t) * nb, st);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  scatter_kernel<<<gridn, 256, 0, st>>>(n, pb, offsets, cursor, sidx);
  const int gridb = (int)std::min<int64_t>((nb + 255) / 256, 8192);
  sort_buckets_kernel<<<gridb, 256, 0, st>>>(nb, offsets, sidx, xy, g, sx, sy);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "bucketing kernels");

  KnnArgs A{};
  A.inv_s1 = 1.0 / theta->sigma1sq;
  A.inv_s1f = (float)A.inv_s1;
  A.xy = xy;
  A.t = t;
  A.n = n;
  A.m = m;
  A.th = th;
  A.lagd = lagd;
  A.lagf = lagf;
  A.g = g;
  A.offsets = offsets;
  A.sidx = sidx;
  A.sx = sx;
  A.sy = sy;
  A.binmin = binmin;
  A.nn = nn;
  A.nn_cnt = nn_cnt;
  A.tie_rows = tie_rows;
  A.tie_cap = tie_rows ? tie_cap : 0;
  A.hdr = hdr;
  A.n_cand = n_cand;
  A.row0 = row0;
  const int nu = nu_code(theta->nu);
  {
    ProfileScope ps(kProfKnn, st);
    e = nu == 0 ? launch_knn<0>(A, st) : nu == 1 ? launch_knn<1>(A, st) : launch_knn<2>(A, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "knn kernel");
  return VST_OK;
}

}  // namespace vst

using namespace vst;

extern "C" vst_status vif_build_neighbors(const vst_points* pts, const vst_theta* theta, int m,
                                          const vst_inducing* ind, int32_t* nn, int32_t* nn_cnt,
                                          int64_t* tie_rows, int64_t tie_cap, void* ws, size_t ws_bytes,
                                          void* stream) {
  if (!pts) return fail(VST_EINVAL, "pts is NULL");
  const int64_t n = pts->n;
  if (n < 0 || n >= (int64_t(1) << 30)) return fail(VST_EINVAL, "n out of range [0, 2^30)");
  if (m < 0 || m > VST_MAX_M) return fail(VST_EINVAL, "m=%d out of range [0, %d]", m, VST_MAX_M);
  vst_status s = check_theta(theta);
  if (s != VST_OK) return s;
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256) return fail(VST_EINVAL, "workspace NULL or not 256-byte aligned");
  const int64_t kind = (ind && ind->k > 0) ? ind->k : 0;
  s = check_inducing(ind);
  if (s != VST_OK) return s;
  if (ws_bytes < vst_workspace_size(n, m, kind)) return fail(VST_ENOMEM, "workspace too small");
  if (n > 0 && (!pts->xy || !pts->t || !nn_cnt || (m > 0 && !nn))) return fail(VST_EINVAL, "NULL array");
  if (tie_cap < 0) return fail(VST_EINVAL, "tie_cap < 0");
  cudaStream_t st = (cudaStream_t)stream;
  const WsLayout L = ws_layout(n, m, 0);
  char* base = static_cast<char*>(ws);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(base + L.hdr);
  launch_init_header(hdr, st);
  if (n == 0) return VST_OK;
  if (m == 0) {
    cudaError_t e = cudaMemsetAsync(nn_cnt, 0, sizeof(int32_t) * n, st);
    return e == cudaSuccess ? VST_OK : cuda_fail(e, "memset");
  }
  if (kind > 0) {
    return vif_knn(pts, theta, m, ind, nu_code(theta->nu), nn, nn_cnt, tie_rows, tie_cap, base, hdr, st);
  }
  return plain_knn(pts->xy, pts->t, n, theta, m, nn, nn_cnt, tie_rows, tie_cap, base, L, hdr, n, 0, st);
}

