// Gradient of the VIF negative log-likelihood (Sect. 4.3) with respect to
// (sigma1^2, c, a, gamma, nugget), FP64, by an adjoint through the Woodbury
// terms and the residual blocks.
//
// With Sigma_VIF = U U^T + S, S = B^{-1} D B^{-T} the Vecchia factor of the
// residual R~ = C - U U^T + nugget I, U = Sigma_nk L^{-T}, L L^T = Sigma_kk,
// alpha = Sigma_VIF^{-1} y and Q = Sigma_VIF^{-1} - alpha alpha^T:
//   dNLL = 1/2 <Q, dU U^T + U dU^T> + 1/2 <Q, dS>.
// In terms of what the NLL already computes (W = D^{-1/2} B U, e =
// D^{-1/2} B y, M = I + W^T W, v = W^T e) and Y = W M^{-1}:
//   eps = e - Y v,  beta = y - U M^{-1} v,  s = W^T eps,
//   Q U = B^T F,  F = D^{-1/2} (Y - eps s^T),
//   1/2 <Q, dS> = sum_i Abar_i . dA_i + Dbar_i dD_i,
//     Abar_iq = -(Y_i . U_nn(i,q) + eps_i beta_nn(i,q)) / sqrt(D_i),
//     Dbar_i  = (1 - Y_i . W_i - eps_i^2) / (2 D_i),
// and through each residual block (A_i = K_N^{-1} k, D_i = K_ii - k.A_i)
//   Abar . dA + Dbar dD = sum_pq Wb_pq dK_pq,
//   Wb = Dbar a~ a~^T + (a~ b~^T + b~ a~^T) / 2,  a~ = (-A_i, 1),
//   b~ = (K_N^{-1} Abar_i, 0).
// dK = dC + dnugget I - (dU_p . U_q + U_p . dU_q): the first part is the
// fused row kernel's adjoint pass (kModeVifAdj); the second adds
// -2 Wb U_block to the U sensitivity of the block's rows.  Wb has rank 2, so
// with alpha_i = U_block^T a~ = (B U)_i = sqrt(D_i) W_i, beta_i =
// U_block^T b~ and gamma_i = Dbar_i alpha_i + beta_i / 2 the block adds
// -2 gamma_i to row i and 2 A_iq gamma_i - b~_q alpha_i to its neighbour
// N(i)_q.  Altogether, with Phi_i = F_i - 2 gamma_i,
//   G_U[r] = Phi_r - sum over (i, q) with N(i)_q = r of (A_iq Phi_i + b~_iq alpha_i),
// gathered per row through the reverse neighbour index.  With
// H = G_U L^{-1} and J = H^T U,
//   <G_U, dU> = <H, dSigma_nk> - <J, dL>,  dL = L Phi(L^{-1} dSigma_kk L^{-T})
// (Phi: lower triangle, halved diagonal), and <J, dL> = <Omega, dSigma_kk>,
// Omega = L^{-T} Psi L^{-1}, Psi the symmetric part of L^T J with the strict
// lower triangle halved on each side and the diagonal halved.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "dgemm.cuh"
#include "kernels.h"
#include "profile.h"
#include "vif.h"
#include "workspace.h"

namespace vst {

vst_status fail(vst_status s, const char* fmt, ...);
vst_status cuda_fail(cudaError_t e, const char* where);
vst_status chol64(double* A, int k, WsHeader* hdr, int err_code, cudaStream_t st);
__global__ void trinv_kernel(const double* L, int k, double* X);
void launch_lag_table(const DevTheta& th, LagD* d, LagF* f, cudaStream_t st);
void launch_reduce_partials(const double* p0, int64_t w0, const double* p1, int64_t w1, double nll_const,
                            double* nll, double* grad, cudaStream_t st);
void apply_launch_shape(RowArgs& g, int batched, int precision, int nu, int pm);

namespace {

constexpr int kChunks = kDgemmChunks;

struct GradLayout {
  size_t LinvM, Minv, Y, GU, H, abar, dbar, eps, beta, qd, wv, svec, spart, btil, roff, rcur, rent, bsum,
      t1part, Jpart, J, Kp, Psi, T1, Omega, t2part, grows, ltab, ltabf, xyf, xykf, svf, tcg, tcpart, total;
};

GradLayout grad_layout(int64_t n, int m, int64_t k) {
  GradLayout G{};
  size_t off = 0;
  auto take = [&off](size_t b) {
    const size_t at = off;
    off = (off + b + 255) & ~size_t(255);
    return at;
  };
  const size_t nn = (size_t)std::max<int64_t>(n, 1), kk = (size_t)std::max<int64_t>(k, 1);
  const size_t mm = (size_t)std::max(m, 1);
  G.LinvM = take(8 * kk * kk);
  G.Minv = take(8 * kk * kk);
  G.Y = take(8 * nn * kk);
  G.GU = take(8 * nn * kk);
  G.H = take(8 * nn * kk);
  G.abar = take(8 * nn * mm);
  G.dbar = take(8 * nn);
  G.eps = take(8 * nn);
  G.beta = take(8 * nn);
  G.qd = take(8 * nn);
  G.wv = take(8 * kk);
  G.svec = take(8 * kk);
  G.spart = take(8 * kk * kChunks);
  G.btil = take(8 * nn * mm);
  G.roff = take(8 * (nn + 1));
  G.rcur = take(4 * nn);
  G.rent = take(8 * nn * mm);
  G.bsum = take(8 * (nn / 1024 + 2));
  G.t1part = take(8 * 4 * 4096);
  G.Jpart = take(8 * kk * kk * kChunks);
  G.J = take(8 * kk * kk);
  G.Kp = take(8 * kk * kk);
  G.Psi = take(8 * kk * kk);
  G.T1 = take(8 * kk * kk);
  G.Omega = take(8 * kk * kk);
  G.t2part = take(8 * 4 * 4096);
  G.grows = take(8 * 8);
  G.ltab = take(sizeof(LagD) * (size_t)kVifMaxDays * kk);
  G.ltabf = take(16 * (size_t)kVifMaxDays * kk);
  G.xyf = take(8 * nn);
  G.xykf = take(8 * kk);
  G.svf = take(8 * kk);
  G.tcg = take(tc_operand_bytes(n, k));  // H^T U's second operand (the first in the NLL's Ap)
  G.tcpart = take(tc_gram_part_bytes(k));
  G.total = off;
  return G;
}

// y = A x for a k x k row-major A
__global__ void gemv_kernel(const double* A, const double* x, int k, double* y) {
  const int lane = threadIdx.x & 31;
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= k) return;
  double s = 0.0;
  for (int c = lane; c < k; c += 32) s += A[(int64_t)r * k + c] * x[c];
  s = warp_sum(s);
  if (lane == 0) y[r] = s;
}

// per row: eps = e - Y v, beta = y - U wv, qd = Y . W (T: the storage type of
// Y, W and U; FP64 products and sums)
template <typename T>
__global__ void rowvec_kernel(int64_t n, int k, const T* Y, const T* WE, const T* U, const double* v,
                              const double* wv, const double* y, double* eps, double* beta, double* qd) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w; i < n; i += nw) {
    double a = 0.0, b = 0.0, c = 0.0;
    const T* Yi = Y + i * k;
    const T* Wi = WE + i * (int64_t)(k + 1);
    const T* Ui = U + i * k;
    for (int p = lane; p < k; p += 32) {
      const double yp = (double)Yi[p];
      a = fma(yp, v[p], a);
      b = fma((double)Ui[p], wv[p], b);
      c = fma(yp, (double)Wi[p], c);
    }
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    if (lane == 0) {
      eps[i] = (double)Wi[k] - a;
      beta[i] = y[i] - b;
      qd[i] = c;
    }
  }
}

// s = W^T eps: per row chunk, partial column sums
template <typename T>
__global__ void wteps_kernel(int64_t n, int k, const T* WE, const double* eps, int64_t chunk, double* part) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  const int64_t r0 = (int64_t)blockIdx.y * chunk, r1 = n < r0 + chunk ? n : r0 + chunk;
  double s = 0.0;
  for (int64_t i = r0; i < r1; ++i) s = fma((double)WE[i * (int64_t)(k + 1) + c], eps[i], s);
  part[(int64_t)blockIdx.y * k + c] = s;
}

// Abar and Dbar per row (dot products: T products, summed in T per lane and
// in FP64 across the lanes)
template <typename T>
__global__ void adj_kernel(int64_t n, int m, int k, const int32_t* nn, const int32_t* nn_cnt, const T* Y,
                           const T* U, const double* D, const double* eps, const double* beta,
                           const double* qd, double* abar, double* dbar) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w; i < n; i += nw) {
    const int cnt = min(max(nn_cnt[i], 0), m);
    const double Di = D[i], sd = 1.0 / sqrt(Di);
    const T* Yi = Y + i * k;
    for (int q = 0; q < m; ++q) {
      double val = 0.0;
      if (q < cnt) {
        const int j = nn[i * m + q];
        if (j >= 0 && j < i) {
          T sl = T(0);
          const T* Uj = U + (int64_t)j * k;
          for (int p = lane; p < k; p += 32) sl = fma(Yi[p], Uj[p], sl);
          const double s = warp_sum((double)sl);
          val = -(s + eps[i] * beta[j]) * sd;
        }
      }
      if (lane == 0) abar[i * m + q] = val;
    }
    if (lane == 0) dbar[i] = 0.5 * (1.0 - qd[i] - eps[i] * eps[i]) / Di;
  }
}

// ---- reverse index: for every row r the (block row i, slot q) pairs with
// N(i)_q = r, in increasing (i, q)
__global__ void rcount_kernel(int64_t n, int m, const int32_t* nn, const int32_t* nn_cnt, int64_t* cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = min(max(nn_cnt[i], 0), m);
    for (int q = 0; q < c; ++q) {
      const int j = nn[i * m + q];
      if (j >= 0 && j < i) atomicAdd(reinterpret_cast<unsigned long long*>(&cnt[j + 1]), 1ull);
    }
  }
}
// inclusive scan of cnt[1..n] in place (three passes)
__global__ void rscan_blocks_kernel(int64_t* a, int64_t n, int64_t* bsum) {
  __shared__ int64_t s[1024];
  const int64_t i = blockIdx.x * 1024 + threadIdx.x;
  s[threadIdx.x] = i < n ? a[i] : 0;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int64_t add = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
    __syncthreads();
    s[threadIdx.x] += add;
    __syncthreads();
  }
  if (i < n) a[i] = s[threadIdx.x];
  if (threadIdx.x == 1023) bsum[blockIdx.x] = s[1023];
}
__global__ void rscan_sums_kernel(int64_t* bsum, int nb) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    for (int b = 1; b < nb; ++b) bsum[b] += bsum[b - 1];
}
__global__ void rscan_add_kernel(int64_t* a, int64_t n, const int64_t* bsum) {
  const int64_t i = blockIdx.x * 1024 + threadIdx.x;
  if (i < n && blockIdx.x > 0) a[i] += bsum[blockIdx.x - 1];
}
__global__ void rfill_kernel(int64_t n, int m, const int32_t* nn, const int32_t* nn_cnt, const int64_t* off,
                             int32_t* cur, int2* ent) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = min(max(nn_cnt[i], 0), m);
    for (int q = 0; q < c; ++q) {
      const int j = nn[i * m + q];
      if (j >= 0 && j < i) ent[off[j] + atomicAdd(&cur[j], 1)] = make_int2((int)i, q);
    }
  }
}
__global__ void rsort_kernel(int64_t n, const int64_t* off, int2* ent) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = off[r], b = off[r + 1];
    for (int64_t x = a + 1; x < b; ++x) {
      const int2 v = ent[x];
      int64_t y = x - 1;
      while (y >= a && (ent[y].x > v.x || (ent[y].x == v.x && ent[y].y > v.y))) {
        ent[y + 1] = ent[y];
        --y;
      }
      ent[y + 1] = v;
    }
  }
}

// per row i: alpha_i = sqrt(D_i) W_i (into `alpha`), and Phi_i = F_i - 2 gamma_i
// (in place over Y_i), F_i = (Y_i - eps_i s) / sqrt(D_i), gamma_i = Dbar_i
// alpha_i + beta_i / 2, beta_i = sum_q b~_iq U_N(i)_q.  One warp per row; the
// neighbours' U rows are streamed one at a time (contiguous, 32 columns per
// lane in registers, blocks of 1024 columns).  The per-column update runs in
// T: in the mixed form every operand and both outputs are FP32, and FP64
// arithmetic there (about 11 FP64-pipe operations per column, 1/61 of the
// FP32 rate) took ~20 ms of the kernel at n = 1.1M, k = 1000.  svf: s in T.
template <typename T>
__global__ void __launch_bounds__(256) phi_kernel(int64_t n, int m, int k, const int32_t* nn,
                                                  const int32_t* nn_cnt, const double* D, const double* dbar,
                                                  const double* eps, const T* svf, const T* WE,
                                                  const double* btil, const T* U, T* Y, T* alpha) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w; i < n; i += nw) {
    const int cnt = min(max(nn_cnt[i], 0), m);
    const double Di = D[i];
    const T sd = (T)(1.0 / sqrt(Di)), sq = (T)sqrt(Di), db = (T)dbar[i], ei = (T)eps[i];
    const T* Wi = WE + i * (int64_t)(k + 1);
    for (int cb = 0; cb < k; cb += 1024) {
      T bt[32];
#pragma unroll
      for (int u = 0; u < 32; ++u) bt[u] = T(0);
      for (int q = 0; q < cnt; ++q) {
        const int j = nn[i * m + q];
        if (j < 0 || j >= i) continue;
        const T wq = (T)btil[i * m + q];
        const T* Uj = U + (int64_t)j * k + cb;
#pragma unroll
        for (int u = 0; u < 32; ++u) {
          const int c = u * 32 + lane;
          if (cb + c < k) bt[u] = fma(wq, Uj[c], bt[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < 32; ++u) {
        const int c = cb + u * 32 + lane;
        if (c < k) {
          const T al = sq * Wi[c];
          const T F = (Y[i * k + c] - ei * svf[c]) * sd;
          Y[i * k + c] = F - T(2) * fma(db, al, T(0.5) * bt[u]);
          alpha[i * k + c] = al;
        }
      }
    }
  }
}

// dst = src rounded to T
template <typename T>
__global__ void to_type_kernel(const double* src, int count, T* dst) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < count) dst[q] = (T)src[q];
}

// G_U[r] = Phi_r - sum over the reverse entries (i, q) of r of
// (A_iq Phi_i + b~_iq alpha_i).  One warp per row; each entry's Phi_i and
// alpha_i rows are streamed contiguously into 32 columns per lane held in
// registers (blocks of 1024 columns).
template <typename T>
__global__ void __launch_bounds__(256) gu_kernel(int64_t n, int m, int k, const int64_t* off, const int2* ent,
                                                 const double* A, const double* btil, const T* Phi,
                                                 const T* alpha, T* GU) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w; r < n; r += nw) {
    const int64_t a = off[r], b = off[r + 1];
    for (int cb = 0; cb < k; cb += 1024) {
      T acc[32];
#pragma unroll
      for (int u = 0; u < 32; ++u) {
        const int c = cb + u * 32 + lane;
        acc[u] = c < k ? Phi[r * k + c] : T(0);
      }
      for (int64_t x = a; x < b; ++x) {
        const int2 en = ent[x];
        const int64_t i = en.x;
        const int64_t iq = i * m + en.y;
        const T na = -(T)A[iq], nb = -(T)btil[iq];
        const T* Pi = Phi + i * k + cb;
        const T* Ai = alpha + i * k + cb;
#pragma unroll
        for (int u = 0; u < 32; ++u) {
          const int c = u * 32 + lane;
          if (cb + c < k) acc[u] = fma(nb, Ai[c], fma(na, Pi[c], acc[u]));
        }
      }
#pragma unroll
      for (int u = 0; u < 32; ++u) {
        const int c = cb + u * 32 + lane;
        if (c < k) GU[r * k + c] = acc[u];
      }
    }
  }
}

// covariance of Eq. (2) and its derivatives with respect to (sigma1^2, c, a, gamma)
template <int NU>
__device__ __forceinline__ void cov_derivs(const DevTheta& th, double dx, double dy, double u, double (&d)[4]) {
  const LagD f = lag_factors(th, u);
  const double x = f.G * sqrt(dx * dx + dy * dy);
  const double E = exp(-x);
  const double C = f.P * matern_M<NU, double>(x, E);
  const double X = f.P * matern_xdM<NU, double>(x, E);  // P x M'(x)
  d[0] = C / th.sigma1sq;
  d[1] = X / th.c;
  d[2] = f.Qa * (-th.p * C - 0.5 * th.gamma * X);
  d[3] = -f.L * (C + 0.5 * X);
}

// lag factors (P, G, Qa, L) of Eq. (2) per (data day dmin + d, inducing point
// p), FP64, when every data time is a whole day within kVifMaxDays days (the
// day range of the low-rank step, info)
__global__ void day_factors_kernel(const double* tk, int k, DevTheta th, const int64_t* info, LagD* tab,
                                   float4* tabf) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (info[2] == 0) return;
  if (id >= info[1] * k) return;
  const int64_t d = id / k;
  const int p = (int)(id % k);
  const LagD f = lag_factors(th, (double)(info[0] + d) - tk[p]);
  tab[id] = f;
  tabf[id] = make_float4((float)f.P, (float)f.G, (float)f.Qa, (float)f.L);
}

// coordinates in FP32 (the mixed form's derivative term)
__global__ void coords_f32_kernel(const double* xy, int64_t n, float2* xyf) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    xyf[i] = make_float2((float)xy[2 * i], (float)xy[2 * i + 1]);
}

// the derivatives of Eq. (2) from given lag factors; T = float evaluates the
// spatial part (h, e^-x, the Matern polynomial) in FP32
template <int NU, typename T>
__device__ __forceinline__ void cov_derivs_f(const DevTheta& th, const LagD& f, double dx, double dy, double (&d)[4]) {
  if constexpr (std::is_same<T, float>::value) {
    const float fx = (float)dx, fy = (float)dy;
    const float x = (float)f.G * sqrtf(fx * fx + fy * fy);
    const float E = expf(-x);
    const float P = (float)f.P;
    const float C = P * matern_M<NU, float>(x, E);
    const float X = P * matern_xdM<NU, float>(x, E);
    d[0] = (double)C / th.sigma1sq;
    d[1] = (double)X / th.c;
    d[2] = f.Qa * (-th.p * (double)C - 0.5 * th.gamma * (double)X);
    d[3] = -f.L * ((double)C + 0.5 * (double)X);
  } else {
    const double x = f.G * sqrt(dx * dx + dy * dy);
    const double E = exp(-x);
    const double C = f.P * matern_M<NU, double>(x, E);
    const double X = f.P * matern_xdM<NU, double>(x, E);
    d[0] = C / th.sigma1sq;
    d[1] = X / th.c;
    d[2] = f.Qa * (-th.p * C - 0.5 * th.gamma * X);
    d[3] = -f.L * (C + 0.5 * X);
  }
}

// sum over (i, p) of H[i][p] dSigma_nk[i][p]/dtheta, per block partials;
// one row per block at a time, threads over p; the lag factors from the day
// table when info says it holds.  T = float: the derivatives and 32-term sums
// in FP32 (FP32 coordinates and table), folded into FP64.
template <int NU, typename T>
__global__ void term1_kernel(int64_t n, int k, const double* xy, const double* t, const double* xyk,
                             const double* tk, DevTheta th, const LagD* tab, const float4* tabf, const float2* xyf,
                             const float2* xykf, const int64_t* info, const T* H, double* part) {
  __shared__ double sh[4][256];
  double acc[4] = {0, 0, 0, 0};
  const bool use_tab = info[2] != 0;
  const int64_t d0 = info[0];
  if constexpr (std::is_same<T, float>::value) {
    const float inv_s1 = (float)(1.0 / th.sigma1sq), inv_c = (float)(1.0 / th.c);
    const float pf = (float)th.p, hg = (float)(0.5 * th.gamma);
    float fa[4] = {0.f, 0.f, 0.f, 0.f};
    int cnt = 0;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
      const float2 xi = xyf[i];
      const int64_t day = use_tab ? (int64_t)t[i] - d0 : 0;
      for (int p = threadIdx.x; p < k; p += blockDim.x) {
        float P, G, Qa, L;
        if (use_tab) {
          const float4 f = tabf[day * k + p];
          P = f.x; G = f.y; Qa = f.z; L = f.w;
        } else {
          const LagD f = lag_factors(th, t[i] - tk[p]);
          P = (float)f.P; G = (float)f.G; Qa = (float)f.Qa; L = (float)f.L;
        }
        const float2 zp = xykf[p];
        const float dx = xi.x - zp.x, dy = xi.y - zp.y;
        const float x = G * sqrtf(dx * dx + dy * dy);
        const float E = expf(-x);
        const float C = P * matern_M<NU, float>(x, E);
        const float X = P * matern_xdM<NU, float>(x, E);
        const float h = H[i * k + p];
        fa[0] = fmaf(h, C * inv_s1, fa[0]);
        fa[1] = fmaf(h, X * inv_c, fa[1]);
        fa[2] = fmaf(h, Qa * (-pf * C - hg * X), fa[2]);
        fa[3] = fmaf(h, -L * (C + 0.5f * X), fa[3]);
        if (++cnt == 32) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[j] += (double)fa[j];
            fa[j] = 0.f;
          }
          cnt = 0;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] += (double)fa[j];
  } else {
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
      for (int p = threadIdx.x; p < k; p += blockDim.x) {
        const LagD f = use_tab ? tab[((int64_t)t[i] - d0) * k + p] : lag_factors(th, t[i] - tk[p]);
        double d[4];
        cov_derivs_f<NU, double>(th, f, xy[2 * i] - xyk[2 * p], xy[2 * i + 1] - xyk[2 * p + 1], d);
        const double h = (double)H[i * k + p];
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[j] = fma(h, d[j], acc[j]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) sh[j][threadIdx.x] = acc[j];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int j = 0; j < 4; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int j = 0; j < 4; ++j) part[(int64_t)blockIdx.x * 4 + j] = sh[j][0];
}

// sum over (a, b) of Omega[a][b] dSigma_kk[a][b]/dtheta
template <int NU>
__global__ void term2_kernel(int k, const double* xyk, const double* tk, DevTheta th, const double* Om,
                             double* part) {
  __shared__ double sh[4][256];
  double acc[4] = {0, 0, 0, 0};
  const int64_t total = (int64_t)k * k;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(q / k), b = (int)(q % k);
    double d[4];
    cov_derivs<NU>(th, xyk[2 * a] - xyk[2 * b], xyk[2 * a + 1] - xyk[2 * b + 1], tk[a] - tk[b], d);
    const double o = Om[q];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = fma(o, d[j], acc[j]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) sh[j][threadIdx.x] = acc[j];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int j = 0; j < 4; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int j = 0; j < 4; ++j) part[(int64_t)blockIdx.x * 4 + j] = sh[j][0];
}

// Psi from K' = L^T J: strict lower part halved onto both triangles, diagonal halved
__global__ void psi_kernel(int k, const double* Kp, double* Psi) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= (int64_t)k * k) return;
  const int a = (int)(q / k), b = (int)(q % k);
  Psi[q] = a > b ? 0.5 * Kp[q] : (a < b ? 0.5 * Kp[(int64_t)b * k + a] : 0.5 * Kp[q]);
}

// grad = row-kernel sums + term1 - term2 (first four), nugget from the rows
__global__ void combine_kernel(const double* grows, const double* t1, int n1, const double* t2, int n2,
                               double* grad) {
  const int j = threadIdx.x;
  if (j >= 5) return;
  double v = grows[j];
  if (j < 4) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < n1; ++q) a += t1[q * 4 + j];
    for (int q = 0; q < n2; ++q) b += t2[q * 4 + j];
    v += a - b;
  }
  grad[j] = v;
}

}  // namespace

size_t vif_grad_extra_bytes(int64_t n, int m, int64_t k) { return grad_layout(n, m, k).total; }

// VIF NLL and gradient.  T = double: the FP64 NLL and FP64 throughout.
// T = float: the mixed NLL (U, W and the residual Gram in FP32 from the
// tensor-core path; A_i, D_i refined, M in FP64), the products Y = W M^{-1},
// H = G_U L^{-1} and J = H^T U on the split-BF16 tensor cores (J with
// double-float drains of its accumulators), the gathers in FP32, every other
// n-long reduction and the k x k algebra in FP64.  The workspace is ws_layout(n, m,
// k) followed by the gradient scratch (vif_grad_extra_bytes).
template <typename T>
vst_status vif_nll_grad_T(const vst_points* pts, const vst_theta* theta, int m, const vst_inducing* ind, int nu,
                          const int32_t* nn, const int32_t* nn_cnt, const double* y, int precision, double* nll,
                          double* grad, void* ws, cudaStream_t st) {
  constexpr bool F32 = std::is_same<T, float>::value;
  const int64_t n = pts->n;
  const int k = (int)ind->k;
  vst_status s = vif_nll(pts, theta, m, ind, nu, nn, nn_cnt, y, precision, nll, ws, st);
  if (s != VST_OK) return s;
  if (n == 0) return cudaMemsetAsync(grad, 0, 5 * sizeof(double), st) == cudaSuccess ? VST_OK : VST_ECUDA;
  char* base = static_cast<char*>(ws);
  const WsLayout L = ws_layout(n, m, k);
  char* vb = base + L.vif;
  const VifLayout V = vif_layout(n, m, k);
  char* gb = base + L.total;
  const GradLayout G = grad_layout(n, m, k);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(base + L.hdr);
  auto P = [&](size_t o) { return reinterpret_cast<double*>(gb + o); };
  auto PT = [&](size_t o) { return reinterpret_cast<T*>(gb + o); };
  const double* A = reinterpret_cast<const double*>(base + L.sA);
  const double* D = reinterpret_cast<const double*>(base + L.sD);
  const T* U = reinterpret_cast<const T*>(vb + V.U);
  const double* X = reinterpret_cast<const double*>(vb + V.X);   // L^{-1}
  const double* Lkk = reinterpret_cast<const double*>(vb + V.S);  // L (lower, in place)
  const T* WE = reinterpret_cast<const T*>(vb + V.WE);
  const double* LM = reinterpret_cast<const double*>(vb + V.M);   // Cholesky factor of M
  const double* v = reinterpret_cast<const double*>(vb + V.v);    // W^T e
  const DevTheta th = dev_theta_vif(theta);
  const int64_t gridw = std::min<int64_t>((n + 7) / 8, 65535);  // 8 warps per block of 256
  const int64_t kk2 = (int64_t)k * k;

  // M^{-1} = L_M^{-T} L_M^{-1}
  {
    const int wpb = 4;
    const size_t smem = sizeof(double) * k * wpb;
    if (smem > 48 * 1024) cudaFuncSetAttribute(trinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    trinv_kernel<<<(k + wpb - 1) / wpb, 32 * wpb, smem, st>>>(LM, k, P(G.LinvM));
    gemm_tn(P(G.LinvM), k, P(G.LinvM), k, k, k, k, false, P(G.Jpart), P(G.Minv), st);
  }
  // FP64 form: the dense products on the FP64 tile GEMM
  const T* MinvT = reinterpret_cast<const T*>(P(G.Minv));
  const T* XT = reinterpret_cast<const T*>(X);
  // Y = W M^{-1} (mixed: on the tensor cores, M^{-1} symmetric); wv = M^{-1} v
  const int terms = precision == VST_MIXED_BF16X3 ? 3 : 6;
  if constexpr (F32) {
    s = tc_product(reinterpret_cast<const float*>(WE), k + 1, n, P(G.Minv), 1, k, reinterpret_cast<float*>(PT(G.Y)),
                   terms, vb, V, hdr, st);
    if (s != VST_OK) return s;
  } else {
    gemm_nn(WE, k + 1, MinvT, k, PT(G.Y), k, n, k, k, false, st);
  }
  gemv_kernel<<<(k * 32 + 255) / 256, 256, 0, st>>>(P(G.Minv), v, k, P(G.wv));
  rowvec_kernel<T><<<(unsigned)gridw, 256, 0, st>>>(n, k, PT(G.Y), WE, U, v, P(G.wv), y, P(G.eps), P(G.beta),
                                                    P(G.qd));
  {
    const int64_t chunk = (n + kChunks - 1) / kChunks;
    wteps_kernel<T><<<dim3((k + 255) / 256, kChunks), 256, 0, st>>>(n, k, WE, P(G.eps), chunk, P(G.spart));
    sum_parts_kernel<<<(k + 255) / 256, 256, 0, st>>>(P(G.spart), kChunks, k, P(G.svec));
  }
  adj_kernel<T><<<(unsigned)gridw, 256, 0, st>>>(n, m, k, nn, nn_cnt, PT(G.Y), U, D, P(G.eps), P(G.beta),
                                                 P(G.qd), P(G.abar), P(G.dbar));
  // residual-block pass (FP64 row kernel on the NLL's residual Gram):
  // covariance part of the gradient, b~ out
  {
    LagD* lagd = reinterpret_cast<LagD*>(base + L.lagd);
    LagF* lagf = reinterpret_cast<LagF*>(base + L.lagf);
    launch_lag_table(th, lagd, lagf, st);
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
    g.flag = reinterpret_cast<uint8_t*>(base + L.flag);
    g.hdr = hdr;
    g.tau = kDefaultTau;
    g.partial = reinterpret_cast<double*>(base + L.partial);
    if constexpr (F32) g.gram_f = reinterpret_cast<const float*>(vb + V.gram);
    else g.gram_d = reinterpret_cast<const double*>(vb + V.gram);
    g.abar = P(G.abar);
    g.dbar = P(G.dbar);
    g.btil = P(G.btil);
    int64_t w = 0, w1 = 0;
    cudaError_t e = cudaSuccess;
    if constexpr (F32) {
      // mixed row kernel (the NLL's per-point records and double-float lag
      // table), then the FP64 kernel for the rows it flags
      g.prep = reinterpret_cast<const PrepPt*>(base + L.prep);
      g.lagdf = reinterpret_cast<const float4*>(vb + V.lagdf);
      apply_launch_shape(g, 0, VST_MIXED, nu, m + 1);
      e = cudaMemsetAsync(g.flag, 0, (size_t)n, st);
      if (e == cudaSuccess) e = launch_rows(true, nu, m + 1, kModeVifAdj, g, st, &w);
      if (e != cudaSuccess) return cuda_fail(e, "VIF adjoint row kernel");
      g.partial = reinterpret_cast<double*>(base + L.partial) + kMaxPartialWarps * 8;
      g.fallback_only = 1;
      e = launch_rows(false, nu, m + 1, kModeVifAdj, g, st, &w1);
      if (e != cudaSuccess) return cuda_fail(e, "VIF adjoint fallback kernel");
    } else {
      apply_launch_shape(g, 0, VST_FP64, nu, m + 1);
      e = launch_rows(false, nu, m + 1, kModeVifAdj, g, st, &w);
      if (e != cudaSuccess) return cuda_fail(e, "VIF adjoint row kernel");
    }
    if (w > kMaxPartialWarps || w1 > kMaxPartialWarps) return fail(VST_EINTERNAL, "too many warps");
    double* part0 = reinterpret_cast<double*>(base + L.partial);
    launch_reduce_partials(part0, w, part0 + kMaxPartialWarps * 8, w1, 0.0, P(G.grows) + 5, P(G.grows), st);
  }
  // Phi and alpha per row, then G_U through the reverse index
  to_type_kernel<T><<<(k + 255) / 256, 256, 0, st>>>(P(G.svec), k, PT(G.svf));
  phi_kernel<T><<<(unsigned)gridw, 256, 0, st>>>(n, m, k, nn, nn_cnt, D, P(G.dbar), P(G.eps), PT(G.svf), WE,
                                                 P(G.btil), U, PT(G.Y), PT(G.H));
  {
    int64_t* off = reinterpret_cast<int64_t*>(gb + G.roff);
    int32_t* cur = reinterpret_cast<int32_t*>(gb + G.rcur);
    int2* ent = reinterpret_cast<int2*>(gb + G.rent);
    int64_t* bsum = reinterpret_cast<int64_t*>(gb + G.bsum);
    cudaError_t e = cudaMemsetAsync(off, 0, 8 * (size_t)(n + 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cur, 0, 4 * (size_t)n, st);
    if (e != cudaSuccess) return cuda_fail(e, "memset");
    const unsigned g1 = (unsigned)std::min<int64_t>((n + 255) / 256, 8192);
    rcount_kernel<<<g1, 256, 0, st>>>(n, m, nn, nn_cnt, off);
    const int nb = (int)((n + 1 + 1023) / 1024);
    rscan_blocks_kernel<<<nb, 1024, 0, st>>>(off, n + 1, bsum);
    rscan_sums_kernel<<<1, 32, 0, st>>>(bsum, nb);
    rscan_add_kernel<<<nb, 1024, 0, st>>>(off, n + 1, bsum);
    rfill_kernel<<<g1, 256, 0, st>>>(n, m, nn, nn_cnt, off, cur, ent);
    rsort_kernel<<<g1, 256, 0, st>>>(n, off, ent);
    gu_kernel<T><<<(unsigned)gridw, 256, 0, st>>>(n, m, k, off, ent, A, P(G.btil), PT(G.Y), PT(G.H), PT(G.GU));
  }
  // H = G_U L^{-1} (mixed: on the tensor cores, B[c][p] = (L^{-1})[p][c]);
  // term1 = <H, dSigma_nk>; J = H^T U
  if constexpr (F32) {
    s = tc_product(reinterpret_cast<const float*>(PT(G.GU)), k, n, X, 2, k, reinterpret_cast<float*>(PT(G.H)), terms,
                   vb, V, hdr, st);
    if (s != VST_OK) return s;
  } else {
    gemm_nn(PT(G.GU), k, XT, k, PT(G.H), k, n, k, k, true, st);
  }
  const int nb1 = (int)std::min<int64_t>(n, 4096);
  {
    const int64_t* info = reinterpret_cast<const int64_t*>(vb + V.dinfo);  // day range of the low-rank step
    LagD* tab = reinterpret_cast<LagD*>(gb + G.ltab);
    float4* tabf = reinterpret_cast<float4*>(gb + G.ltabf);
    float2* xyf = reinterpret_cast<float2*>(gb + G.xyf);
    float2* xykf = reinterpret_cast<float2*>(gb + G.xykf);
    day_factors_kernel<<<(unsigned)((kVifMaxDays * (int64_t)k + 255) / 256), 256, 0, st>>>(ind->t, k, th, info, tab,
                                                                                            tabf);
    if constexpr (F32) {
      coords_f32_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(pts->xy, n, xyf);
      coords_f32_kernel<<<(k + 255) / 256, 256, 0, st>>>(ind->xy, k, xykf);
    }
    auto t1 = [&](auto kern) {
      kern<<<nb1, 256, 0, st>>>(n, k, pts->xy, pts->t, ind->xy, ind->t, th, tab, tabf, xyf, xykf, info, PT(G.H),
                                P(G.t1part));
    };
    if (nu == 0) t1(term1_kernel<0, T>);
    else if (nu == 1) t1(term1_kernel<1, T>);
    else t1(term1_kernel<2, T>);
  }
  if constexpr (F32) {
    // (the NLL's operand-part buffers, free once the products above are
    // formed, take H's parts)
    s = tc_gram(reinterpret_cast<const float*>(PT(G.H)), k, reinterpret_cast<const float*>(U), k, n, k, P(G.J),
                vb + V.Ap, gb + G.tcg, P(G.tcpart), hdr, st);
    if (s != VST_OK) return s;
  } else {
    gemm_tn(PT(G.H), k, U, k, n, k, k, false, P(G.Jpart), P(G.J), st);
  }
  // K' = L^T J, Psi, Omega = X^T (Psi X), term2 = <Omega, dSigma_kk>
  gemm_tn(Lkk, k, P(G.J), k, k, k, k, true, P(G.Jpart), P(G.Kp), st);
  psi_kernel<<<(unsigned)((kk2 + 255) / 256), 256, 0, st>>>(k, P(G.Kp), P(G.Psi));
  gemm_nn(P(G.Psi), k, X, k, P(G.T1), k, k, k, k, true, st);
  gemm_tn(X, k, P(G.T1), k, k, k, k, true, P(G.Jpart), P(G.Omega), st);
  const int nb2 = (int)std::min<int64_t>((kk2 + 255) / 256, 4096);
  if (nu == 0) term2_kernel<0><<<nb2, 256, 0, st>>>(k, ind->xy, ind->t, th, P(G.Omega), P(G.t2part));
  else if (nu == 1) term2_kernel<1><<<nb2, 256, 0, st>>>(k, ind->xy, ind->t, th, P(G.Omega), P(G.t2part));
  else term2_kernel<2><<<nb2, 256, 0, st>>>(k, ind->xy, ind->t, th, P(G.Omega), P(G.t2part));
  combine_kernel<<<1, 32, 0, st>>>(P(G.grows), P(G.t1part), nb1, P(G.t2part), nb2, grad);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VST_OK : cuda_fail(e, "VIF gradient kernels");
}

vst_status vif_nll_grad(const vst_points* pts, const vst_theta* theta, int m, const vst_inducing* ind, int nu,
                        const int32_t* nn, const int32_t* nn_cnt, const double* y, int precision, double* nll,
                        double* grad, void* ws, cudaStream_t st) {
  if (precision == VST_FP64)
    return vif_nll_grad_T<double>(pts, theta, m, ind, nu, nn, nn_cnt, y, precision, nll, grad, ws, st);
  return vif_nll_grad_T<float>(pts, theta, m, ind, nu, nn, nn_cnt, y, precision, nll, grad, ws, st);
}

}  // namespace vst
