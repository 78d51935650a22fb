// Dense FP64 tile GEMMs (64 x 64 output tiles, 4 x 4 per thread, K step 16)
// shared by the FP64 VIF kernels: A B (gemm_nn), A^T B over long row ranges in
// fixed-order row chunks (gemm_tn, deterministic), A B^T (gemm_nt).  Each
// translation unit that includes this gets its own copies.
#pragma once

#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

namespace vst {
namespace {

constexpr int kDgemmChunks = 32;  // row chunks of the deterministic A^T B
constexpr int kChunksDg = kDgemmChunks;

// ---- dense GEMMs, 64 x 64 output tiles, 4 x 4 per thread, K step 16
// C[M][N] = A[M][K] B[K][N]; b_lower: B[a][b] = 0 for a < b (rows below the
// column tile's first column skipped)
__global__ void __launch_bounds__(256) gemm_nn_kernel(const double* A, int64_t lda, const double* B, int64_t ldb,
                                                      double* C, int64_t ldc, int64_t M, int N, int K, int b_lower) {
  constexpr int BT = 64, BK = 16;
  __shared__ double As[BK][BT + 2], Bs[BK][BT + 2];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.y * BT;
  const int j0 = blockIdx.x * BT;
  double acc[4][4] = {};
  const int kbeg = b_lower ? (j0 / BK) * BK : 0;
  for (int k0 = kbeg; k0 < K; k0 += BK) {
    __syncthreads();
    for (int q = tid; q < BK * BT; q += 256) {
      const int kk = q & (BK - 1), ii = q >> 4;
      As[kk][ii] = (i0 + ii < M && k0 + kk < K) ? A[(i0 + ii) * lda + k0 + kk] : 0.0;
      const int kb = q / BT, jj = q % BT;
      Bs[kb][jj] = (k0 + kb < K && j0 + jj < N) ? B[(int64_t)(k0 + kb) * ldb + j0 + jj] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[kk][ty * 4 + u];
        b[u] = Bs[kk][tx * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t i = i0 + ty * 4 + u;
    if (i >= M) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = j0 + tx * 4 + v;
      if (j < N) C[i * ldc + j] = acc[u][v];
    }
  }
}

// partial C[a][b] = sum over rows i of the chunk of A[i][a] B[i][b]
// (A: rows x Na, B: rows x Nb); a_lower: A[i][a] = 0 for i < a
__global__ void __launch_bounds__(256) gemm_tn_kernel(const double* A, int64_t lda, const double* B, int64_t ldb,
                                                      int64_t rows, int Na, int Nb, int64_t chunk, int a_lower,
                                                      double* part) {
  constexpr int BT = 64, BK = 16;
  __shared__ double As[BK][BT + 2], Bs[BK][BT + 2];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int a0 = blockIdx.y * BT, b0 = blockIdx.x * BT;
  int64_t r0 = (int64_t)blockIdx.z * chunk;
  const int64_t r1 = rows < r0 + chunk ? rows : r0 + chunk;
  if (a_lower && r0 < a0) r0 = r1 < (int64_t)a0 ? r1 : (int64_t)a0;
  double acc[4][4] = {};
  for (int64_t k0 = r0; k0 < r1; k0 += BK) {
    __syncthreads();
    for (int q = tid; q < BK * BT; q += 256) {
      const int kk = q / BT, jj = q % BT;
      const int64_t r = k0 + kk;
      As[kk][jj] = (r < r1 && a0 + jj < Na && (!a_lower || r >= a0 + jj)) ? A[r * lda + a0 + jj] : 0.0;
      Bs[kk][jj] = (r < r1 && b0 + jj < Nb) ? B[r * ldb + b0 + jj] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[kk][ty * 4 + u];
        b[u] = Bs[kk][tx * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
  }
  double* P = part + (int64_t)blockIdx.z * Na * Nb;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int a = a0 + ty * 4 + u;
    if (a >= Na) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int b = b0 + tx * 4 + v;
      if (b < Nb) P[(int64_t)a * Nb + b] = acc[u][v];
    }
  }
}

__global__ void sum_parts_kernel(const double* part, int nparts, int64_t count, double* out) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count; q += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nparts; ++c) s += part[(int64_t)c * count + q];
    out[q] = s;
  }
}

// C[M][N] = A[M][K] B[N][K]^T (both operands K-contiguous); b_lower:
// B[c][p] = 0 for p > c (the K range of a column tile ends at its last column)
__global__ void __launch_bounds__(256) gemm_nt_kernel(const double* A, int64_t lda, const double* B, int64_t ldb,
                                                      double* C, int64_t ldc, int64_t M, int N, int K, int b_lower) {
  constexpr int BT = 64, BK = 16;
  __shared__ double As[BK][BT + 2], Bs[BK][BT + 2];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.y * BT;
  const int j0 = blockIdx.x * BT;
  double acc[4][4] = {};
  const int kend = b_lower ? (K < j0 + BT ? K : j0 + BT) : K;
  for (int k0 = 0; k0 < kend; k0 += BK) {
    __syncthreads();
    for (int q = tid; q < BK * BT; q += 256) {
      const int kk = q & (BK - 1), ii = q >> 4;
      As[kk][ii] = (i0 + ii < M && k0 + kk < K) ? A[(i0 + ii) * lda + k0 + kk] : 0.0;
      Bs[kk][ii] = (j0 + ii < N && k0 + kk < K) ? B[(int64_t)(j0 + ii) * ldb + k0 + kk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[kk][ty * 4 + u];
        b[u] = Bs[kk][tx * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t i = i0 + ty * 4 + u;
    if (i >= M) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = j0 + tx * 4 + v;
      if (j < N) C[i * ldc + j] = acc[u][v];
    }
  }
}

void gemm_nn(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, int64_t M, int N,
             int K, bool b_lower, cudaStream_t st) {
  constexpr int64_t kRowsPerLaunch = 65535 * 64;  // grid.y limit
  for (int64_t r0 = 0; r0 < M; r0 += kRowsPerLaunch) {
    const int64_t rows = std::min(kRowsPerLaunch, M - r0);
    const dim3 grid((unsigned)((N + 63) / 64), (unsigned)((rows + 63) / 64));
    gemm_nn_kernel<<<grid, 256, 0, st>>>(A + r0 * lda, lda, B, ldb, C + r0 * ldc, ldc, rows, N, K, b_lower ? 1 : 0);
  }
}
// C[Na][Nb] = A^T B over `rows` rows, deterministic: kChunksDg row chunks then a fixed-order sum
void gemm_tn(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t rows, int Na, int Nb, bool a_lower,
             double* part, double* C, cudaStream_t st) {
  const int64_t chunk = std::max<int64_t>((rows + kChunksDg - 1) / kChunksDg, 16);
  const int nch = (int)std::max<int64_t>(1, (rows + chunk - 1) / chunk);
  const dim3 grid((unsigned)((Nb + 63) / 64), (unsigned)((Na + 63) / 64), (unsigned)nch);
  gemm_tn_kernel<<<grid, 256, 0, st>>>(A, lda, B, ldb, rows, Na, Nb, chunk, a_lower ? 1 : 0, part);
  const int64_t count = (int64_t)Na * Nb;
  sum_parts_kernel<<<(unsigned)std::min<int64_t>((count + 255) / 256, 4096), 256, 0, st>>>(part, nch, count, C);
}

// C = A B^T, row blocks launched in chunks of the grid's y limit
void gemm_nt(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, int64_t M, int N,
             int K, bool b_lower, cudaStream_t st) {
  constexpr int64_t kRowsPerLaunch = 65535 * 64;
  for (int64_t r0 = 0; r0 < M; r0 += kRowsPerLaunch) {
    const int64_t rows = std::min(kRowsPerLaunch, M - r0);
    const dim3 grid((unsigned)((N + 63) / 64), (unsigned)((rows + 63) / 64));
    gemm_nt_kernel<<<grid, 256, 0, st>>>(A + r0 * lda, lda, B, ldb, C + r0 * ldc, ldc, rows, N, K, b_lower ? 1 : 0);
  }
}

}  // namespace
}  // namespace vst
