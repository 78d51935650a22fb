// Internal declarations of the VIF path (vif.cu).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kernels.h"
#include "workspace.h"

namespace vst {

DevTheta dev_theta(const vst_theta* th);
inline DevTheta dev_theta_vif(const vst_theta* th) { return dev_theta(th); }

// covariance of Eq. (2) for one pair, FP64 (any lag)
template <int NU>
__device__ __forceinline__ double cov64(const DevTheta& th, double dx, double dy, double u) {
  const LagD f = lag_factors(th, u);
  const double x = f.G * sqrt(dx * dx + dy * dy);
  return f.P * matern_M<NU, double>(x, exp(-x));
}

// the same in FP32 for the mixed form (psi powers through log2/exp2)
template <int NU>
__device__ __forceinline__ float cov32(const DevTheta& th, float dx, float dy, float u) {
  const float au = fabsf(u);
  const float l2 = au > 0.f ? log2f(au) : -126.f;
  const float psi = au > 0.f ? fmaf((float)th.a, exp2f(2.0f * (float)th.alpha * l2), 1.0f) : 1.0f;
  const float lp = log2f(psi);
  const float P = (float)th.sigma1sq * exp2f(-(float)th.p * lp);
  const float G = (float)th.c * exp2f(-0.5f * (float)th.gamma * lp);
  const float d2 = dx * dx + dy * dy;
  const float x = G * (d2 >= kFltMinNormal ? d2 * rsqrt_ftz(d2) : 0.f);
  return P * matern_M<NU, float>(x, expf(-x));
}

// U (FP32 [n][k]) of the mixed form by the split-BF16 tensor-core GEMM
// (vif_tc.cu); split_terms = 3 or 6.  Needs X = L^{-1}, the day range and the
// day lag table of the workspace already computed.  Also forms the residual
// variances r_i = sigma1^2 - ||U_i||^2 (workspace r) from the GEMM epilogue.
vst_status lowrank_tc(const vst_points* pts, const vst_theta* theta, const vst_inducing* ind, int nu,
                      int split_terms, char* vbase, const VifLayout& V, WsHeader* hdr, cudaStream_t st);

// C[i][c] = sum_p A[i][p] B[c][p] on the tensor cores (vif_tc.cu), A FP32
// [n][k] with row stride lda, B from the FP64 k x k matrix M (bmode 1: M; 2:
// B[c][p] = M[p][c] of a lower-triangular M), C FP32 [n][k]
vst_status tc_product(const float* A, int64_t lda, int64_t n, const double* M, int bmode, int k, float* C,
                      int split_terms, char* vbase, const VifLayout& V, WsHeader* hdr, cudaStream_t st);

// C = A^T B (FP64 kc x kc) for FP32 A, B [n][kc] (row strides lda, ldb) on
// the tensor cores (vif_tc.cu): fixed-point BF16 parts (three) with an
// exponent per column and 128-row block, split K over the n rows,
// double-float drains of the tensor-memory accumulators, segments summed in
// FP64 in a fixed order.  opa, opb: tc_operand_bytes(n, kc) bytes each
// (workspace.h); part: tc_gram_part_bytes(kc) bytes.
size_t tc_gram_part_bytes(int64_t kc);
vst_status tc_gram(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t n, int kc, double* C,
                   void* opa, void* opb, double* part, WsHeader* hdr, cudaStream_t st);
// C = A^T A (FP64 kc x kc, both triangles) on the same kernel, lower triangle
// of tiles only; opa: tc_operand_bytes(n, kc) bytes.
vst_status tc_syrk(const float* A, int64_t lda, int64_t n, int kc, double* C, void* opa, double* part,
                   WsHeader* hdr, cudaStream_t st);

// mixed VIF: the per-row residual Gram gram[i][pair] (FP32 [n][528]) for
// local blocks of 32 positions on the tensor cores (vif_gram_tc.cu); parts:
// scratch of 3 n vif_kp(k) BF16 values, uscale: n ceil(k / 64) floats
vst_status gram_tc_rows(const int32_t* nn, const int32_t* nn_cnt, int64_t n, int m, int k, const float* U,
                        __nv_bfloat16* parts, float* uscale, float* gram, WsHeader* hdr, cudaStream_t st);

// 2-D TMA map of a row-major BF16 matrix rows x cols (cols contiguous, a
// multiple of 8), box 64 columns x box_rows rows, 128-byte swizzle (vif_tc.cu)
bool tc_make_map_bf16(CUtensorMap* map, const void* ptr, uint64_t rows, uint64_t cols, uint32_t box_rows);

// residual-correlation neighbours (vif_knn.cu); base: the whole workspace
vst_status vif_knn(const vst_points* pts, const vst_theta* theta, int m, const vst_inducing* ind, int nu,
                   int32_t* nn, int32_t* nn_cnt, int64_t* tie_rows, int64_t tie_cap, char* base,
                   WsHeader* hdr, cudaStream_t st);
vst_status vif_lowrank(const vst_points* pts, const vst_theta* theta, const vst_inducing* ind, int nu,
                       int precision, char* vbase, const VifLayout& V, WsHeader* hdr, cudaStream_t st);
vst_status vif_factor(const vst_points* pts, const vst_theta* theta, int m, const vst_inducing* ind, int nu,
                      const int32_t* nn, const int32_t* nn_cnt, int precision, double* A, double* D, void* ws,
                      cudaStream_t st);
vst_status vif_nll(const vst_points* pts, const vst_theta* theta, int m, const vst_inducing* ind, int nu,
                   const int32_t* nn, const int32_t* nn_cnt, const double* y, int precision, double* nll, void* ws,
                   cudaStream_t st);

// VIF NLL and its gradient (vif_grad.cu), FP64 or mixed; the workspace is
// ws_layout(n, m, k) followed by vif_grad_extra_bytes(n, m, k) bytes.
size_t vif_grad_extra_bytes(int64_t n, int m, int64_t k);
vst_status vif_nll_grad(const vst_points* pts, const vst_theta* theta, int m, const vst_inducing* ind, int nu,
                        const int32_t* nn, const int32_t* nn_cnt, const double* y, int precision, double* nll,
                        double* grad, void* ws, cudaStream_t st);

}  // namespace vst
