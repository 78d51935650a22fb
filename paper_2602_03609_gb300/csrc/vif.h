// Internal declarations of the VIF path (vif.cu).
#pragma once

#include <cuda_runtime.h>

#include "kernels.h"
#include "workspace.h"

namespace vst {

DevTheta dev_theta(const vst_theta* th);
inline DevTheta dev_theta_vif(const vst_theta* th) { return dev_theta(th); }

vst_status vif_knn(const vst_points* pts, const vst_theta* theta, int m, const vst_inducing* ind, int nu,
                   int32_t* nn, int32_t* nn_cnt, int64_t* tie_rows, int64_t tie_cap, char* vbase,
                   const VifLayout& V, WsHeader* hdr, cudaStream_t st);
vst_status vif_factor(const vst_points* pts, const vst_theta* theta, int m, const vst_inducing* ind, int nu,
                      const int32_t* nn, const int32_t* nn_cnt, int precision, double* A, double* D, void* ws,
                      cudaStream_t st);
vst_status vif_nll(const vst_points* pts, const vst_theta* theta, int m, const vst_inducing* ind, int nu,
                   const int32_t* nn, const int32_t* nn_cnt, const double* y, int precision, double* nll, void* ws,
                   cudaStream_t st);

}  // namespace vst
