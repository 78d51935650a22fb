// RAII event pair around one kernel launch when profiling is enabled.
#pragma once

#include <cuda_runtime.h>

namespace vst {

enum ProfileClass {
  kProfRows = 0,
  kProfFallback = 1,
  kProfKnn = 2,
  kProfSample = 3,
  kProfVifGemm = 4,  // VIF low-rank U GEMM (tensor-core or FP64)
  kProfVifGram = 5,  // VIF per-row residual Gram
  kProfVifSyrk = 6,  // VIF [W e]^T [W e]
  kProfVifFilter = 7,  // VIF residual-correlation candidate filter (tensor cores)
  kProfClasses = 8
};

class ProfileScope {
 public:
  ProfileScope(int cls, cudaStream_t st);
  ~ProfileScope();

 private:
  int cls_;
  cudaStream_t st_;
  int rec_;
};

}  // namespace vst
