// Internal launchers shared between the translation units of libvst.
#pragma once

#include <cuda_runtime.h>

#include "rows_impl.cuh"

namespace vst {

constexpr int kRowWarps = 4;          // warps per block of the row kernels
constexpr int64_t kMaxPartialWarps = 1 << 16;

// Launch the fused row kernel for (precision, nu code, padded size, mode) as a
// persistent grid (resident blocks x SMs).  *warps_out = warps launched.
cudaError_t launch_rows(bool mixed, int nu_code, int pm, int mode, const RowArgs& g, cudaStream_t st,
                        int64_t* warps_out);

// Per-point records of the mixed form for rows [0, n) (y may be NULL: zero
// response), and zeroed FP64-fallback flags when flag is not NULL.
void launch_prep_points(int64_t n, const double* xy, const double* t, const double* y, PrepPt* out,
                        uint8_t* flag, cudaStream_t st);

template <typename T, int NU>
cudaError_t launch_rows_tn(int pm, int mode, const RowArgs& g, cudaStream_t st, int64_t* warps_out);

}  // namespace vst
