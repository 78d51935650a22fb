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

// Per-call options (vst_options) after validation.
struct CallOpts {
  float tau = kDefaultTau;
  int64_t row_begin = 0, row_end = 0;  // rows [row_begin, row_end) of n
  uint8_t* fallback_rows = nullptr;
  int64_t wait_limit = 0;
};
// Validate *o (NULL: defaults) for a call over n rows; a row range other than
// all rows is accepted only when allow_range.
vst_status resolve_options(const vst_options* o, int64_t n, bool allow_range, CallOpts* out);

// The fused row kernels (mixed + FP64 fallback, or FP64) over rows
// [opt->row_begin, opt->row_end) (all n rows when opt is NULL) and the fixed-
// order reduction of their partial sums into nll / grad.
vst_status run_rows(const vst_points* pts, const vst_theta* theta, int m, const int32_t* nn,
                    const int32_t* nn_cnt, const double* y, int precision, int mode, double* nll,
                    double* grad, double* A, double* D, void* ws, cudaStream_t st,
                    const CallOpts* opt = nullptr);

template <typename T, int NU>
cudaError_t launch_rows_tn(int pm, int mode, const RowArgs& g, cudaStream_t st, int64_t* warps_out);

}  // namespace vst
