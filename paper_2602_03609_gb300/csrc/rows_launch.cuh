// Instantiation helper for the row kernels: one (T, NU) pair per translation
// unit so the heavy fully unrolled kernels compile in parallel.
#pragma once

#include "kernels.h"

namespace vst {

template <typename T, int NU, int PM, int MODE>
static cudaError_t launch_one(const RowArgs& g, cudaStream_t st, int64_t* warps_out) {
  auto kern = rows_kernel<T, NU, PM, MODE, kRowWarps>;
  const size_t smem = rows_smem_bytes<T, PM, kRowWarps>();
  static int grid = 0;  // resident blocks x SMs, computed once per kernel
  if (grid == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRowWarps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t gmax = kMaxPartialWarps / kRowWarps;
    grid = (int)std::min<int64_t>((int64_t)per_sm * sms, gmax);
  }
  static int per_sm_max = 0, sms_count = 0;
  if (per_sm_max == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms_count, cudaDevAttrMultiProcessorCount, dev);
    per_sm_max = std::max(1, grid / std::max(1, sms_count));
  }
  int launch_grid = grid;
  if (g.blocks_per_sm > 0 && g.blocks_per_sm < per_sm_max) launch_grid = g.blocks_per_sm * sms_count;
  kern<<<launch_grid, kRowWarps * 32, smem, st>>>(g);
  *warps_out = (int64_t)launch_grid * kRowWarps;
  return cudaGetLastError();
}

template <typename T, int NU, int PM>
static cudaError_t launch_pm(int mode, const RowArgs& g, cudaStream_t st, int64_t* w) {
  switch (mode) {
    case kModeNll: return launch_one<T, NU, PM, kModeNll>(g, st, w);
    case kModeNllGrad: return launch_one<T, NU, PM, kModeNllGrad>(g, st, w);
    case kModeVifAdj: return launch_one<T, NU, PM, kModeVifAdj>(g, st, w);
    default: return launch_one<T, NU, PM, kModeFactor>(g, st, w);
  }
}

template <typename T, int NU>
cudaError_t launch_rows_tn(int pm, int mode, const RowArgs& g, cudaStream_t st, int64_t* w) {
  switch (padded_pm(pm)) {
    case 8: return launch_pm<T, NU, 8>(mode, g, st, w);
    case 16: return launch_pm<T, NU, 16>(mode, g, st, w);
    case 24: return launch_pm<T, NU, 24>(mode, g, st, w);
    default: return launch_pm<T, NU, 32>(mode, g, st, w);
  }
}

}  // namespace vst
