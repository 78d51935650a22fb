// Instantiation helper for the row kernels: one (T, NU) pair per translation
// unit so the heavy fully unrolled kernels compile in parallel.
#pragma once

#include <algorithm>
#include <atomic>

#include "kernels.h"

namespace vst {

template <typename T, int NU, int PM, int MODE>
static cudaError_t launch_one(const RowArgs& g, cudaStream_t st, int64_t* warps_out) {
  auto kern = rows_kernel<T, NU, PM, MODE, kRowWarps>;
  const size_t smem = rows_smem_bytes<T, PM, kRowWarps>();
  // per device: resident blocks per SM << 16 | SM count, found on the first
  // launch on that device (a relaxed atomic: two threads racing the first
  // launch store the same value)
  constexpr int kDevCache = 64;
  static std::atomic<int> shape_cache[kDevCache];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int packed = (dev >= 0 && dev < kDevCache) ? shape_cache[dev].load(std::memory_order_relaxed) : 0;
  if (packed == 0) {
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (smem > 48 * 1024) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRowWarps * 32, smem);
    if (e != cudaSuccess) return e;
    packed = (std::max(1, std::min(per_sm, 255)) << 16) | std::max(1, std::min(sms, 65535));
    if (dev >= 0 && dev < kDevCache) shape_cache[dev].store(packed, std::memory_order_relaxed);
  }
  const int per_sm = packed >> 16, sms_count = packed & 0xffff;
  const int grid = (int)std::min<int64_t>((int64_t)per_sm * sms_count, kMaxPartialWarps / kRowWarps);
  const int per_sm_max = std::max(1, grid / sms_count);
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
