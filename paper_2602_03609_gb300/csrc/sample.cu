// Vecchia sampling y = B^{-1} D^{1/2} z (Sect. 4.1: Sigma~s = B^{-1} D B^{-T}),
// i.e. y_i = A_i y_N(i) + sqrt(D_i) z_i in row order.  Rows depend on earlier
// rows only, so one persistent kernel claims rows in increasing order from an
// atomic counter and each warp waits (bounded) for the rows its neighbours
// are on.  Every row it waits for has already been claimed by a running warp,
// which by induction on the row index finishes; no two launches wait on each
// other and blocks need not be co-resident.
#include <cuda/atomic>

#include "kernels.h"
#include "profile.h"
#include "workspace.h"

namespace vst {

vst_status fail(vst_status s, const char* fmt, ...);
vst_status cuda_fail(cudaError_t e, const char* where);
vst_status check_common(const vst_points* pts, const vst_theta* theta, int m, const int32_t* nn,
                        const int32_t* nn_cnt, void* ws, size_t ws_bytes, int64_t k);

constexpr long long kSpinLimit = 1ll << 22;  // about a second of polling with backoff

__global__ void sample_kernel(int64_t n, int m, const int32_t* nn, const int32_t* nn_cnt, const double* A,
                              const double* D, const double* z, double* y, int32_t* ready,
                              unsigned long long* counter, WsHeader* hdr, long long spin_limit) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long row = 0;
    if (lane == 0) row = atomicAdd(counter, 1ull);
    row = __shfl_sync(kFull, row, 0);
    if (row >= (unsigned long long)n) break;
    const int64_t i = (int64_t)row;
    const int cnt = nn_cnt[i];
    double term = 0.0;
    bool timed_out = false;
    if (lane < cnt) {
      const int j = nn[i * m + lane];
      if (j >= 0 && j < i) {
        cuda::atomic_ref<int32_t, cuda::thread_scope_device> f(ready[j]);
        long long spins = 0;
        while (f.load(cuda::memory_order_acquire) == 0) {
          if (++spins > spin_limit) { timed_out = true; break; }
          __nanosleep(256);
        }
        term = A[i * m + lane] * __ldcg(y + j);
      } else {
        timed_out = true;  // not a predecessor: reported as an error below
      }
    }
    const bool bad = __any_sync(kFull, timed_out);
    term = warp_sum(term);
    if (lane == 0) {
      const double v = bad ? nan("") : term + sqrt(D[i]) * z[i];
      __stcg(y + i, v);
      if (bad) report_error(hdr, VST_ETIMEOUT, i);
      cuda::atomic_ref<int32_t, cuda::thread_scope_device> f(ready[i]);
      f.store(1, cuda::memory_order_release);
    }
  }
}

}  // namespace vst

using namespace vst;

extern "C" vst_status vecchia_sample_ex(const vst_points* pts, const vst_theta* theta, int m, const int32_t* nn,
                                        const int32_t* nn_cnt, const double* z, double* y, const vst_options* opts,
                                        void* ws, size_t ws_bytes, void* stream) {
  vst_status s = check_common(pts, theta, m, nn, nn_cnt, ws, ws_bytes, 0);
  if (s != VST_OK) return s;
  CallOpts o;
  s = resolve_options(opts, pts->n, false, &o);
  if (s != VST_OK) return s;
  if (opts && (opts->tau != 0 || opts->fallback_rows))
    return fail(VST_EINVAL, "vecchia_sample_ex: only wait_limit applies");
  if (pts->n > 0 && (!z || !y)) return fail(VST_EINVAL, "z/y is NULL");
  const int64_t n = pts->n;
  if (n == 0) return VST_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const WsLayout L = ws_layout(n, m, 0);
  char* base = static_cast<char*>(ws);
  double* A = reinterpret_cast<double*>(base + L.sA);
  double* D = reinterpret_cast<double*>(base + L.sD);
  s = run_rows(pts, theta, m, nn, nn_cnt, nullptr, VST_FP64, kModeFactor, nullptr, nullptr, A, D, ws, st);
  if (s != VST_OK) return s;
  int32_t* ready = reinterpret_cast<int32_t*>(base + L.ready);
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(base + L.counter);
  cudaError_t e = cudaMemsetAsync(ready, 0, sizeof(int32_t) * n, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(base + L.hdr);
  {
    ProfileScope ps(kProfSample, st);
    sample_kernel<<<sms * 4, 256, 0, st>>>(n, m, nn, nn_cnt, A, D, z, y, ready, counter, hdr,
                                           o.wait_limit > 0 ? (long long)o.wait_limit : kSpinLimit);
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? VST_OK : cuda_fail(e, "sample kernel");
}

extern "C" vst_status vecchia_sample(const vst_points* pts, const vst_theta* theta, int m, const int32_t* nn,
                                     const int32_t* nn_cnt, const double* z, double* y, void* ws,
                                     size_t ws_bytes, void* stream) {
  return vecchia_sample_ex(pts, theta, m, nn, nn_cnt, z, y, nullptr, ws, ws_bytes, stream);
}
