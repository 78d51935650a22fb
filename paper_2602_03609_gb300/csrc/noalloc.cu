// vecchia_nll_grad_noalloc: the NLL + gradient entry point for callers that
// cannot allocate device memory.  Its scratch memory (status header, lag
// tables, per-warp partial sums, FP64-fallback row flags) lives in one
// file-scope device array instead of a caller-provided workspace.
#include <cuda.h>  // CUresult / CUcontext types of the driver entry point looked up below

#include <mutex>

#include "kernels.h"
#include "profile.h"

namespace vst {

vst_status fail(vst_status s, const char* fmt, ...);
vst_status cuda_fail(cudaError_t e, const char* where);
vst_status check_theta(const vst_theta* th);
DevTheta dev_theta(const vst_theta* th);
int nu_code(double nu);
void launch_lag_table(const DevTheta& th, LagD* d, LagF* f, cudaStream_t st);
void launch_init_header(WsHeader* h, cudaStream_t st);
void launch_reduce_partials(const double* p0, int64_t w0, const double* p1, int64_t w1, double nll_const,
                            double* nll, double* grad, cudaStream_t st);
void apply_launch_shape(RowArgs& g, int batched, int precision, int nu, int pm);
void forced_launch_shape(RowArgs& g);

namespace {

// Layout of the static scratch array (byte offsets, 256-byte aligned).
constexpr size_t kHdrOff = 0;
constexpr size_t kLagDOff = 256;
constexpr size_t kLagFOff = kLagDOff + sizeof(LagD) * kLagTab;
constexpr size_t kPartOff = kLagFOff + sizeof(LagF) * kLagTab;
constexpr size_t kPartBytes = sizeof(double) * 8 * (size_t)kMaxPartialWarps;  // one buffer
constexpr size_t kFlagOff = kPartOff + 2 * kPartBytes;
constexpr size_t kPrepOff = kFlagOff + (size_t)VST_NOALLOC_MAX_N;
constexpr size_t kScratchBytes = kPrepOff + sizeof(PrepPt) * (size_t)VST_NOALLOC_MAX_N;
static_assert(kLagFOff % 256 == 0 && kPartOff % 256 == 0 && kFlagOff % 256 == 0 && kPrepOff % 256 == 0,
              "alignment");

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};  // id of the context the address belongs to (0: unknown)

// cuCtxGetId through the runtime's driver entry point (no link against the
// driver library); NULL if the driver does not provide it
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetIdFn ctx_get_id_fn() {
  static const CtxGetIdFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (CtxGetIdFn) nullptr;
    return reinterpret_cast<CtxGetIdFn>(p);
  }();
  return fn;
}
// id of the current context (unique for the life of the process), 0 if unknown
unsigned long long current_ctx_id() {
  const CtxGetIdFn f = ctx_get_id_fn();
  unsigned long long id = 0;
  if (f == nullptr || f(nullptr, &id) != CUDA_SUCCESS) return 0;
  return id;
}

}  // namespace

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array on the current device.  The host-side
// symbol itself is not a device address: the address is looked up
// (cudaGetSymbolAddress, with the device current) on the first call on each
// device and cached together with the id of the context it belongs to.  A
// later call in another context on that device (after cudaDeviceReset, the
// module is loaded again, possibly at another address) looks it up again;
// so does every call when the context id cannot be read.
static vst_status scratch_address(char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(VST_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  const unsigned long long ctx = current_ctx_id();
  if (g_scratch_ptr[dev] == nullptr || ctx == 0 || ctx != g_scratch_ctx[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    g_scratch_ptr[dev] = p;
    // the lookup makes the device's primary context current if none was
    g_scratch_ctx[dev] = ctx != 0 ? ctx : current_ctx_id();
  }
  *out = static_cast<char*>(g_scratch_ptr[dev]);
  return VST_OK;
}

}  // namespace vst

using namespace vst;

extern "C" size_t vst_noalloc_scratch_bytes(void) { return kScratchBytes; }

extern "C" vst_status vecchia_nll_grad_noalloc(const vst_points* pts, const vst_theta* theta, int m,
                                               const int32_t* nn, const int32_t* nn_cnt, const double* y,
                                               int precision, double* nll, double* grad, void* stream) {
  if (!pts) return fail(VST_EINVAL, "pts is NULL");
  const int64_t n = pts->n;
  if (n < 0) return fail(VST_EINVAL, "n=%lld is negative", (long long)n);
  if (n > VST_NOALLOC_MAX_N)
    return fail(VST_EINVAL, "n=%lld exceeds the no-allocation limit VST_NOALLOC_MAX_N=%d; use vecchia_nll_grad "
                "with a caller-provided workspace", (long long)n, VST_NOALLOC_MAX_N);
  if (m < 0 || m > VST_MAX_M) return fail(VST_EINVAL, "m=%d out of range [0, %d]", m, VST_MAX_M);
  vst_status s = check_theta(theta);
  if (s != VST_OK) return s;
  if (!valid_precision(precision)) return fail(VST_EINVAL, "bad precision %d", precision);
  precision = plain_precision(precision);  // VST_MIXED_BF16X3 only differs for VIF
  if (n > 0 && (!pts->xy || !pts->t || !y || !nn_cnt || (m > 0 && !nn))) return fail(VST_EINVAL, "NULL array");
  if (!nll || !grad) return fail(VST_EINVAL, "nll/grad is NULL");
  char* base = nullptr;
  s = scratch_address(&base);
  if (s != VST_OK) return s;

  cudaStream_t st = (cudaStream_t)stream;
  WsHeader* hdr = reinterpret_cast<WsHeader*>(base + kHdrOff);
  LagD* lagd = reinterpret_cast<LagD*>(base + kLagDOff);
  LagF* lagf = reinterpret_cast<LagF*>(base + kLagFOff);
  double* part0 = reinterpret_cast<double*>(base + kPartOff);
  double* part1 = reinterpret_cast<double*>(base + kPartOff + kPartBytes);
  uint8_t* flag = reinterpret_cast<uint8_t*>(base + kFlagOff);
  const DevTheta th = dev_theta(theta);
  const bool mixed = precision == VST_MIXED;

  // the array keeps the previous call's contents: reset what must start at zero
  launch_init_header(hdr, st);
  launch_lag_table(th, lagd, lagf, st);
  PrepPt* prep = reinterpret_cast<PrepPt*>(base + kPrepOff);
  if (mixed) launch_prep_points(n, pts->xy, pts->t, y, prep, flag, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "launch");

  RowArgs g{};
  g.xy = pts->xy;
  g.t = pts->t;
  g.y = y;
  g.nn = nn;
  g.nn_cnt = nn_cnt;
  g.n = n;
  g.m = m;
  g.th = th;
  g.lagd = lagd;
  g.lagf = lagf;
  g.flag = flag;
  g.hdr = hdr;
  g.tau = kDefaultTau;
  g.offsets = nullptr;
  g.prep = prep;
  const int nu = nu_code(theta->nu);
  apply_launch_shape(g, 0, precision, nu, m + 1);
  forced_launch_shape(g);
  int64_t w0 = 0, w1 = 0;
  if (n > 0) {
    g.partial = part0;
    g.fallback_only = 0;
    e = launch_rows(mixed, nu, m + 1, kModeNllGrad, g, st, &w0);
    if (e != cudaSuccess) return cuda_fail(e, "row kernel");
    if (mixed) {
      g.partial = part1;
      g.fallback_only = 1;
      e = launch_rows(false, nu, m + 1, kModeNllGrad, g, st, &w1);
      if (e != cudaSuccess) return cuda_fail(e, "fallback row kernel");
    }
  }
  if (w0 > kMaxPartialWarps || w1 > kMaxPartialWarps) return fail(VST_EINTERNAL, "too many warps");
  launch_reduce_partials(part0, w0, part1, w1, 0.5 * (double)n * std::log(2.0 * M_PI), nll, grad, st);
  e = cudaGetLastError();
  return e == cudaSuccess ? VST_OK : cuda_fail(e, "reduce kernel");
}

extern "C" vst_status vst_noalloc_status(void* stream, vst_ws_info* info) {
  char* base = nullptr;
  vst_status s = scratch_address(&base);
  if (s != VST_OK) return s;
  return vst_workspace_status(base + kHdrOff, stream, info);
}
