// Batched form: many independent datasets, each with its own covariance
// parameters and size, evaluated by one persistent launch of the fused row
// kernel (rows of all datasets in one index space), followed by a segmented
// fixed-order reduction into one NLL and one gradient per dataset.  The whole
// sequence is asynchronous, so it can be captured into a CUDA graph once and
// replayed after each parameter update (vst_graph_* below).  Also: the
// launch-shape autotuner and its cache.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "kernels.h"
#include "profile.h"
#include "workspace.h"

namespace vst {

vst_status fail(vst_status s, const char* fmt, ...);
vst_status cuda_fail(cudaError_t e, const char* where);
int nu_code(double nu);
void launch_init_header(WsHeader* h, cudaStream_t st);
__global__ void lag_table_kernel(const DevTheta* thetas, DevTheta th1, LagD* d, LagF* f);

// ---------------------------------------------------------------------------
// tuned launch shapes
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tuned;  // (batched, prec, nu, pm) -> (bps, chunk)
int env_int(const char* name) {
  const char* v = std::getenv(name);
  return v ? std::atoi(v) : 0;
}
}  // namespace

void apply_launch_shape(RowArgs& g, int batched, int precision, int nu, int pm) {
  g.blocks_per_sm = 0;
  g.row_chunk = 1;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(std::make_tuple(batched, precision, nu, padded_pm(pm)));
    if (it != g_tuned.end()) {
      g.blocks_per_sm = it->second.first;
      g.row_chunk = it->second.second;
    }
  }
  const int eb = env_int("VST_BLOCKS_PER_SM"), ec = env_int("VST_ROW_CHUNK");
  if (eb > 0) g.blocks_per_sm = eb;
  if (ec > 0) g.row_chunk = ec;
}

static void tuned_store(int batched, int precision, int nu, int pm, int bps, int chunk) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tuned[std::make_tuple(batched, precision, nu, padded_pm(pm))] = {bps, chunk};
}

// ---------------------------------------------------------------------------
// batched workspace: header | DevTheta[nsets] | LagD[nsets][kLagTab] |
// LagF[nsets][kLagTab] | per-row results [n][6] (48 B) | flags [n]
struct BatchLayout {
  size_t hdr, th, lagd, lagf, rows, flag, prep, total;
};
static BatchLayout batch_layout(int nsets, int64_t n) {
  BatchLayout L{};
  size_t off = 0;
  auto take = [&off](size_t b) {
    const size_t at = off;
    off = align256(off + b);
    return at;
  };
  const size_t ns = nsets > 0 ? (size_t)nsets : 1, nn = n > 0 ? (size_t)n : 1;
  L.hdr = take(256);
  L.th = take(sizeof(DevTheta) * ns);
  L.lagd = take(sizeof(LagD) * kLagTab * ns);
  L.lagf = take(sizeof(LagF) * kLagTab * ns);
  L.rows = take(48 * nn);
  L.flag = take(nn);
  L.prep = take(sizeof(PrepPt) * nn);
  L.total = off;
  return L;
}

// Validate per-dataset parameters and offsets on the device (they live in
// device memory so that a captured graph can be replayed after an update),
// and derive the kernel-side parameter records.
__global__ void prep_sets_kernel(int nsets, int64_t n_total, const int64_t* offsets, const vst_theta* thetas,
                                 double nu, DevTheta* out, WsHeader* hdr) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d == 0) {
    bool ok = offsets[0] == 0 && offsets[nsets] == n_total;
    for (int q = 0; q < nsets && ok; ++q) ok = offsets[q + 1] >= offsets[q];
    if (!ok) report_error(hdr, VST_EINVAL, -2);
  }
  if (d >= nsets) return;
  const vst_theta th = thetas[d];
  const bool nu_ok = th.nu == nu;  // one Matern order per batch (the kernel is specialised on it)
  const bool ok = isfinite(th.sigma1sq) && th.sigma1sq > 0 && isfinite(th.c) && th.c > 0 && isfinite(th.a) &&
                  th.a > 0 && th.gamma >= 0 && th.gamma <= 1 && isfinite(th.nugget) && th.nugget >= 0 &&
                  th.alpha > 0 && th.alpha <= 1 && isfinite(th.delta) && th.delta >= 0 &&
                  th.delta + th.gamma > 0 && nu_ok;
  if (!ok) report_error(hdr, VST_EINVAL, d);
  DevTheta o;
  o.sigma1sq = ok ? th.sigma1sq : 1.0;
  o.c = ok ? th.c : 1.0;
  o.a = ok ? th.a : 1.0;
  o.gamma = ok ? th.gamma : 0.5;
  o.nugget = ok ? th.nugget : 0.1;
  o.alpha = ok ? th.alpha : 0.5;
  o.delta = ok ? th.delta : 0.5;
  o.nu = ok ? th.nu : 1.5;
  finish_dev_theta(o);
  out[d] = o;
}

// One block per dataset: fixed-order sums of the per-row results.
__global__ void seg_reduce_kernel(int nsets, int64_t n_total, const int64_t* offsets, const double* rows,
                                  const uint8_t* flag, int mixed, double* nll, double* grad) {
  const int d = blockIdx.x;
  if (d >= nsets) return;
  const int64_t b = min(max(offsets[d], (int64_t)0), n_total), e = min(max(offsets[d + 1], b), n_total);
  __shared__ double sh[6][256];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t r = b + threadIdx.x; r < e; r += 256) {
    if (mixed && flag[r] == 0) {
      const float2* f = reinterpret_cast<const float2*>(rows + r * 6);
      for (int q = 0; q < 6; ++q) acc[q] += (double)f[q].x + (double)f[q].y;
    } else {
      for (int q = 0; q < 6; ++q) acc[q] += rows[r * 6 + q];
    }
  }
  for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    nll[d] = 0.5 * (double)(e - b) * log(2.0 * M_PI) + sh[0][0];
    for (int q = 0; q < 5; ++q) grad[(int64_t)d * 5 + q] = sh[q + 1][0];
  }
}

static int g_force_bps = 0, g_force_chunk = 0;  // set by the autotuner while it times a shape

static vst_status batched_setup(int nsets, int64_t n_total, const int64_t* offsets, const vst_theta* thetas,
                                double nu, const double* xy, const double* t, int m, const int32_t* nn,
                                const int32_t* nn_cnt, const double* y, int precision, double* nll, double* grad,
                                void* ws, size_t ws_bytes, cudaStream_t st) {
  if (nsets < 1) return fail(VST_EINVAL, "nsets=%d", nsets);
  if (n_total < 0 || n_total >= (int64_t(1) << 31)) return fail(VST_EINVAL, "n_total out of range");
  if (m < 0 || m > VST_MAX_M) return fail(VST_EINVAL, "m=%d out of range [0, %d]", m, VST_MAX_M);
  if (!offsets || !thetas || !nll || !grad) return fail(VST_EINVAL, "NULL argument");
  if (n_total > 0 && (!xy || !t || !y || !nn_cnt || (m > 0 && !nn))) return fail(VST_EINVAL, "NULL array");
  if (precision != VST_FP64 && precision != VST_MIXED) return fail(VST_EINVAL, "bad precision %d", precision);
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256) return fail(VST_EINVAL, "workspace NULL or not aligned");
  const BatchLayout L = batch_layout(nsets, n_total);
  if (ws_bytes < L.total) return fail(VST_ENOMEM, "workspace has %zu bytes, %zu needed", ws_bytes, L.total);
  char* base = static_cast<char*>(ws);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(base + L.hdr);
  DevTheta* dth = reinterpret_cast<DevTheta*>(base + L.th);
  LagD* lagd = reinterpret_cast<LagD*>(base + L.lagd);
  LagF* lagf = reinterpret_cast<LagF*>(base + L.lagf);
  uint8_t* flag = reinterpret_cast<uint8_t*>(base + L.flag);
  launch_init_header(hdr, st);
  prep_sets_kernel<<<(nsets + 127) / 128, 128, 0, st>>>(nsets, n_total, offsets, thetas, nu, dth, hdr);
  lag_table_kernel<<<dim3((kLagTab + 127) / 128, nsets), 128, 0, st>>>(dth, DevTheta{}, lagd, lagf);
  cudaError_t e = cudaSuccess;
  if (precision == VST_MIXED)
    launch_prep_points(n_total, xy, t, y, reinterpret_cast<PrepPt*>(base + L.prep), flag, st);
  else if (n_total > 0)
    e = cudaMemsetAsync(flag, 0, (size_t)n_total, st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "batched setup");
  return VST_OK;
}

static vst_status launch_batched_rows(RowArgs& g, int nu, int precision, int m, int nsets, const int64_t* offsets,
                                      double* nll, double* grad, cudaStream_t st, uint8_t* fallback_rows) {
  const bool mixed = precision == VST_MIXED;
  apply_launch_shape(g, 1, precision, nu, m + 1);
  if (g_force_bps > 0) g.blocks_per_sm = g_force_bps;
  if (g_force_chunk > 0) g.row_chunk = g_force_chunk;
  int64_t w = 0;
  cudaError_t e = cudaSuccess;
  if (g.n > 0) {
    g.fallback_only = 0;
    {
      ProfileScope ps(kProfRows, st);
      e = launch_rows(mixed, nu, m + 1, kModeNllGrad, g, st, &w);
    }
    if (e != cudaSuccess) return cuda_fail(e, "batched row kernel");
    if (mixed) {
      g.fallback_only = 1;
      ProfileScope ps(kProfFallback, st);
      e = launch_rows(false, nu, m + 1, kModeNllGrad, g, st, &w);
      if (e != cudaSuccess) return cuda_fail(e, "batched fallback kernel");
    }
  }
  seg_reduce_kernel<<<nsets, 256, 0, st>>>(nsets, g.n, offsets, g.row_out, g.flag, mixed ? 1 : 0, nll, grad);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "segmented reduction");
  if (fallback_rows && g.n > 0) {
    e = mixed ? cudaMemcpyAsync(fallback_rows, g.flag, (size_t)g.n, cudaMemcpyDeviceToDevice, st)
              : cudaMemsetAsync(fallback_rows, 0, (size_t)g.n, st);
    if (e != cudaSuccess) return cuda_fail(e, "fallback rows");
  }
  return VST_OK;
}

}  // namespace vst

using namespace vst;

extern "C" size_t vst_workspace_size_batched(int nsets, int64_t n_total, int m) {
  (void)m;
  return batch_layout(nsets, n_total).total;
}

static vst_status batched_entry(int nsets, int64_t n_total, const int64_t* offsets, const vst_theta* thetas,
                                double nu, const double* xy, const double* t, int m, const int32_t* nn,
                                const int32_t* nn_cnt, const double* y, int precision, double* nll, double* grad,
                                void* ws, size_t ws_bytes, cudaStream_t st, const vst_options* opts = nullptr) {
  const int nuc = nu_code(nu);
  if (nuc < 0) return fail(VST_EINVAL, "nu=%g: only 0.5, 1.5, 2.5 are supported", nu);
  CallOpts o;
  vst_status so = resolve_options(opts, n_total, false, &o);
  if (so != VST_OK) return so;
  vst_status s = batched_setup(nsets, n_total, offsets, thetas, nu, xy, t, m, nn, nn_cnt, y, precision, nll, grad,
                               ws, ws_bytes, st);
  if (s != VST_OK) return s;
  const BatchLayout L = batch_layout(nsets, n_total);
  char* base = static_cast<char*>(ws);
  RowArgs g{};
  g.xy = xy;
  g.t = t;
  g.y = y;
  g.nn = nn;
  g.nn_cnt = nn_cnt;
  g.n = n_total;
  g.m = m;
  g.flag = reinterpret_cast<uint8_t*>(base + L.flag);
  g.hdr = reinterpret_cast<WsHeader*>(base + L.hdr);
  g.tau = o.tau;
  g.offsets = offsets;
  g.thetas = reinterpret_cast<DevTheta*>(base + L.th);
  g.lagd_sets = reinterpret_cast<LagD*>(base + L.lagd);
  g.lagf_sets = reinterpret_cast<LagF*>(base + L.lagf);
  g.nsets = nsets;
  g.row_out = reinterpret_cast<double*>(base + L.rows);
  g.prep = reinterpret_cast<const PrepPt*>(base + L.prep);
  return launch_batched_rows(g, nuc, precision, m, nsets, offsets, nll, grad, st, o.fallback_rows);
}

extern "C" vst_status vecchia_nll_grad_batched(int nsets, int64_t n_total, const int64_t* offsets,
                                               const vst_theta* thetas, double nu, const double* xy,
                                               const double* t, int m, const int32_t* nn, const int32_t* nn_cnt,
                                               const double* y, int precision, double* nll, double* grad,
                                               void* ws, size_t ws_bytes, void* stream) {
  return batched_entry(nsets, n_total, offsets, thetas, nu, xy, t, m, nn, nn_cnt, y, precision, nll, grad, ws,
                       ws_bytes, (cudaStream_t)stream);
}

extern "C" vst_status vecchia_nll_grad_batched_ex(int nsets, int64_t n_total, const int64_t* offsets,
                                                  const vst_theta* thetas, double nu, const double* xy,
                                                  const double* t, int m, const int32_t* nn, const int32_t* nn_cnt,
                                                  const double* y, int precision, const vst_options* opts,
                                                  double* nll, double* grad, void* ws, size_t ws_bytes,
                                                  void* stream) {
  return batched_entry(nsets, n_total, offsets, thetas, nu, xy, t, m, nn, nn_cnt, y, precision, nll, grad, ws,
                       ws_bytes, (cudaStream_t)stream, opts);
}

// ---------------------------------------------------------------------------
// CUDA graph of one batched evaluation

struct vst_graph_s {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

extern "C" vst_status vst_graph_capture_nll_grad_batched(int nsets, int64_t n_total, const int64_t* offsets,
                                                         const vst_theta* thetas, double nu, const double* xy,
                                                         const double* t, int m, const int32_t* nn,
                                                         const int32_t* nn_cnt, const double* y, int precision,
                                                         double* nll, double* grad, void* ws, size_t ws_bytes,
                                                         vst_graph* out) {
  if (!out) return fail(VST_EINVAL, "out is NULL");
  *out = nullptr;
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
  // run once outside capture so that one-time kernel set-up (attributes,
  // occupancy queries) happens before capture begins
  vst_status s = batched_entry(nsets, n_total, offsets, thetas, nu, xy, t, m, nn, nn_cnt, y, precision, nll, grad,
                               ws, ws_bytes, cs);
  if (s == VST_OK) e = cudaStreamSynchronize(cs);
  if (s != VST_OK || e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return s != VST_OK ? s : cuda_fail(e, "pre-capture run");
  }
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return cuda_fail(e, "cudaStreamBeginCapture");
  }
  s = batched_entry(nsets, n_total, offsets, thetas, nu, xy, t, m, nn, nn_cnt, y, precision, nll, grad, ws,
                    ws_bytes, cs);
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
  cudaStreamDestroy(cs);
  if (s != VST_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  vst_graph g = new vst_graph_s{graph, exec};
  *out = g;
  return VST_OK;
}

extern "C" vst_status vst_graph_launch(vst_graph g, void* stream) {
  if (!g) return fail(VST_EINVAL, "graph is NULL");
  cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
  return e == cudaSuccess ? VST_OK : cuda_fail(e, "cudaGraphLaunch");
}

extern "C" vst_status vst_graph_destroy(vst_graph g) {
  if (!g) return VST_OK;
  cudaGraphExecDestroy(g->exec);
  cudaGraphDestroy(g->graph);
  delete g;
  return VST_OK;
}

// ---------------------------------------------------------------------------
// autotuner: time each launch shape, keep the fastest

static const int kShapeBps[] = {1, 2, 3, 0};       // 0 = as many blocks as fit
static const int kShapeChunk[] = {1, 4, 16, 64};

template <class F>
static vst_status tune_shapes(F call, cudaStream_t st, vst_tune_result* out) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return fail(VST_ECUDA, "events");
  float best = 3.0e38f;
  int bb = 0, bc = 1;
  vst_status s = VST_OK;
  for (int bps : kShapeBps) {
    for (int ch : kShapeChunk) {
      g_force_bps = bps > 0 ? bps : 1000;
      g_force_chunk = ch;
      s = call(st);  // warm-up
      if (s != VST_OK) break;
      cudaEventRecord(a, st);
      for (int r = 0; r < 3 && s == VST_OK; ++r) s = call(st);
      cudaEventRecord(b, st);
      if (s != VST_OK) break;
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      ms /= 3.0f;
      if (ms < best) {
        best = ms;
        bb = bps;
        bc = ch;
      }
    }
    if (s != VST_OK) break;
  }
  g_force_bps = g_force_chunk = 0;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (s != VST_OK) return s;
  if (out) {
    out->blocks_per_sm = bb;
    out->row_chunk = bc;
    out->ms = best;
  }
  return VST_OK;
}

namespace vst {
// the single-dataset path reads the forced shape too (see apply_launch_shape use in api.cu)
void forced_launch_shape(RowArgs& g) {
  if (g_force_bps > 0) g.blocks_per_sm = g_force_bps;
  if (g_force_chunk > 0) g.row_chunk = g_force_chunk;
}
}  // namespace vst

extern "C" vst_status vst_autotune_nll_grad(const vst_points* pts, const vst_theta* theta, int m,
                                            const int32_t* nn, const int32_t* nn_cnt, const double* y,
                                            int precision, void* ws, size_t ws_bytes, void* stream,
                                            vst_tune_result* out) {
  vst_tune_result r{};
  // the NLL and gradient of the timing runs land in a workspace area that the
  // NLL path does not use (the neighbour search's bounding-box partials)
  const WsLayout L = ws_layout(pts ? pts->n : 0, m, 0);
  if (!pts || !theta || !ws || ws_bytes < L.total) return fail(VST_EINVAL, "bad arguments or workspace too small");
  double* nll = reinterpret_cast<double*>(static_cast<char*>(ws) + L.bbox_part);
  double* grad = nll + 1;
  auto call = [&](cudaStream_t st) {
    return vecchia_nll_grad(pts, theta, m, nullptr, nn, nn_cnt, y, precision, nll, grad, ws, ws_bytes, st);
  };
  vst_status s = tune_shapes(call, (cudaStream_t)stream, &r);
  if (s != VST_OK) return s;
  tuned_store(0, precision, nu_code(theta->nu), m + 1, r.blocks_per_sm, r.row_chunk);
  if (out) *out = r;
  return VST_OK;
}

extern "C" vst_status vst_autotune_nll_grad_batched(int nsets, int64_t n_total, const int64_t* offsets,
                                                    const vst_theta* thetas, double nu, const double* xy,
                                                    const double* t, int m, const int32_t* nn,
                                                    const int32_t* nn_cnt, const double* y, int precision,
                                                    double* nll, double* grad, void* ws, size_t ws_bytes,
                                                    void* stream, vst_tune_result* out) {
  vst_tune_result r{};
  auto call = [&](cudaStream_t st) {
    return batched_entry(nsets, n_total, offsets, thetas, nu, xy, t, m, nn, nn_cnt, y, precision, nll, grad, ws,
                         ws_bytes, st);
  };
  vst_status s = tune_shapes(call, (cudaStream_t)stream, &r);
  if (s != VST_OK) return s;
  tuned_store(1, precision, nu_code(nu), m + 1, r.blocks_per_sm, r.row_chunk);
  if (out) *out = r;
  return VST_OK;
}

extern "C" void vst_autotune_clear(void) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tuned.clear();
}
