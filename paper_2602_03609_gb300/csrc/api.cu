// Host side of the C ABI declared in include/vst.h: argument validation,
// workspace layout, and the launch sequence of each entry point.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "kernels.h"
#include "profile.h"
#include "vif.h"
#include "workspace.h"

namespace vst {

static thread_local std::string g_last_error;

void apply_launch_shape(RowArgs& g, int batched, int precision, int nu, int pm);
void forced_launch_shape(RowArgs& g);

vst_status fail(vst_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

vst_status cuda_fail(cudaError_t e, const char* where) {
  return fail(VST_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// small kernels

// Lag table of Eq. (2) for integer lags 0..kLagTab-1 (per dataset in the
// batched form: blockIdx.y = dataset).
__global__ void lag_table_kernel(const DevTheta* thetas, DevTheta th1, LagD* d, LagF* f) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int set = blockIdx.y;
  if (u >= kLagTab) return;
  const DevTheta th = thetas ? thetas[set] : th1;
  const LagD v = lag_factors(th, (double)u);
  d[(int64_t)set * kLagTab + u] = v;
  f[(int64_t)set * kLagTab + u] = LagF{(float)v.P, (float)v.G, (float)v.Qa, (float)v.L};
}

// Fixed-order sum of the per-warp partials (two buffers: main + FP64 fallback)
// into nll and grad.  One block of 256 threads.
__global__ void reduce_partials_kernel(const double* p0, int64_t w0, const double* p1, int64_t w1,
                                       double nll_const, double* nll, double* grad) {
  __shared__ double sh[6][256];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t w = threadIdx.x; w < w0; w += 256)
    for (int q = 0; q < 6; ++q) acc[q] += p0[w * 8 + q];
  for (int64_t w = threadIdx.x; w < w1; w += 256)
    for (int q = 0; q < 6; ++q) acc[q] += p1[w * 8 + q];
  for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (nll) *nll = nll_const + sh[0][0];
    if (grad)
      for (int q = 0; q < 5; ++q) grad[q] = sh[q + 1][0];
  }
}

__global__ void init_header_kernel(WsHeader* h) {
  h->status = 0;
  h->reserved = 0;
  h->bad_row = ~0ull;
  h->n_fallback = 0;
  h->n_tie = 0;
}

// ---------------------------------------------------------------------------

void launch_lag_table(const DevTheta& th, LagD* d, LagF* f, cudaStream_t st) {
  lag_table_kernel<<<dim3((kLagTab + 127) / 128, 1), 128, 0, st>>>(nullptr, th, d, f);
}

void launch_init_header(WsHeader* h, cudaStream_t st) { init_header_kernel<<<1, 1, 0, st>>>(h); }

// Per-point records of the mixed form: x, y coordinates and the response
// split into FP32 hi + lo parts, integer day test (same rule as the FP64 row
// kernel: t integral and |t| < 1e9), fallback flags cleared.
__global__ void prep_points_kernel(int64_t n, const double* xy, const double* t, const double* y, PrepPt* out,
                                   uint8_t* flag) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double2 c = make_double2(xy[2 * i], xy[2 * i + 1]);  // xy need not be 16-byte aligned
    const double tt = t[i];
    const double v = y ? y[i] : 0.0;
    PrepPt p;
    p.xhi = (float)c.x;
    p.xlo = (float)(c.x - (double)p.xhi);
    p.yhi = (float)c.y;
    p.ylo = (float)(c.y - (double)p.yhi);
    p.vhi = (float)v;
    p.vlo = (float)(v - (double)p.vhi);
    const bool tint = (tt == floor(tt)) && fabs(tt) < 1.0e9;
    p.td = tint ? (int)tt : 0;
    p.tint = tint ? 1 : 0;
    float4* o = reinterpret_cast<float4*>(out + i);
    o[0] = make_float4(p.xhi, p.xlo, p.yhi, p.ylo);
    o[1] = make_float4(p.vhi, p.vlo, __int_as_float(p.td), __int_as_float(p.tint));
    if (flag) flag[i] = 0;
  }
}

void launch_prep_points(int64_t n, const double* xy, const double* t, const double* y, PrepPt* out,
                        uint8_t* flag, cudaStream_t st) {
  if (n <= 0) return;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n + 255) / 256, cap = (int64_t)(sms > 0 ? sms : 1) * 8;
  prep_points_kernel<<<(unsigned)(want < cap ? want : cap), 256, 0, st>>>(n, xy, t, y, out, flag);
}

void launch_reduce_partials(const double* p0, int64_t w0, const double* p1, int64_t w1, double nll_const,
                            double* nll, double* grad, cudaStream_t st) {
  reduce_partials_kernel<<<1, 256, 0, st>>>(p0, w0, p1, w1, nll_const, nll, grad);
}

int nu_code(double nu) {
  if (nu == 0.5) return 0;
  if (nu == 1.5) return 1;
  if (nu == 2.5) return 2;
  return -1;
}

vst_status check_theta(const vst_theta* th) {
  if (!th) return fail(VST_EINVAL, "theta is NULL");
  const bool ok = std::isfinite(th->sigma1sq) && th->sigma1sq > 0 && std::isfinite(th->c) && th->c > 0 &&
                  std::isfinite(th->a) && th->a > 0 && th->gamma >= 0 && th->gamma <= 1 &&
                  std::isfinite(th->nugget) && th->nugget >= 0 && th->alpha > 0 && th->alpha <= 1 &&
                  std::isfinite(th->delta) && th->delta >= 0 && (th->delta + th->gamma) > 0;
  if (!ok)
    return fail(VST_EINVAL,
                "invalid covariance parameters (sigma1sq=%g c=%g a=%g gamma=%g nugget=%g alpha=%g delta=%g)",
                th->sigma1sq, th->c, th->a, th->gamma, th->nugget, th->alpha, th->delta);
  if (nu_code(th->nu) < 0) return fail(VST_EINVAL, "nu=%g: only 0.5, 1.5, 2.5 are supported", th->nu);
  return VST_OK;
}

DevTheta dev_theta(const vst_theta* th) {
  DevTheta d;
  d.sigma1sq = th->sigma1sq;
  d.c = th->c;
  d.a = th->a;
  d.gamma = th->gamma;
  d.nugget = th->nugget;
  d.alpha = th->alpha;
  d.delta = th->delta;
  d.nu = th->nu;
  finish_dev_theta(d);
  return d;
}

vst_status check_inducing(const vst_inducing* ind) {
  if (!ind || ind->k <= 0) return VST_OK;
  if (ind->k > kVifMaxK) return fail(VST_EINVAL, "k=%lld inducing points exceeds %lld", (long long)ind->k,
                                     (long long)kVifMaxK);
  if (!ind->xy || !ind->t) return fail(VST_EINVAL, "inducing xy/t is NULL");
  return VST_OK;
}

vst_status check_common(const vst_points* pts, const vst_theta* theta, int m, const int32_t* nn,
                        const int32_t* nn_cnt, void* ws, size_t ws_bytes, int64_t k) {
  if (!pts) return fail(VST_EINVAL, "pts is NULL");
  if (pts->n < 0 || pts->n >= (int64_t(1) << 31)) return fail(VST_EINVAL, "n=%lld out of range", (long long)pts->n);
  if (m < 0 || m > VST_MAX_M) return fail(VST_EINVAL, "m=%d out of range [0, %d]", m, VST_MAX_M);
  vst_status s = check_theta(theta);
  if (s != VST_OK) return s;
  if (pts->n > 0 && (!pts->xy || !pts->t)) return fail(VST_EINVAL, "xy/t is NULL");
  if (pts->n > 0 && (!nn_cnt || (m > 0 && !nn))) return fail(VST_EINVAL, "nn/nn_cnt is NULL");
  if (!ws) return fail(VST_EINVAL, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(VST_EINVAL, "workspace must be 256-byte aligned");
  const size_t need = vst_workspace_size(pts->n, m, k);
  if (ws_bytes < need)
    return fail(VST_ENOMEM, "workspace has %zu bytes, %zu needed", ws_bytes, need);
  return VST_OK;
}

vst_status resolve_options(const vst_options* o, int64_t n, bool allow_range, CallOpts* out) {
  CallOpts c;
  c.row_end = n;
  if (o) {
    if (!(o->tau == o->tau)) return fail(VST_EINVAL, "options: tau is NaN");
    if (o->tau > 0) c.tau = o->tau < 3.0e38 ? (float)o->tau : 3.0e38f;
    const int64_t b = o->row_begin, e = o->row_end > 0 ? o->row_end : n;
    if (b != 0 || e != n) {
      if (!allow_range) return fail(VST_EINVAL, "options: a row range is not supported by this call");
      if (b < 0 || b > e || e > n)
        return fail(VST_EINVAL, "options: row range [%lld, %lld) not within [0, %lld]", (long long)b,
                    (long long)e, (long long)n);
    }
    if (o->row_end < 0) return fail(VST_EINVAL, "options: row_end=%lld is negative", (long long)o->row_end);
    if (o->wait_limit < 0) return fail(VST_EINVAL, "options: wait_limit is negative");
    c.row_begin = b;
    c.row_end = e;
    c.fallback_rows = o->fallback_rows;
    c.wait_limit = o->wait_limit;
  }
  *out = c;
  return VST_OK;
}

// Runs the row kernels (mixed + FP64 fallback, or FP64) and the reduction.
vst_status run_rows(const vst_points* pts, const vst_theta* theta, int m, const int32_t* nn,
                    const int32_t* nn_cnt, const double* y, int precision, int mode, double* nll,
                    double* grad, double* A, double* D, void* ws, cudaStream_t st, const CallOpts* opt) {
  WsLayout L = ws_layout(pts->n, m, 0);
  char* base = static_cast<char*>(ws);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(base + L.hdr);
  LagD* lagd = reinterpret_cast<LagD*>(base + L.lagd);
  LagF* lagf = reinterpret_cast<LagF*>(base + L.lagf);
  double* part0 = reinterpret_cast<double*>(base + L.partial);
  double* part1 = part0 + kMaxPartialWarps * 8;
  uint8_t* flag = reinterpret_cast<uint8_t*>(base + L.flag);
  // rows [rb, re): the per-row arrays are addressed from rb (RowArgs::out0),
  // the points (neighbours of any earlier row) from 0
  const int64_t rb = opt ? opt->row_begin : 0, re = opt ? opt->row_end : pts->n;
  const DevTheta th = dev_theta(theta);
  const int nu = nu_code(theta->nu);
  const bool mixed = precision == VST_MIXED;

  init_header_kernel<<<1, 1, 0, st>>>(hdr);
  lag_table_kernel<<<dim3((kLagTab + 127) / 128, 1), 128, 0, st>>>(nullptr, th, lagd, lagf);
  PrepPt* prep = reinterpret_cast<PrepPt*>(base + L.prep);
  if (mixed) launch_prep_points(re, pts->xy, pts->t, mode == kModeFactor ? nullptr : y, prep, flag, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "launch");

  RowArgs g{};
  g.xy = pts->xy;
  g.t = pts->t;
  g.y = y;
  g.nn = nn ? nn + rb * m : nn;
  g.nn_cnt = nn_cnt ? nn_cnt + rb : nn_cnt;
  g.n = re;
  g.out0 = rb;
  g.m = m;
  g.th = th;
  g.lagd = lagd;
  g.lagf = lagf;
  g.A = A ? A + rb * m : A;
  g.D = D ? D + rb : D;
  g.flag = flag;
  g.hdr = hdr;
  g.tau = opt ? opt->tau : kDefaultTau;
  g.offsets = nullptr;
  g.prep = prep;
  const int pm = m + 1;
  apply_launch_shape(g, 0, precision, nu, pm);
  forced_launch_shape(g);
  int64_t w0 = 0, w1 = 0;
  if (re > rb) {
    g.partial = part0;
    g.fallback_only = 0;
    {
      ProfileScope ps(kProfRows, st);
      e = launch_rows(mixed, nu, pm, mode, g, st, &w0);
    }
    if (e != cudaSuccess) return cuda_fail(e, "row kernel");
    if (mixed) {
      g.partial = part1;
      g.fallback_only = 1;
      {
        ProfileScope ps(kProfFallback, st);
        e = launch_rows(false, nu, pm, mode, g, st, &w1);
      }
      if (e != cudaSuccess) return cuda_fail(e, "fallback row kernel");
    }
  }
  if (mode != kModeFactor) {
    const double c = 0.5 * (double)(re - rb) * std::log(2.0 * M_PI);
    reduce_partials_kernel<<<1, 256, 0, st>>>(part0, w0, part1, w1, c, nll,
                                               mode == kModeNllGrad ? grad : nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "reduce kernel");
  }
  if (opt && opt->fallback_rows && re > rb) {
    // the flags of rows rb.. sit at flag[0..) (indexed like the per-row arrays)
    e = mixed ? cudaMemcpyAsync(opt->fallback_rows + rb, flag, (size_t)(re - rb), cudaMemcpyDeviceToDevice, st)
              : cudaMemsetAsync(opt->fallback_rows + rb, 0, (size_t)(re - rb), st);
    if (e != cudaSuccess) return cuda_fail(e, "fallback rows");
  }
  return VST_OK;
}

cudaError_t launch_rows(bool mixed, int nu, int pm, int mode, const RowArgs& g, cudaStream_t st, int64_t* w) {
  if (mixed) {
    if (nu == 0) return launch_rows_tn<float, 0>(pm, mode, g, st, w);
    if (nu == 1) return launch_rows_tn<float, 1>(pm, mode, g, st, w);
    return launch_rows_tn<float, 2>(pm, mode, g, st, w);
  }
  if (nu == 0) return launch_rows_tn<double, 0>(pm, mode, g, st, w);
  if (nu == 1) return launch_rows_tn<double, 1>(pm, mode, g, st, w);
  return launch_rows_tn<double, 2>(pm, mode, g, st, w);
}

}  // namespace vst

using namespace vst;

extern "C" {

const char* vst_last_error(void) { return g_last_error.c_str(); }

int vst_version(void) { return 100; }

vst_status vst_theta_from_ranges(double sigma1sq, double range_s, double range_t, double gamma, double nugget,
                                 double alpha, double delta, double nu, vst_theta* out) {
  if (!out) return fail(VST_EINVAL, "out is NULL");
  if (!(range_s > 0) || !(range_t > 0) || !(delta + gamma > 0)) return fail(VST_EINVAL, "invalid ranges");
  // x* with M_nu(x*) = 0.05: Newton on log M_nu, M_nu decreasing on x > 0
  const int code = nu_code(nu);
  if (code < 0) return fail(VST_EINVAL, "nu=%g unsupported", nu);
  auto M = [code](double x) {
    if (code == 0) return std::exp(-x);
    if (code == 1) return (1 + x) * std::exp(-x);
    return (1 + x + x * x / 3) * std::exp(-x);
  };
  auto xdlogM = [code](double x) {  // x * d/dx log M
    if (code == 0) return -x;
    if (code == 1) return -x * x / (1 + x);
    return -(x * x / 3) * (1 + x) / (1 + x + x * x / 3);
  };
  double x = 3.0;
  for (int it = 0; it < 100; ++it) {
    const double f = std::log(M(x)) - std::log(0.05);
    const double step = f * x / xdlogM(x);
    x -= step;
    if (std::fabs(step) < 1e-15 * x) break;
  }
  out->sigma1sq = sigma1sq;
  out->c = x / range_s;
  out->a = (std::pow(0.05, -1.0 / (delta + gamma)) - 1.0) / std::pow(range_t, 2.0 * alpha);
  out->gamma = gamma;
  out->nugget = nugget;
  out->alpha = alpha;
  out->delta = delta;
  out->nu = nu;
  return VST_OK;
}

size_t vst_workspace_size(int64_t n, int m, int64_t k) { return ws_layout(n, m, k).total; }

size_t vst_workspace_size_vif_grad(int64_t n, int m, int64_t k) {
  return ws_layout(n, m, k).total + vif_grad_extra_bytes(n, m, k);
}

vst_status vecchia_factor(const vst_points* pts, const vst_theta* theta, int m, const vst_inducing* ind,
                          const int32_t* nn, const int32_t* nn_cnt, int precision, double* A, double* D,
                          void* ws, size_t ws_bytes, void* stream) {
  const int64_t k = (ind && ind->k > 0) ? ind->k : 0;
  vst_status s = check_inducing(ind);
  if (s == VST_OK) s = check_common(pts, theta, m, nn, nn_cnt, ws, ws_bytes, k);
  if (s != VST_OK) return s;
  if (!valid_precision(precision)) return fail(VST_EINVAL, "bad precision %d", precision);
  if (pts->n > 0 && (!D || (m > 0 && !A))) return fail(VST_EINVAL, "A/D is NULL");
  if (k > 0) {
    const WsLayout L = ws_layout(pts->n, m, k);
    launch_init_header(reinterpret_cast<WsHeader*>(static_cast<char*>(ws) + L.hdr), (cudaStream_t)stream);
    return vif_factor(pts, theta, m, ind, nu_code(theta->nu), nn, nn_cnt, precision, A, D, ws, (cudaStream_t)stream);
  }
  return run_rows(pts, theta, m, nn, nn_cnt, nullptr, plain_precision(precision), kModeFactor, nullptr, nullptr, A,
                  D, ws, (cudaStream_t)stream);
}

vst_status vecchia_nll(const vst_points* pts, const vst_theta* theta, int m, const vst_inducing* ind,
                       const int32_t* nn, const int32_t* nn_cnt, const double* y, int precision, double* nll,
                       void* ws, size_t ws_bytes, void* stream) {
  const int64_t k = (ind && ind->k > 0) ? ind->k : 0;
  vst_status s = check_inducing(ind);
  if (s == VST_OK) s = check_common(pts, theta, m, nn, nn_cnt, ws, ws_bytes, k);
  if (s != VST_OK) return s;
  if (!valid_precision(precision)) return fail(VST_EINVAL, "bad precision %d", precision);
  if (!nll || (pts->n > 0 && !y)) return fail(VST_EINVAL, "y/nll is NULL");
  if (k > 0) {
    const WsLayout L = ws_layout(pts->n, m, k);
    launch_init_header(reinterpret_cast<WsHeader*>(static_cast<char*>(ws) + L.hdr), (cudaStream_t)stream);
    return vif_nll(pts, theta, m, ind, nu_code(theta->nu), nn, nn_cnt, y, precision, nll, ws, (cudaStream_t)stream);
  }
  return run_rows(pts, theta, m, nn, nn_cnt, y, plain_precision(precision), kModeNll, nll, nullptr, nullptr,
                  nullptr, ws, (cudaStream_t)stream);
}

vst_status vecchia_nll_grad(const vst_points* pts, const vst_theta* theta, int m, const vst_inducing* ind,
                            const int32_t* nn, const int32_t* nn_cnt, const double* y, int precision, double* nll,
                            double* grad, void* ws, size_t ws_bytes, void* stream) {
  const int64_t k = (ind && ind->k > 0) ? ind->k : 0;
  vst_status s = check_inducing(ind);
  if (s == VST_OK) s = check_common(pts, theta, m, nn, nn_cnt, ws, ws_bytes, k);
  if (s != VST_OK) return s;
  if (!valid_precision(precision)) return fail(VST_EINVAL, "bad precision %d", precision);
  if (!nll || !grad || (pts->n > 0 && !y)) return fail(VST_EINVAL, "y/nll/grad is NULL");
  if (k > 0) {
    const size_t need = vst_workspace_size_vif_grad(pts->n, m, k);
    if (ws_bytes < need) return fail(VST_ENOMEM, "workspace has %zu bytes, %zu needed", ws_bytes, need);
    const WsLayout L = ws_layout(pts->n, m, k);
    launch_init_header(reinterpret_cast<WsHeader*>(static_cast<char*>(ws) + L.hdr), (cudaStream_t)stream);
    return vif_nll_grad(pts, theta, m, ind, nu_code(theta->nu), nn, nn_cnt, y, precision, nll, grad, ws,
                        (cudaStream_t)stream);
  }
  return run_rows(pts, theta, m, nn, nn_cnt, y, plain_precision(precision), kModeNllGrad, nll, grad, nullptr,
                  nullptr, ws, (cudaStream_t)stream);
}

vst_status vecchia_nll_grad_ex(const vst_points* pts, const vst_theta* theta, int m, const vst_inducing* ind,
                               const int32_t* nn, const int32_t* nn_cnt, const double* y, int precision,
                               const vst_options* opts, double* nll, double* grad, void* ws, size_t ws_bytes,
                               void* stream) {
  if (ind && ind->k > 0) return fail(VST_EINVAL, "vecchia_nll_grad_ex: plain Vecchia only (no inducing points)");
  vst_status s = check_common(pts, theta, m, nn, nn_cnt, ws, ws_bytes, 0);
  if (s != VST_OK) return s;
  if (!valid_precision(precision)) return fail(VST_EINVAL, "bad precision %d", precision);
  if (!nll || !grad || (pts->n > 0 && !y)) return fail(VST_EINVAL, "y/nll/grad is NULL");
  CallOpts o;
  s = resolve_options(opts, pts->n, true, &o);
  if (s != VST_OK) return s;
  return run_rows(pts, theta, m, nn, nn_cnt, y, plain_precision(precision), kModeNllGrad, nll, grad, nullptr,
                  nullptr, ws, (cudaStream_t)stream, &o);
}

vst_status vst_workspace_status(const void* ws, void* stream, vst_ws_info* info) {
  if (!ws) return fail(VST_EINVAL, "workspace is NULL");
  WsHeader h;
  cudaError_t e = cudaMemcpyAsync(&h, ws, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "vst_workspace_status");
  vst_ws_info out;
  out.status = h.status;
  out.reserved = 0;
  out.bad_row = h.bad_row == ~0ull ? -1 : (int64_t)h.bad_row;
  out.n_fallback = (int64_t)h.n_fallback;
  out.n_tie = (int64_t)h.n_tie;
  if (info) *info = out;
  if (h.status != 0)
    fail((vst_status)h.status, "device reported status %d at row %lld", h.status, (long long)out.bad_row);
  return (vst_status)h.status;
}

}  // extern "C"
