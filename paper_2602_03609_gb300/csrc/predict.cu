// Vecchia prediction at new space-time points.
//
// The predictive distribution of Sect. 3.1 (mean Sigma_{n,np}^T Sigma~^{-1} Y,
// covariance Sigma_np + sigma^2 I - Sigma_{n,np}^T Sigma~^{-1} Sigma_{n,np})
// under the Vecchia approximation: every prediction point p conditions on its
// m training points of largest correlation (the d_c metric of Sect. 4.4.1,
// every training point a candidate), so that
//   mean_p = A_p y_N(p),   var_p = Sigma~_pp - A_p Sigma~_{N(p),p},
//   A_p = Sigma~_{p,N(p)} Sigma~_{N(p)}^{-1},
// the factor row of p placed after the training points (Sect. 4.1).  The
// latent variance leaves out the nugget.
//
// The prediction points are appended to the training points in the
// workspace; the bucketed exact search runs for the appended rows with the
// training rows as candidates, and the fused factor row kernel runs for the
// appended rows only.
#include <algorithm>

#include "kernels.h"
#include "profile.h"
#include "workspace.h"

namespace vst {

vst_status fail(vst_status s, const char* fmt, ...);
vst_status cuda_fail(cudaError_t e, const char* where);
vst_status check_theta(const vst_theta* th);
DevTheta dev_theta(const vst_theta* th);
int nu_code(double nu);
void launch_init_header(WsHeader* h, cudaStream_t st);
void launch_lag_table(const DevTheta& th, LagD* d, LagF* f, cudaStream_t st);
void apply_launch_shape(RowArgs& g, int batched, int precision, int nu, int pm);
vst_status plain_knn(const double* xy, const double* t, int64_t n, const vst_theta* theta, int m, int32_t* nn,
                     int32_t* nn_cnt, int64_t* tie_rows, int64_t tie_cap, char* base, const WsLayout& L,
                     WsHeader* hdr, int64_t n_cand, int64_t row0, cudaStream_t st);

namespace {

struct PredLayout {
  WsLayout L;  // the single-dataset workspace of the concatenated points
  size_t xy, t, nn, cnt, A, D, total;
};

PredLayout pred_layout(int64_t n_train, int64_t n_pred, int m) {
  const int64_t nt = n_train + n_pred;
  PredLayout P{};
  P.L = ws_layout(nt, m, 0);
  size_t off = P.L.total;
  auto take = [&off](size_t b) {
    const size_t at = off;
    off = align256(off + b);
    return at;
  };
  const size_t np = (size_t)std::max<int64_t>(n_pred, 1), mm = (size_t)std::max(m, 1);
  P.xy = take(16 * (size_t)std::max<int64_t>(nt, 1));
  P.t = take(8 * (size_t)std::max<int64_t>(nt, 1));
  P.nn = take(4 * np * mm);
  P.cnt = take(4 * np);
  P.A = take(8 * np * mm);
  P.D = take(8 * np);
  P.total = off;
  return P;
}

__global__ void predict_finish_kernel(int64_t np, int m, const int32_t* nn, const int32_t* cnt, const double* A,
                                      const double* D, const double* y, double nugget, int latent, double* mean,
                                      double* var) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
    const int c = cnt[p];
    double s = 0.0;
    for (int q = 0; q < c; ++q) s = fma(A[p * m + q], y[nn[p * m + q]], s);
    mean[p] = s;
    var[p] = latent ? D[p] - nugget : D[p];
  }
}

}  // namespace
}  // namespace vst

using namespace vst;

extern "C" size_t vst_workspace_size_predict(int64_t n_train, int64_t n_pred, int m) {
  return pred_layout(n_train, n_pred, m).total;
}

extern "C" vst_status vecchia_predict(const vst_points* train, const vst_theta* theta, int m, const double* y,
                                      const vst_points* pred, int precision, int latent, double* mean,
                                      double* var, int32_t* nn_out, void* ws, size_t ws_bytes, void* stream) {
  if (!train || !pred) return fail(VST_EINVAL, "train/pred is NULL");
  const int64_t n_train = train->n, n_pred = pred->n;
  if (n_train < 0 || n_pred < 0) return fail(VST_EINVAL, "negative point count");
  if (n_train + n_pred >= (int64_t(1) << 30)) return fail(VST_EINVAL, "n_train + n_pred out of range [0, 2^30)");
  if (m < 0 || m > VST_MAX_M) return fail(VST_EINVAL, "m=%d out of range [0, %d]", m, VST_MAX_M);
  vst_status s = check_theta(theta);
  if (s != VST_OK) return s;
  if (!valid_precision(precision)) return fail(VST_EINVAL, "bad precision %d", precision);
  precision = plain_precision(precision);
  if (n_train > 0 && (!train->xy || !train->t || !y)) return fail(VST_EINVAL, "training xy/t/y is NULL");
  if (n_pred > 0 && (!pred->xy || !pred->t || !mean || !var)) return fail(VST_EINVAL, "pred xy/t or mean/var is NULL");
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256) return fail(VST_EINVAL, "workspace NULL or not 256-byte aligned");
  const PredLayout P = pred_layout(n_train, n_pred, m);
  if (ws_bytes < P.total) return fail(VST_ENOMEM, "workspace has %zu bytes, %zu needed", ws_bytes, P.total);
  if (n_pred == 0) return VST_OK;

  cudaStream_t st = (cudaStream_t)stream;
  char* base = static_cast<char*>(ws);
  const WsLayout& L = P.L;
  WsHeader* hdr = reinterpret_cast<WsHeader*>(base + L.hdr);
  const int64_t nt = n_train + n_pred;
  double* xy = reinterpret_cast<double*>(base + P.xy);
  double* t = reinterpret_cast<double*>(base + P.t);
  int32_t* nn = reinterpret_cast<int32_t*>(base + P.nn);
  int32_t* cnt = reinterpret_cast<int32_t*>(base + P.cnt);
  double* A = reinterpret_cast<double*>(base + P.A);
  double* D = reinterpret_cast<double*>(base + P.D);
  cudaError_t e = cudaSuccess;
  if (n_train > 0) e = cudaMemcpyAsync(xy, train->xy, 16 * (size_t)n_train, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(xy + 2 * n_train, pred->xy, 16 * (size_t)n_pred, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && n_train > 0) e = cudaMemcpyAsync(t, train->t, 8 * (size_t)n_train, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(t + n_train, pred->t, 8 * (size_t)n_pred, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "copies");
  launch_init_header(hdr, st);

  // neighbours of the appended rows among the training rows
  const DevTheta th = dev_theta(theta);
  LagD* lagd = reinterpret_cast<LagD*>(base + L.lagd);
  LagF* lagf = reinterpret_cast<LagF*>(base + L.lagf);
  if (m == 0 || n_train == 0) {
    e = cudaMemsetAsync(cnt, 0, 4 * (size_t)n_pred, st);
    if (e == cudaSuccess && m > 0) e = cudaMemsetAsync(nn, 0xff, 4 * (size_t)n_pred * m, st);  // -1 padding
    if (e != cudaSuccess) return cuda_fail(e, "memset");
    launch_lag_table(th, lagd, lagf, st);
  } else {
    s = plain_knn(xy, t, nt, theta, m, nn, cnt, nullptr, 0, base, L, hdr, n_train, n_train, st);
    if (s != VST_OK) return s;
  }

  // factor rows of the appended points
  const bool mixed = precision == VST_MIXED;
  uint8_t* flag = reinterpret_cast<uint8_t*>(base + L.flag);
  PrepPt* prep = reinterpret_cast<PrepPt*>(base + L.prep);
  if (mixed) launch_prep_points(nt, xy, t, nullptr, prep, flag, st);
  RowArgs g{};
  g.xy = xy;
  g.t = t;
  g.nn = nn;
  g.nn_cnt = cnt;
  g.n = nt;
  g.m = m;
  g.th = th;
  g.lagd = lagd;
  g.lagf = lagf;
  g.A = A;
  g.D = D;
  g.flag = flag;
  g.hdr = hdr;
  g.tau = kDefaultTau;
  g.prep = prep;
  g.out0 = n_train;
  g.partial = reinterpret_cast<double*>(base + L.partial);
  const int nu = nu_code(theta->nu);
  apply_launch_shape(g, 0, precision, nu, m + 1);
  int64_t w = 0;
  {
    ProfileScope ps(kProfRows, st);
    e = launch_rows(mixed, nu, m + 1, kModeFactor, g, st, &w);
  }
  if (e != cudaSuccess) return cuda_fail(e, "prediction row kernel");
  if (mixed) {
    g.fallback_only = 1;
    e = launch_rows(false, nu, m + 1, kModeFactor, g, st, &w);
    if (e != cudaSuccess) return cuda_fail(e, "prediction fallback kernel");
  }
  predict_finish_kernel<<<(unsigned)std::min<int64_t>((n_pred + 255) / 256, 4096), 256, 0, st>>>(
      n_pred, m, nn, cnt, A, D, y, theta->nugget, latent ? 1 : 0, mean, var);
  e = cudaGetLastError();
  if (e == cudaSuccess && nn_out && m > 0)
    e = cudaMemcpyAsync(nn_out, nn, 4 * (size_t)n_pred * m, cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? VST_OK : cuda_fail(e, "prediction");
}
