// Space-time separated kMeans++ inducing points (Algorithm 3): kMeans++ on
// the unique time points (m_t centres) and, separately, on the unique
// locations (m_s centres); the inducing points are the Cartesian product.
//   m_s = round(sqrt(m n / |T|^2)),  m_t = round(sqrt(m |T|^2 / n))
// (round = floor(x + 1/2), clamped to [1, |S|] and [1, |T|]).
//
// kMeans++ (Arthur and Vassilvitskii, 2007): the first centre uniformly at
// random, every further centre with probability proportional to the squared
// distance D^2 to the nearest chosen centre; then `lloyd_iters` Lloyd steps
// (assignment to the nearest centre, ties to the smaller centre index; new
// centre = mean of its points, an empty cluster keeps its centre).
//
// Every discrete choice is made from exact integers so that the result does
// not depend on the order of parallel sums:
//   * draws: SplitMix64 (Steele, Lea and Flood, 2014) as a counter-based
//     generator, u_j = (mix(x0 + j gamma) >> 11) 2^-53, with x0 = seed for the
//     times and seed ^ 0xD1B54A32D192ED03 for the locations;
//   * D^2 sampling: weights w_i = floor(D2_i * 2^32 / max D2), summed in
//     64-bit integers; the chosen point is the first whose prefix sum exceeds
//     min(floor(u_j * sum), sum - 1);
//   * Lloyd means: coordinates quantised to q = rint((x - lo) 2^32 / span),
//     summed in 64-bit integers, centre = lo + (sum / count) / (2^32 / span);
//   * squared distances are dx*dx + dy*dy with no fused multiply-add.
// Unique points are sorted (times ascending, locations lexicographically by
// (x, y)); centre j of the output product is (location j / m_t, time j % m_t).
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <vector>

#include "kernels.h"

namespace vst {

vst_status fail(vst_status s, const char* fmt, ...);
vst_status cuda_fail(cudaError_t e, const char* where);

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kLocStream = 0xD1B54A32D192ED03ull;
constexpr double kFix = 4294967296.0;  // 2^32: sums of up to 2^30 values stay below 2^62

__host__ __device__ inline uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ inline double sm_uniform(uint64_t x0, int64_t j) {
  return (double)(sm_mix(x0 + (uint64_t)(j + 1) * kGamma) >> 11) * 0x1.0p-53;
}

struct KmLayout {
  size_t table, ux, uy, cnt, d2, cx, cy, sumx, sumy, ccount, tmp, total;
  int64_t tsize, sortn;
};

int64_t pow2_at_least(int64_t v) {
  int64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

KmLayout km_layout(int64_t n) {
  KmLayout L{};
  size_t off = 0;
  auto take = [&off](size_t b) {
    const size_t at = off;
    off = (off + b + 255) & ~size_t(255);
    return at;
  };
  const int64_t nn = std::max<int64_t>(n, 1);
  L.tsize = pow2_at_least(2 * nn);
  L.sortn = pow2_at_least(nn);
  L.table = take(sizeof(int32_t) * (size_t)L.tsize);
  L.ux = take(sizeof(double) * (size_t)L.sortn);  // unique values (sorted in place, +inf padded)
  L.uy = take(sizeof(double) * (size_t)L.sortn);
  L.cnt = take(sizeof(unsigned long long) * 4);
  L.d2 = take(sizeof(double) * (size_t)nn);
  L.cx = take(sizeof(double) * (size_t)nn);  // centres (at most the unique count)
  L.cy = take(sizeof(double) * (size_t)nn);
  L.sumx = take(sizeof(unsigned long long) * (size_t)nn);
  L.sumy = take(sizeof(unsigned long long) * (size_t)nn);
  L.ccount = take(sizeof(unsigned long long) * (size_t)nn);
  L.tmp = take(sizeof(double) * 8);
  L.total = off;
  return L;
}

__device__ inline uint64_t key_hash(double x, double y) {
  return sm_mix(__double_as_longlong(x) * 0x9E3779B97F4A7C15ull ^ (uint64_t)__double_as_longlong(y));
}

// Insert point i (x[i*stride], y[i*stride] or 0 when dim == 1) into the open
// addressing table; the first occurrence of each distinct value claims a
// slot, and a unique-count increments.
__global__ void unique_insert_kernel(const double* a, int stride, int dim, int64_t n, int32_t* table,
                                     int64_t tsize, double* ux, double* uy, unsigned long long* count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = a[i * stride], y = dim == 2 ? a[i * stride + 1] : 0.0;
    int64_t slot = (int64_t)(key_hash(x, y) & (uint64_t)(tsize - 1));
    for (int64_t probe = 0; probe < tsize; ++probe) {
      const int32_t cur = atomicCAS(&table[slot], -1, (int32_t)i);
      int32_t owner = cur == -1 ? (int32_t)i : cur;
      if (cur == -1) {
        const unsigned long long u = atomicAdd(count, 1ull);
        ux[u] = x;
        uy[u] = y;
        break;
      }
      const double ox = a[(int64_t)owner * stride], oy = dim == 2 ? a[(int64_t)owner * stride + 1] : 0.0;
      if (ox == x && oy == y) break;  // already present
      slot = (slot + 1) & (tsize - 1);
    }
  }
}

__global__ void pad_kernel(double* ux, double* uy, int64_t from, int64_t to) {
  for (int64_t i = from + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < to; i += (int64_t)gridDim.x * blockDim.x) {
    ux[i] = DBL_MAX;
    uy[i] = DBL_MAX;
  }
}

// one bitonic merge step over the padded array, lexicographic by (x, y)
__global__ void bitonic_kernel(double* ux, double* uy, int64_t n, int64_t j, int64_t k) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = i ^ j;
    if (l <= i) continue;
    const bool up = (i & k) == 0;
    const double xi = ux[i], yi = uy[i], xl = ux[l], yl = uy[l];
    const bool gt = xi > xl || (xi == xl && yi > yl);
    if (gt == up) {
      ux[i] = xl; uy[i] = yl;
      ux[l] = xi; uy[l] = yi;
    }
  }
}

__device__ inline double d2_nofma(double ax, double ay, double bx, double by) {
  const double dx = __dsub_rn(ax, bx), dy = __dsub_rn(ay, by);
  return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

// kMeans++ seeding of k centres among the N unique points, one block
template <int T>
__global__ void __launch_bounds__(T) seed_kernel(const double* px, const double* py, int64_t N, int k, uint64_t x0,
                                                 double* d2, double* cx, double* cy) {
  __shared__ double smax[T];
  __shared__ unsigned long long ssum[T];
  __shared__ int64_t schosen;
  const int tid = threadIdx.x;
  // first centre uniformly
  int64_t c0 = (int64_t)(sm_uniform(x0, 0) * (double)N);
  if (c0 >= N) c0 = N - 1;
  for (int64_t i = tid; i < N; i += T) d2[i] = d2_nofma(px[i], py[i], px[c0], py[c0]);
  if (tid == 0) { cx[0] = px[c0]; cy[0] = py[c0]; }
  __syncthreads();
  for (int j = 1; j < k; ++j) {
    // scale of the integer weights
    double mx = 0.0;
    for (int64_t i = tid; i < N; i += T) mx = fmax(mx, d2[i]);
    smax[tid] = mx;
    __syncthreads();
    for (int w = T / 2; w > 0; w >>= 1) {
      if (tid < w) smax[tid] = fmax(smax[tid], smax[tid + w]);
      __syncthreads();
    }
    const double dmax = smax[0];
    __syncthreads();
    if (!(dmax > 0.0)) break;  // every point is a centre
    const double s = __ddiv_rn(kFix, dmax);
    unsigned long long tot = 0;
    for (int64_t i = tid; i < N; i += T) tot += (unsigned long long)floor(__dmul_rn(d2[i], s));
    ssum[tid] = tot;
    __syncthreads();
    for (int w = T / 2; w > 0; w >>= 1) {
      if (tid < w) ssum[tid] += ssum[tid + w];
      __syncthreads();
    }
    const unsigned long long total = ssum[0];
    unsigned long long target = (unsigned long long)floor(sm_uniform(x0, j) * (double)total);
    if (target >= total) target = total - 1;  // u * total may round up to total
    __syncthreads();
    // first i with prefix(i) > target: chunks of T, inclusive block scan
    if (tid == 0) schosen = -1;
    unsigned long long before = 0;
    for (int64_t c = 0; c < N; c += T) {
      const int64_t i = c + tid;
      const unsigned long long wv = i < N ? (unsigned long long)floor(__dmul_rn(d2[i], s)) : 0ull;
      ssum[tid] = wv;
      __syncthreads();
      for (int o = 1; o < T; o <<= 1) {
        const unsigned long long add = tid >= o ? ssum[tid - o] : 0ull;
        __syncthreads();
        ssum[tid] += add;
        __syncthreads();
      }
      const unsigned long long incl = before + ssum[tid];
      const unsigned long long excl = incl - wv;
      if (i < N && wv > 0 && excl <= target && target < incl) schosen = i;
      before += ssum[T - 1];
      __syncthreads();
      if (schosen >= 0) break;
    }
    int64_t ch = schosen;
    if (ch < 0) ch = N - 1;  // unreachable when total > 0
    if (tid == 0) { cx[j] = px[ch]; cy[j] = py[ch]; }
    for (int64_t i = tid; i < N; i += T) d2[i] = fmin(d2[i], d2_nofma(px[i], py[i], px[ch], py[ch]));
    __syncthreads();
  }
}

struct Quant {
  double lox, loy, sx, sy;  // q = rint((x - lo) * s)
};

__global__ void lloyd_assign_kernel(const double* px, const double* py, int64_t N, const double* cx,
                                    const double* cy, int k, Quant q, unsigned long long* sumx,
                                    unsigned long long* sumy, unsigned long long* cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = px[i], y = py[i];
    int best = 0;
    double bd = d2_nofma(x, y, cx[0], cy[0]);
    for (int j = 1; j < k; ++j) {
      const double d = d2_nofma(x, y, cx[j], cy[j]);
      if (d < bd) { bd = d; best = j; }
    }
    atomicAdd(&sumx[best], (unsigned long long)rint(__dmul_rn(__dsub_rn(x, q.lox), q.sx)));
    atomicAdd(&sumy[best], (unsigned long long)rint(__dmul_rn(__dsub_rn(y, q.loy), q.sy)));
    atomicAdd(&cnt[best], 1ull);
  }
}

__global__ void lloyd_update_kernel(int k, Quant q, const unsigned long long* sumx, const unsigned long long* sumy,
                                    const unsigned long long* cnt, double* cx, double* cy) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k || cnt[j] == 0) return;
  const double c = (double)cnt[j];
  cx[j] = __dadd_rn(q.lox, __ddiv_rn(__ddiv_rn((double)sumx[j], c), q.sx));
  cy[j] = __dadd_rn(q.loy, __ddiv_rn(__ddiv_rn((double)sumy[j], c), q.sy));
}

__global__ void product_kernel(const double* sx, const double* sy, int ms, const double* tc, int mt, double* xyk,
                               double* tk) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= (int64_t)ms * mt) return;
  const int a = (int)(id / mt), b = (int)(id % mt);
  xyk[2 * id] = sx[a];
  xyk[2 * id + 1] = sy[a];
  tk[id] = tc[b];
}

// unique sorted values of a (dim 1: times, dim 2: locations) into ux, uy;
// returns the unique count (one synchronisation)
vst_status unique_sorted(const double* a, int stride, int dim, int64_t n, const KmLayout& L, char* base,
                         int64_t* nu, cudaStream_t st) {
  int32_t* table = reinterpret_cast<int32_t*>(base + L.table);
  double* ux = reinterpret_cast<double*>(base + L.ux);
  double* uy = reinterpret_cast<double*>(base + L.uy);
  unsigned long long* count = reinterpret_cast<unsigned long long*>(base + L.cnt);
  cudaError_t e = cudaMemsetAsync(table, 0xff, sizeof(int32_t) * (size_t)L.tsize, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
  unique_insert_kernel<<<grid, 256, 0, st>>>(a, stride, dim, n, table, L.tsize, ux, uy, count);
  unsigned long long h = 0;
  e = cudaMemcpyAsync(&h, count, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "unique count");
  const int64_t u = (int64_t)h, p2 = pow2_at_least(std::max<int64_t>(u, 1));
  if (p2 > L.sortn) return fail(VST_EINTERNAL, "unique count exceeds the sort buffer");
  if (p2 > u) pad_kernel<<<(int)std::min<int64_t>((p2 - u + 255) / 256, 4096), 256, 0, st>>>(ux, uy, u, p2);
  const int sg = (int)std::min<int64_t>((p2 + 255) / 256, 4096);
  for (int64_t k = 2; k <= p2; k <<= 1)
    for (int64_t j = k >> 1; j > 0; j >>= 1) bitonic_kernel<<<sg, 256, 0, st>>>(ux, uy, p2, j, k);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "unique sort");
  *nu = u;
  return VST_OK;
}

// kMeans++ with Lloyd steps on the N points in (ux, uy); centres to (cx, cy)
vst_status kmeanspp(const double* ux, const double* uy, int64_t N, int k, uint64_t x0, int iters, const KmLayout& L,
                    char* base, double* cx, double* cy, cudaStream_t st) {
  double* d2 = reinterpret_cast<double*>(base + L.d2);
  seed_kernel<1024><<<1, 1024, 0, st>>>(ux, uy, N, k, x0, d2, cx, cy);
  if (iters > 0) {
    // quantisation box from the sorted points (x sorted; y needs a pass)
    double hb[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(&hb[0], ux, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hb[1], ux + (N - 1), sizeof(double), cudaMemcpyDeviceToHost, st);
    std::vector<double> hy((size_t)N);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hy.data(), uy, sizeof(double) * (size_t)N, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "lloyd box");
    const double ylo = *std::min_element(hy.begin(), hy.end()), yhi = *std::max_element(hy.begin(), hy.end());
    Quant q;
    q.lox = hb[0];
    q.loy = ylo;
    q.sx = hb[1] > hb[0] ? kFix / (hb[1] - hb[0]) : 1.0;
    q.sy = yhi > ylo ? kFix / (yhi - ylo) : 1.0;
    unsigned long long* sx = reinterpret_cast<unsigned long long*>(base + L.sumx);
    unsigned long long* sy = reinterpret_cast<unsigned long long*>(base + L.sumy);
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(base + L.ccount);
    const int grid = (int)std::min<int64_t>((N + 255) / 256, 4096);
    for (int it = 0; it < iters; ++it) {
      e = cudaMemsetAsync(sx, 0, sizeof(unsigned long long) * k, st);
      if (e == cudaSuccess) e = cudaMemsetAsync(sy, 0, sizeof(unsigned long long) * k, st);
      if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * k, st);
      if (e != cudaSuccess) return cuda_fail(e, "memset");
      lloyd_assign_kernel<<<grid, 256, 0, st>>>(ux, uy, N, cx, cy, k, q, sx, sy, cnt);
      lloyd_update_kernel<<<(k + 255) / 256, 256, 0, st>>>(k, q, sx, sy, cnt, cx, cy);
    }
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VST_OK : cuda_fail(e, "kmeans++");
}

}  // namespace
}  // namespace vst

using namespace vst;

extern "C" size_t vst_workspace_size_kmeans(int64_t n) { return km_layout(n).total; }

extern "C" vst_status vst_sts_kmeanspp(const vst_points* pts, int64_t m, uint64_t seed, int lloyd_iters,
                                       double* xyk, double* tk, int64_t k_cap, int64_t* k_out, int64_t* ms_out,
                                       int64_t* mt_out, void* ws, size_t ws_bytes, void* stream) {
  if (!pts) return fail(VST_EINVAL, "pts is NULL");
  const int64_t n = pts->n;
  if (n <= 0 || n >= (int64_t(1) << 30)) return fail(VST_EINVAL, "n=%lld out of range [1, 2^30)", (long long)n);
  if (m < 1) return fail(VST_EINVAL, "m=%lld < 1", (long long)m);
  if (lloyd_iters < 0) return fail(VST_EINVAL, "lloyd_iters < 0");
  if (!pts->xy || !pts->t || !xyk || !tk || !k_out) return fail(VST_EINVAL, "NULL argument");
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256) return fail(VST_EINVAL, "workspace NULL or not 256-byte aligned");
  const KmLayout L = km_layout(n);
  if (ws_bytes < L.total) return fail(VST_ENOMEM, "workspace has %zu bytes, %zu needed", ws_bytes, L.total);
  cudaStream_t st = (cudaStream_t)stream;
  char* base = static_cast<char*>(ws);
  double* ux = reinterpret_cast<double*>(base + L.ux);
  double* uy = reinterpret_cast<double*>(base + L.uy);
  double* cx = reinterpret_cast<double*>(base + L.cx);
  double* cy = reinterpret_cast<double*>(base + L.cy);

  // unique times (sorted), their centres into tk's tail temporarily (tc)
  int64_t nt = 0, ns = 0;
  vst_status s = unique_sorted(pts->t, 1, 1, n, L, base, &nt, st);
  if (s != VST_OK) return s;
  const double fn = (double)n, ft = (double)nt;
  int64_t ms = (int64_t)std::floor(std::sqrt((double)m * fn / (ft * ft)) + 0.5);
  int64_t mt = (int64_t)std::floor(std::sqrt((double)m * ft * ft / fn) + 0.5);
  mt = std::min<int64_t>(std::max<int64_t>(mt, 1), nt);
  // times: kMeans++ on (t, 0); keep the centres on the host meanwhile
  s = kmeanspp(ux, uy, nt, (int)mt, seed, lloyd_iters, L, base, cx, cy, st);
  if (s != VST_OK) return s;
  std::vector<double> tcent((size_t)mt);
  cudaError_t e = cudaMemcpyAsync(tcent.data(), cx, sizeof(double) * (size_t)mt, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "time centres");
  // locations
  s = unique_sorted(pts->xy, 2, 2, n, L, base, &ns, st);
  if (s != VST_OK) return s;
  ms = std::min<int64_t>(std::max<int64_t>(ms, 1), ns);
  if (ms * mt > k_cap) return fail(VST_EINVAL, "m_s * m_t = %lld exceeds k_cap = %lld", (long long)(ms * mt),
                                   (long long)k_cap);
  s = kmeanspp(ux, uy, ns, (int)ms, seed ^ kLocStream, lloyd_iters, L, base, cx, cy, st);
  if (s != VST_OK) return s;
  double* tdev = reinterpret_cast<double*>(base + L.d2);  // reuse: the time centres
  e = cudaMemcpyAsync(tdev, tcent.data(), sizeof(double) * (size_t)mt, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "time centres");
  const int64_t k = ms * mt;
  product_kernel<<<(unsigned)((k + 255) / 256), 256, 0, st>>>(cx, cy, (int)ms, tdev, (int)mt, xyk, tk);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // tcent must outlive the copy
  if (e != cudaSuccess) return cuda_fail(e, "product");
  *k_out = k;
  if (ms_out) *ms_out = ms;
  if (mt_out) *mt_out = mt;
  return VST_OK;
}
