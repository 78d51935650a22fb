// Plain CPU oracle for the Vecchia / VIF space-time likelihood path.
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the
// benchmark's CPU-baseline leg load this library.  It shares no code, header,
// table or constant with the CUDA path: every quantity below is written out
// from its definition in the paper (arXiv 2602.03609), in FP64, with loops in
// index order and no blocking, fusion or reordering.
//
// Notation (paper): sigma1^2 marginal variance, c spatial decay, a temporal
// scale, alpha temporal smoothness, nu Matern smoothness, gamma interaction,
// delta temporal decay, sigma^2 nugget.  m = Vecchia neighbours, k = inducing
// points.
//
// Parity status of each function is stated at its definition ("pinned by").
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

struct Theta {  // native parameters of Eq. (2) plus the nugget of Eq. (1)
  double sigma1sq, c, a, gamma, nugget, alpha, delta, nu;
};

// ---------------------------------------------------------------------------
// Matern part of Eq. (2):  M_nu(x) = 2^{1-nu}/Gamma(nu) * x^nu * K_nu(x),
// with M_nu(0) = 1.  For nu in {0.5, 1.5, 2.5} the half-integer Bessel
// function has the elementary form used on GPUs (Sect. 4.5); any other nu
// goes through std::cyl_bessel_k.
// Pinned by: scipy.special.kv at many (nu, x); the effective ranges printed
// in Table A3 (nu = 1) and the temperature parameter table (nu = 1.5).
double matern(double nu, double x) {
  if (x <= 0.0) return 1.0;
  if (nu == 0.5) return std::exp(-x);
  if (nu == 1.5) return (1.0 + x) * std::exp(-x);
  if (nu == 2.5) return (1.0 + x + x * x / 3.0) * std::exp(-x);
  return std::pow(2.0, 1.0 - nu) / std::tgamma(nu) * std::pow(x, nu) * std::cyl_bessel_k(nu, x);
}

// x * dM_nu/dx for the three closed forms (used only by the gradient).
double x_dmatern(double nu, double x) {
  if (x <= 0.0) return 0.0;
  if (nu == 0.5) return -x * std::exp(-x);
  if (nu == 1.5) return -x * x * std::exp(-x);
  if (nu == 2.5) return -(x * x / 3.0) * (1.0 + x) * std::exp(-x);
  return NAN;
}

// psi(u) = a |u|^{2 alpha} + 1, the temporal factor of Eq. (2).
double psi_of(const Theta& th, double u) { return th.a * std::pow(std::fabs(u), 2.0 * th.alpha) + 1.0; }

// Latent covariance c((s_i,t_i),(s_j,t_j)) of Eq. (2) with d = 2:
//   sigma1^2 * psi^{-(delta + gamma d/2)} * M_nu( c h / psi^{gamma/2} ).
// Pinned by: C(0,0) = sigma1^2, the gamma = 0 separable factorisation, the
// u = 0 pure-Matern reduction, and the printed effective ranges.
double cov_latent(const Theta& th, double h, double u) {
  const double psi = psi_of(th, u);
  const double x = th.c * h / std::pow(psi, th.gamma / 2.0);
  return th.sigma1sq / std::pow(psi, th.delta + th.gamma) * matern(th.nu, x);
}

// Partial derivatives of the latent covariance with respect to
// (sigma1^2, c, a, gamma), written out by hand from Eq. (2).
// Pinned by: central finite differences of cov_latent.
void cov_latent_grad(const Theta& th, double h, double u, double out[4]) {
  const double au = std::pow(std::fabs(u), 2.0 * th.alpha);  // d psi / d a
  const double psi = th.a * au + 1.0;
  const double p = th.delta + th.gamma;
  const double g = std::pow(psi, -th.gamma / 2.0);
  const double x = th.c * h * g;
  const double M = matern(th.nu, x);
  const double xM = x_dmatern(th.nu, x);  // x M'(x)
  const double pp = std::pow(psi, -p);
  const double lpsi = std::log(psi);
  out[0] = pp * M;                                            // d/d sigma1^2
  out[1] = th.sigma1sq * pp * (th.c > 0 ? xM / th.c : 0.0);    // d/d c   (dx/dc = x/c)
  // d/da: d psi^{-p}/da = -p psi^{-p-1} au ; dx/da = -(gamma/2) x au / psi
  out[2] = th.sigma1sq * pp * (-p * M / psi - 0.5 * th.gamma * xM / psi) * au;
  // d/dgamma: d psi^{-p}/dgamma = -ln(psi) psi^{-p} ; dx/dgamma = -(1/2) ln(psi) x
  out[3] = th.sigma1sq * pp * (-lpsi * M - 0.5 * lpsi * xM);
}

double dist2(const double* xy, int64_t i, int64_t j) {
  const double dx = xy[2 * i] - xy[2 * j];
  const double dy = xy[2 * i + 1] - xy[2 * j + 1];
  return std::sqrt(dx * dx + dy * dy);
}

// Entry (i, j) of the response covariance Sigma~ = Sigma + sigma^2 I (Sect. 3.1).
double cov_resp(const Theta& th, const double* xy, const double* t, int64_t i, int64_t j) {
  double v = cov_latent(th, dist2(xy, i, j), t[i] - t[j]);
  if (i == j) v += th.nugget;
  return v;
}

// d Sigma~_ij / d theta for theta = (sigma1^2, c, a, gamma, nugget).
void cov_resp_grad(const Theta& th, const double* xy, const double* t, int64_t i, int64_t j, double out[5]) {
  cov_latent_grad(th, dist2(xy, i, j), t[i] - t[j], out);
  out[4] = (i == j) ? 1.0 : 0.0;
}

// Plain Cholesky A = L L^T of a dense row-major p x p matrix (lower part used).
// Returns false if a pivot is not positive.
bool cholesky(std::vector<double>& A, int p) {
  for (int j = 0; j < p; ++j) {
    double s = A[j * p + j];
    for (int k = 0; k < j; ++k) s -= A[j * p + k] * A[j * p + k];
    if (!(s > 0.0)) return false;
    const double d = std::sqrt(s);
    A[j * p + j] = d;
    for (int i = j + 1; i < p; ++i) {
      double v = A[i * p + j];
      for (int k = 0; k < j; ++k) v -= A[i * p + k] * A[j * p + k];
      A[i * p + j] = v / d;
    }
  }
  return true;
}

// Solve (L L^T) x = b in place, L from cholesky().
void chol_solve(const std::vector<double>& L, int p, double* b) {
  for (int i = 0; i < p; ++i) {
    double v = b[i];
    for (int k = 0; k < i; ++k) v -= L[i * p + k] * b[k];
    b[i] = v / L[i * p + i];
  }
  for (int i = p - 1; i >= 0; --i) {
    double v = b[i];
    for (int k = i + 1; k < p; ++k) v -= L[k * p + i] * b[k];
    b[i] = v / L[i * p + i];
  }
}

template <class F>
void parallel_rows(int64_t n, int threads, F f) {
  if (threads <= 1 || n < 64) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::vector<std::thread> pool;
  for (int w = 0; w < threads; ++w)
    pool.emplace_back([=, &f]() {
      for (int64_t i = w; i < n; i += threads) f(i);
    });
  for (auto& th : pool) th.join();
}

Theta mk(const double* th8) {
  return Theta{th8[0], th8[1], th8[2], th8[3], th8[4], th8[5], th8[6], th8[7]};
}

// One Vecchia row (Sect. 4.1 applied to Sigma~): A_i = Sigma~_{i,N} Sigma~_N^{-1},
// D_i = Sigma~_ii - A_i Sigma~_{i,N}^T.  Returns false if Sigma~_N is not SPD.
struct RowFactor {
  std::vector<double> L;   // Cholesky factor of Sigma~_N
  std::vector<double> a;   // A_i
  std::vector<double> k;   // Sigma~_{N,i}
  double D;
};

bool factor_row(const Theta& th, const double* xy, const double* t, int64_t i, const int32_t* N, int cnt,
                RowFactor& rf) {
  rf.L.assign((size_t)cnt * cnt, 0.0);
  rf.k.assign(cnt, 0.0);
  for (int r = 0; r < cnt; ++r) {
    for (int s = 0; s < cnt; ++s) rf.L[r * cnt + s] = cov_resp(th, xy, t, N[r], N[s]);
    rf.k[r] = cov_resp(th, xy, t, N[r], i);
  }
  if (!cholesky(rf.L, cnt)) return false;
  rf.a = rf.k;
  chol_solve(rf.L, cnt, rf.a.data());
  double D = cov_resp(th, xy, t, i, i);
  for (int r = 0; r < cnt; ++r) D -= rf.a[r] * rf.k[r];
  rf.D = D;
  return true;
}

}  // namespace

extern "C" {

// ---------------------------------------------------------------------------
// Covariance primitives (exported for the pins).
double orc_matern(double nu, double x) { return matern(nu, x); }

double orc_cov(const double* th8, double h, double u) { return cov_latent(mk(th8), h, u); }

void orc_cov_grad(const double* th8, double h, double u, double* out4) { cov_latent_grad(mk(th8), h, u, out4); }

// Map effective-range parameters to the native parameters of Eq. (2).
// Effective ranges are the distance / lag at which the correlation decays to
// 0.05 (Sect. 6.1 parameter table, Table A3):
//   spatial:  M_nu(c * range_s) = 0.05          ->  c = x*_nu / range_s
//   temporal: psi(range_t)^{-(delta+gamma)} = 0.05 -> a = (0.05^{-1/(delta+gamma)} - 1) / range_t^{2 alpha}
// x*_nu is found by bisection on M_nu (decreasing on x > 0).
// Pinned by: the printed (c, range) and (a, alpha, gamma, delta, range) pairs.
int orc_theta_from_ranges(double sigma1sq, double range_s, double range_t, double gamma, double nugget,
                          double alpha, double delta, double nu, double* out8) {
  if (!(range_s > 0) || !(range_t > 0) || !(delta + gamma > 0)) return 1;
  double lo = 0.0, hi = 1.0;
  while (matern(nu, hi) > 0.05) hi *= 2.0;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (matern(nu, mid) > 0.05) lo = mid; else hi = mid;
  }
  const double xstar = 0.5 * (lo + hi);
  out8[0] = sigma1sq;
  out8[1] = xstar / range_s;
  out8[2] = (std::pow(0.05, -1.0 / (delta + gamma)) - 1.0) / std::pow(range_t, 2.0 * alpha);
  out8[3] = gamma;
  out8[4] = nugget;
  out8[5] = alpha;
  out8[6] = delta;
  out8[7] = nu;
  return 0;
}

// ---------------------------------------------------------------------------
// Correlation-based neighbour selection by brute force (Sect. 4.4.1).
// For each requested row i: among predecessors j < i, the min(i, m) points with
// the largest |rho_ij| = |Sigma_ij| / sqrt(Sigma_ii Sigma_jj) (latent Sigma, no
// nugget; equivalently the smallest d_c = sqrt(1 - |rho|)); ties broken by the
// smaller index; sorted by decreasing |rho|.  Also returns, per row, the
// m-th and (m+1)-th largest |rho| (NaN when absent) so that cut-off ties can
// be listed.
// Pinned by: a pure-Python sort over all predecessors on tiny inputs.
void orc_knn_rows(int64_t n, const double* xy, const double* t, const double* th8, int m,
                  int64_t n_rows, const int64_t* rows, int32_t* nn, int32_t* nn_cnt,
                  double* rho_m, double* rho_m1, int threads) {
  const Theta th = mk(th8);
  (void)n;
  parallel_rows(n_rows, threads, [&](int64_t r) {
    const int64_t i = rows[r];
    std::vector<std::pair<double, int64_t>> cand;
    cand.reserve((size_t)i);
    const double cii = cov_latent(th, 0.0, 0.0);
    for (int64_t j = 0; j < i; ++j) {
      const double cij = cov_latent(th, dist2(xy, i, j), t[i] - t[j]);
      const double cjj = cov_latent(th, 0.0, 0.0);
      cand.emplace_back(std::fabs(cij) / std::sqrt(cii * cjj), j);
    }
    const int64_t keep = std::min<int64_t>((int64_t)m + 1, i);
    auto better = [](const std::pair<double, int64_t>& A, const std::pair<double, int64_t>& B) {
      return A.first > B.first || (A.first == B.first && A.second < B.second);
    };
    std::partial_sort(cand.begin(), cand.begin() + keep, cand.end(), better);
    const int cnt = (int)std::min<int64_t>(m, i);
    for (int q = 0; q < m; ++q) nn[r * m + q] = q < cnt ? (int32_t)cand[q].second : -1;
    nn_cnt[r] = cnt;
    rho_m[r] = (cnt == m && cnt > 0) ? cand[m - 1].first : NAN;
    rho_m1[r] = (i > m) ? cand[m].first : NAN;
  });
}

// ---------------------------------------------------------------------------
// Correlation neighbours by the cover tree of Sect. 4.4.1 (Algorithm 1:
// construction in index order; Algorithm 2: the pruned search), under the
// metric d_c(x, y) = sqrt(1 - |rho(x, y)|), rho the latent correlation.
//
// Construction: the root is point 0 and covers every other point.  For level
// l = 1, 2, ... with radius R_l = 2^-l, each knot k of level l turns its
// covered set into knots of level l + 1: repeatedly the point of smallest
// index in the set becomes a new knot (a child of k), and the points of the
// set within d_c <= R_l of it become its covered set.  Every covered point
// has a larger index than its knot, so a knot's descendants all come after it.
//
// Search for row i (its m + 1 nearest predecessors, to list cut-off ties):
// Q = {root}; for j = 1 .. depth: C = Q and the children of Q's knots with
// index < i; D = the (m + 1)-th smallest d_c from i over C (1 if C is
// smaller); Q = {x in C : d_c(x, i) <= D + 2^-(j - 1)}; finally the nearest
// points of Q by brute force (the same order as orc_knn_rows: larger |rho|
// first, then the smaller index).
// Pinned by: orc_knn_rows (brute force) on small inputs, and the tree's
// invariants (every point a knot once, children after their knot, covered
// points within the level's radius).
namespace {

double corr_abs(const Theta& th, const double* xy, const double* t, int64_t i, int64_t j) {
  const double cij = cov_latent(th, dist2(xy, i, j), t[i] - t[j]);
  const double c0 = cov_latent(th, 0.0, 0.0);
  return std::fabs(cij) / c0;
}
double d_c(double rho_abs) { return std::sqrt(std::max(0.0, 1.0 - rho_abs)); }

struct CoverTree {
  std::vector<std::vector<int64_t>> children;  // per point: its child knots
  std::vector<int> level;                      // per point: the level it is a knot of
  int depth = 0;
};

CoverTree build_cover_tree(const Theta& th, const double* xy, const double* t, int64_t n) {
  CoverTree T;
  T.children.assign((size_t)n, {});
  T.level.assign((size_t)n, 0);
  if (n == 0) return T;
  std::vector<std::vector<int64_t>> cover((size_t)n);
  cover[0].reserve((size_t)n);
  for (int64_t p = 1; p < n; ++p) cover[0].push_back(p);
  T.level[0] = 1;
  std::vector<int64_t> current = {0};
  int l = 1;
  int64_t knots = 1;
  while (knots < n) {
    const double R = std::ldexp(1.0, -l);
    std::vector<int64_t> next;
    for (int64_t k : current) {
      std::vector<int64_t> S = std::move(cover[k]);
      cover[k].clear();
      size_t head = 0;  // S[head..] is the set still to cover, in increasing index order
      while (head < S.size()) {
        const int64_t v = S[head++];
        T.children[k].push_back(v);
        T.level[v] = l + 1;
        next.push_back(v);
        ++knots;
        std::vector<int64_t> rest, cv;
        for (size_t q = head; q < S.size(); ++q) {
          const int64_t p = S[q];
          if (d_c(corr_abs(th, xy, t, p, v)) <= R) cv.push_back(p);
          else rest.push_back(p);
        }
        cover[v] = std::move(cv);
        S = std::move(rest);
        head = 0;
      }
    }
    current = std::move(next);
    ++l;
  }
  T.depth = l;
  return T;
}

}  // namespace

void* orc_cover_tree_build(int64_t n, const double* xy, const double* t, const double* th8) {
  return new CoverTree(build_cover_tree(mk(th8), xy, t, n));
}
void orc_cover_tree_free(void* tree) { delete static_cast<CoverTree*>(tree); }
int orc_cover_tree_depth(const void* tree) { return static_cast<const CoverTree*>(tree)->depth; }
// per point: its level and parent (-1 for the root), for the invariant checks
void orc_cover_tree_structure(const void* tree, int64_t n, int32_t* level, int64_t* parent) {
  const CoverTree& T = *static_cast<const CoverTree*>(tree);
  for (int64_t p = 0; p < n; ++p) {
    level[p] = T.level[p];
    parent[p] = -1;
  }
  for (int64_t p = 0; p < n; ++p)
    for (int64_t c : T.children[p]) parent[c] = p;
}

void orc_knn_cover_tree(const void* tree, int64_t n, const double* xy, const double* t, const double* th8, int m,
                        int64_t n_rows, const int64_t* rows, int32_t* nn, int32_t* nn_cnt, double* rho_m,
                        double* rho_m1, int threads) {
  const CoverTree& T = *static_cast<const CoverTree*>(tree);
  const Theta th = mk(th8);
  (void)n;
  parallel_rows(n_rows, threads, [&](int64_t r) {
    const int64_t i = rows[r];
    const int K = m + 1;
    // Q: (d_c from i, point, whether its children are in C already); a
    // knot's children enter C once, in the step after the knot itself
    struct Ent {
      double d;
      int64_t p;
      bool expanded;
    };
    std::vector<Ent> Q;
    if (i > 0) Q.push_back({d_c(corr_abs(th, xy, t, 0, i)), 0, false});
    for (int j = 1; j <= T.depth && i > 0; ++j) {
      std::vector<Ent> C = Q;
      const size_t nq = C.size();
      for (size_t q = 0; q < nq; ++q) {
        if (C[q].expanded) continue;
        C[q].expanded = true;
        for (int64_t c : T.children[C[q].p])
          if (c < i) C.push_back({d_c(corr_abs(th, xy, t, c, i)), c, false});
      }
      double D = 1.0;
      if ((int64_t)C.size() >= K) {
        std::vector<double> ds;
        ds.reserve(C.size());
        for (const auto& c : C) ds.push_back(c.d);
        std::nth_element(ds.begin(), ds.begin() + (K - 1), ds.end());
        D = ds[K - 1];
      }
      const double lim = D + std::ldexp(1.0, -(j - 1));
      Q.clear();
      for (const auto& c : C)
        if (c.d <= lim) Q.push_back(c);
    }
    // brute force over Q, ranked by |rho| (then the smaller index)
    std::vector<std::pair<double, int64_t>> cand;
    cand.reserve(Q.size());
    for (const auto& q : Q) cand.emplace_back(corr_abs(th, xy, t, i, q.p), q.p);
    const int64_t keep = std::min<int64_t>((int64_t)K, (int64_t)cand.size());
    auto better = [](const std::pair<double, int64_t>& A, const std::pair<double, int64_t>& B) {
      return A.first > B.first || (A.first == B.first && A.second < B.second);
    };
    std::partial_sort(cand.begin(), cand.begin() + keep, cand.end(), better);
    const int cnt = (int)std::min<int64_t>(m, i);
    for (int q = 0; q < m; ++q) nn[r * m + q] = q < cnt ? (int32_t)cand[q].second : -1;
    nn_cnt[r] = cnt;
    rho_m[r] = (cnt == m && cnt > 0) ? cand[m - 1].first : NAN;
    rho_m1[r] = (i > m) ? cand[m].first : NAN;
  });
}

// ---------------------------------------------------------------------------
// Vecchia factor on the response covariance (Sect. 4.1 with Sigma~ of Sect. 3.1):
// A[i, q] = (A_i)_q for neighbour nn[i, q]  (B_{i, nn[i,q]} = -A[i, q]), D[i] = D_i.
// Returns the first row whose Sigma~_N is not SPD, or -1.
// Pinned by: exactness at m = n-1 against the dense likelihood (numpy), the
// bounds sigma^2 <= D_i <= sigma1^2 + sigma^2, and the whitening identity.
int64_t orc_factor(int64_t n, const double* xy, const double* t, const double* th8, int m,
                   const int32_t* nn, const int32_t* nn_cnt, double* A, double* D, int threads) {
  const Theta th = mk(th8);
  std::vector<int64_t> bad(threads > 1 ? threads : 1, -1);
  int64_t first_bad = -1;
  parallel_rows(n, threads, [&](int64_t i) {
    RowFactor rf;
    const int cnt = nn_cnt[i];
    if (!factor_row(th, xy, t, i, nn + i * m, cnt, rf)) {
      D[i] = NAN;
      return;
    }
    for (int q = 0; q < m; ++q) A[i * m + q] = q < cnt ? rf.a[q] : 0.0;
    D[i] = rf.D;
  });
  for (int64_t i = 0; i < n; ++i)
    if (!(D[i] > 0)) { first_bad = i; break; }
  return first_bad;
}

// The factor of selected rows only (for spot checks at large n): for each r,
// row rows[r] with neighbour list nn_rows[r][0..cnt[r]).  Same definition as
// orc_factor.  A_rows [R][m], D_rows [R] (NaN if the block is not SPD).
void orc_factor_rows(int64_t n, const double* xy, const double* t, const double* th8, int m, int64_t n_rows,
                     const int64_t* rows, const int32_t* nn_rows, const int32_t* cnt_rows, double* A_rows,
                     double* D_rows, int threads) {
  const Theta th = mk(th8);
  (void)n;
  parallel_rows(n_rows, threads, [&](int64_t r) {
    RowFactor rf;
    const int cnt = cnt_rows[r];
    if (!factor_row(th, xy, t, rows[r], nn_rows + r * m, cnt, rf)) {
      D_rows[r] = NAN;
      return;
    }
    for (int q = 0; q < m; ++q) A_rows[r * m + q] = q < cnt ? rf.a[q] : 0.0;
    D_rows[r] = rf.D;
  });
}

// Vecchia negative log-likelihood (Sect. 3.1 likelihood with Sigma~ replaced by
// its Vecchia approximation (B^T D^{-1} B)^{-1}):
//   n/2 log(2 pi) + 1/2 sum_i log D_i + 1/2 sum_i (y_i - A_i y_N(i))^2 / D_i.
// Optional per-row terms: term[i] = 1/2 log D_i + 1/2 r_i^2 / D_i.
// Sums are taken in index order.
double orc_nll(int64_t n, const double* xy, const double* t, const double* th8, int m,
               const int32_t* nn, const int32_t* nn_cnt, const double* y, double* term, int threads) {
  const Theta th = mk(th8);
  std::vector<double> row(n);
  parallel_rows(n, threads, [&](int64_t i) {
    RowFactor rf;
    const int cnt = nn_cnt[i];
    if (!factor_row(th, xy, t, i, nn + i * m, cnt, rf)) { row[i] = NAN; return; }
    double r = y[i];
    for (int q = 0; q < cnt; ++q) r -= rf.a[q] * y[nn[i * m + q]];
    row[i] = 0.5 * std::log(rf.D) + 0.5 * r * r / rf.D;
  });
  double s = 0.5 * (double)n * std::log(2.0 * M_PI);
  for (int64_t i = 0; i < n; ++i) {
    s += row[i];
    if (term) term[i] = row[i];
  }
  return s;
}

// Gradient of the Vecchia NLL w.r.t. (sigma1^2, c, a, gamma, nugget), by direct
// differentiation of each row's conditional (not an adjoint):
//   dD   = dSigma~_ii - 2 dk.A + A dK_N A^T
//   dA   = (dk^T - A dK_N) K_N^{-1}
//   dNLL_i = 1/2 dD/D - r (dA y_N)/D - 1/2 r^2 dD/D^2,   r = y_i - A y_N.
// grad[0..4]; optional per-row gradient terms gterm[i*5 + p].  Returns the NLL.
// Pinned by: the dense trace formula of Sect. 3.1 at m = n-1 (numpy), central
// finite differences of orc_nll, and the variance-scaling identity.
double orc_nll_grad(int64_t n, const double* xy, const double* t, const double* th8, int m,
                    const int32_t* nn, const int32_t* nn_cnt, const double* y, double* grad,
                    double* gterm, int threads) {
  const Theta th = mk(th8);
  std::vector<double> row(n), rowg((size_t)n * 5);
  parallel_rows(n, threads, [&](int64_t i) {
    RowFactor rf;
    const int cnt = nn_cnt[i];
    const int32_t* N = nn + i * m;
    if (!factor_row(th, xy, t, i, N, cnt, rf)) {
      row[i] = NAN;
      return;
    }
    double r = y[i];
    for (int q = 0; q < cnt; ++q) r -= rf.a[q] * y[N[q]];
    const double D = rf.D;
    row[i] = 0.5 * std::log(D) + 0.5 * r * r / D;
    // derivative blocks for the 5 parameters
    std::vector<double> dK((size_t)5 * cnt * cnt), dk((size_t)5 * cnt);
    double dKii[5], g5[5];
    for (int u = 0; u < cnt; ++u) {
      for (int v = 0; v < cnt; ++v) {
        cov_resp_grad(th, xy, t, N[u], N[v], g5);
        for (int p = 0; p < 5; ++p) dK[(size_t)p * cnt * cnt + u * cnt + v] = g5[p];
      }
      cov_resp_grad(th, xy, t, N[u], i, g5);
      for (int p = 0; p < 5; ++p) dk[(size_t)p * cnt + u] = g5[p];
    }
    cov_resp_grad(th, xy, t, i, i, dKii);
    std::vector<double> w(cnt);
    for (int p = 0; p < 5; ++p) {
      const double* dKp = &dK[(size_t)p * cnt * cnt];
      const double* dkp = &dk[(size_t)p * cnt];
      double dD = dKii[p];
      for (int u = 0; u < cnt; ++u) dD -= 2.0 * dkp[u] * rf.a[u];
      for (int u = 0; u < cnt; ++u)
        for (int v = 0; v < cnt; ++v) dD += rf.a[u] * dKp[u * cnt + v] * rf.a[v];
      // w = (dk - dK_N A^T), then dA^T = K_N^{-1} w
      for (int u = 0; u < cnt; ++u) {
        double s = dkp[u];
        for (int v = 0; v < cnt; ++v) s -= dKp[u * cnt + v] * rf.a[v];
        w[u] = s;
      }
      if (cnt > 0) chol_solve(rf.L, cnt, w.data());
      double dAy = 0.0;
      for (int u = 0; u < cnt; ++u) dAy += w[u] * y[N[u]];
      rowg[(size_t)i * 5 + p] = 0.5 * dD / D - r * dAy / D - 0.5 * r * r * dD / (D * D);
    }
  });
  double s = 0.5 * (double)n * std::log(2.0 * M_PI);
  for (int p = 0; p < 5; ++p) grad[p] = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    s += row[i];
    for (int p = 0; p < 5; ++p) grad[p] += rowg[(size_t)i * 5 + p];
  }
  if (gterm) std::memcpy(gterm, rowg.data(), sizeof(double) * 5 * (size_t)n);
  return s;
}

// NLL and gradient terms of selected rows only, each with its own neighbour
// list (same definitions as orc_nll_grad, without the n/2 log 2pi constant):
// returns sum_r NLL_rows[r], grad = sum_r dNLL_rows[r].  Used to time the
// oracle on a bounded sample of a large problem.
double orc_nll_grad_rows(int64_t n, const double* xy, const double* t, const double* th8, int m,
                         int64_t n_rows, const int64_t* rows, const int32_t* nn_rows, const int32_t* cnt_rows,
                         const double* y, double* grad, int threads) {
  const Theta th = mk(th8);
  (void)n;
  std::vector<double> out((size_t)n_rows * 6, 0.0);
  parallel_rows(n_rows, threads, [&](int64_t q) {
    const int64_t i = rows[q];
    const int cnt = cnt_rows[q];
    const int32_t* N = nn_rows + q * m;
    RowFactor rf;
    if (!factor_row(th, xy, t, i, N, cnt, rf)) { out[q * 6] = NAN; return; }
    double r = y[i];
    for (int u = 0; u < cnt; ++u) r -= rf.a[u] * y[N[u]];
    const double D = rf.D;
    out[q * 6] = 0.5 * std::log(D) + 0.5 * r * r / D;
    std::vector<double> dK((size_t)cnt * cnt), dk(cnt), w(cnt);
    double g5[5];
    for (int p = 0; p < 5; ++p) {
      for (int u = 0; u < cnt; ++u) {
        for (int v = 0; v < cnt; ++v) { cov_resp_grad(th, xy, t, N[u], N[v], g5); dK[u * cnt + v] = g5[p]; }
        cov_resp_grad(th, xy, t, N[u], i, g5);
        dk[u] = g5[p];
      }
      cov_resp_grad(th, xy, t, i, i, g5);
      double dD = g5[p];
      for (int u = 0; u < cnt; ++u) dD -= 2.0 * dk[u] * rf.a[u];
      for (int u = 0; u < cnt; ++u)
        for (int v = 0; v < cnt; ++v) dD += rf.a[u] * dK[u * cnt + v] * rf.a[v];
      for (int u = 0; u < cnt; ++u) {
        double s = dk[u];
        for (int v = 0; v < cnt; ++v) s -= dK[u * cnt + v] * rf.a[v];
        w[u] = s;
      }
      if (cnt > 0) chol_solve(rf.L, cnt, w.data());
      double dAy = 0.0;
      for (int u = 0; u < cnt; ++u) dAy += w[u] * y[N[u]];
      out[q * 6 + 1 + p] = 0.5 * dD / D - r * dAy / D - 0.5 * r * r * dD / (D * D);
    }
  });
  double s = 0.0;
  for (int p = 0; p < 5; ++p) grad[p] = 0.0;
  for (int64_t q = 0; q < n_rows; ++q) {
    s += out[q * 6];
    for (int p = 0; p < 5; ++p) grad[p] += out[q * 6 + 1 + p];
  }
  return s;
}

// Vecchia sampling: y_i = A_i y_N(i) + sqrt(D_i) z_i for i = 0..n-1 in order,
// i.e. y = B^{-1} D^{1/2} z (Sect. 4.1, Sigma~s = B^{-1} D B^{-T}).
void orc_vecchia_sample(int64_t n, int m, const int32_t* nn, const int32_t* nn_cnt, const double* A,
                        const double* D, const double* z, double* y) {
  for (int64_t i = 0; i < n; ++i) {
    double v = std::sqrt(D[i]) * z[i];
    for (int q = 0; q < nn_cnt[i]; ++q) v += A[i * m + q] * y[nn[i * m + q]];
    y[i] = v;
  }
}

// ---------------------------------------------------------------------------
// Exact Gaussian likelihood (Sect. 3.1) with the dense n x n Sigma~:
//   NLL = n/2 log 2pi + 1/2 log det Sigma~ + 1/2 y^T Sigma~^{-1} y
//   dNLL/dtheta = 1/2 tr(Sigma~^{-1} dSigma~) - 1/2 y^T Sigma~^{-1} dSigma~ Sigma~^{-1} y.
// grad may be NULL.  Returns NAN if Sigma~ is not SPD.  For n up to a few
// thousand.  Pinned by: numpy slogdet / solve on the same matrix.
double orc_dense_nll(int64_t n, const double* xy, const double* t, const double* th8, const double* y,
                     double* grad) {
  const Theta th = mk(th8);
  std::vector<double> S((size_t)n * n);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) S[i * n + j] = cov_resp(th, xy, t, i, j);
  if (!cholesky(S, (int)n)) return NAN;
  double logdet = 0.0;
  for (int64_t i = 0; i < n; ++i) logdet += 2.0 * std::log(S[i * n + i]);
  std::vector<double> alpha(y, y + n);
  chol_solve(S, (int)n, alpha.data());
  double quad = 0.0;
  for (int64_t i = 0; i < n; ++i) quad += y[i] * alpha[i];
  const double nll = 0.5 * (double)n * std::log(2.0 * M_PI) + 0.5 * logdet + 0.5 * quad;
  if (grad) {
    // explicit inverse, column by column
    std::vector<double> inv((size_t)n * n), e(n);
    for (int64_t j = 0; j < n; ++j) {
      std::fill(e.begin(), e.end(), 0.0);
      e[j] = 1.0;
      chol_solve(S, (int)n, e.data());
      for (int64_t i = 0; i < n; ++i) inv[i * n + j] = e[i];
    }
    for (int p = 0; p < 5; ++p) grad[p] = 0.0;
    double g5[5];
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) {
        cov_resp_grad(th, xy, t, i, j, g5);
        for (int p = 0; p < 5; ++p) grad[p] += 0.5 * inv[i * n + j] * g5[p] - 0.5 * alpha[i] * g5[p] * alpha[j];
      }
  }
  return nll;
}

// y = L z with Sigma~ = L L^T (exact simulation of the model of Eq. (1)).
int orc_dense_sample(int64_t n, const double* xy, const double* t, const double* th8, const double* z,
                     double* y) {
  const Theta th = mk(th8);
  std::vector<double> S((size_t)n * n);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) S[i * n + j] = cov_resp(th, xy, t, i, j);
  if (!cholesky(S, (int)n)) return 1;
  for (int64_t i = 0; i < n; ++i) {
    double v = 0.0;
    for (int64_t k = 0; k <= i; ++k) v += S[i * n + k] * z[k];
    y[i] = v;
  }
  return 0;
}

// Dense covariance matrices for the pins (row-major).
void orc_cov_matrix(int64_t n1, const double* xy1, const double* t1, int64_t n2, const double* xy2,
                    const double* t2, const double* th8, double* out) {
  const Theta th = mk(th8);
  for (int64_t i = 0; i < n1; ++i)
    for (int64_t j = 0; j < n2; ++j) {
      const double dx = xy1[2 * i] - xy2[2 * j], dy = xy1[2 * i + 1] - xy2[2 * j + 1];
      out[i * n2 + j] = cov_latent(th, std::sqrt(dx * dx + dy * dy), t1[i] - t2[j]);
    }
}

int orc_version() { return 1; }

}  // extern "C"
