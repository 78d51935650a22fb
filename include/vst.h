/*
 * vst.h -- C ABI of the GB300 (sm_103a) Vecchia / VIF space-time likelihood
 * library (libvst.so).
 *
 * Method: Gyger, Furrer & Sigrist, "Scalable non-separable spatio-temporal
 * Gaussian process models for large-scale short-term weather prediction"
 * (arXiv 2602.03609).  The library evaluates, on one GPU, the hot path of
 * fitting the Gaussian model Y = b + eps of Eq. (1) with the non-separable
 * Gneiting covariance of Eq. (2) under a Vecchia approximation (Sect. 4.1):
 *
 *   1. correlation-based neighbour selection (Sect. 4.4.1),
 *   2. the per-row Vecchia factor A_i, D_i (Sect. 4.1),
 *   3. the negative log-likelihood (Sect. 3.1) and its gradient with respect
 *      to the covariance parameters.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All array arguments are DEVICE pointers (cudaMalloc'd memory, or the
 *    storage of a CUDA tensor) on the current device, unless stated otherwise.
 *    The caller owns every buffer; the library allocates nothing and keeps no
 *    state between calls.  Scratch memory is the caller's `workspace`
 *    (`ws_bytes` >= vst_workspace_size(...), 256-byte aligned).  A workspace
 *    may not be shared by calls that can overlap on the GPU.
 *  - Points are already in Vecchia order: row i may condition only on rows
 *    j < i.  Layouts: xy[n][2] (x, y interleaved, FP64), t[n] (FP64, time in
 *    the unit of the temporal range), y[n] (FP64 responses with the mean
 *    removed), nn[n][m] (int32 neighbour indices, -1 padded), nn_cnt[n]
 *    (int32, number of valid entries of row i of nn), A[n][m] (FP64, A[i][q]
 *    multiplies neighbour nn[i][q]; B_{i, nn[i][q]} = -A[i][q]), D[n] (FP64).
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) unless stated otherwise.  The returned status covers argument
 *    validation and launch errors.  Errors found on the device (a local
 *    covariance block that is not positive definite, a neighbour index that is
 *    not a predecessor, a bounded wait that ran out) are recorded in the
 *    workspace header and returned by vst_workspace_status(), which
 *    synchronises the stream.
 *  - Sizes: 0 <= n < 2^31, 0 <= m <= VST_MAX_M.  n == 0 is valid (the NLL is 0).
 *  - Covariance parameters (vst_theta) must satisfy sigma1sq > 0, c > 0,
 *    a > 0, 0 <= gamma <= 1, nugget >= 0, 0 < alpha <= 1, delta >= 0,
 *    delta + gamma > 0 and nu in {0.5, 1.5, 2.5} (the closed-form Matern
 *    orders, Sect. 4.5); otherwise VST_EINVAL.
 */
#ifndef VST_H
#define VST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VST_MAX_M 31

typedef enum {
  VST_OK = 0,
  VST_EINVAL = 1,     /* bad argument (message in vst_last_error) */
  VST_ENOMEM = 2,     /* workspace too small */
  VST_ENOTSPD = 3,    /* a local covariance block is not positive definite */
  VST_ETIMEOUT = 4,   /* a bounded device-side wait ran out */
  VST_ECUDA = 5,      /* a CUDA runtime call failed */
  VST_EINTERNAL = 6   /* an internal consistency check failed on the device */
} vst_status;

typedef enum {
  VST_FP64 = 0,   /* every step in FP64 */
  VST_MIXED = 1,  /* FP32 covariance + Cholesky, one refinement step of the
                     solve with double-float residuals, FP64 log-determinant
                     and accumulation; rows whose local condition estimate
                     exceeds the threshold, or whose FP32 Cholesky fails, are
                     redone in FP64.  VIF: U = Sigma_nk L^{-T} on the tensor
                     cores, each FP32 operand split into three BF16 parts,
                     six products accumulated in FP32 (about FP32 accuracy);
                     the per-row residual Gram (blocks of 32 positions) and
                     the contractions over the points (W^T W, W^T e, e^T e,
                     the gradient's H^T U) on the tensor cores with three
                     fixed-point BF16 parts, leading sums exact per block */
  VST_MIXED_BF16X3 = 2  /* as VST_MIXED, but the VIF low-rank product (and the
                           gradient's n x k products) split each operand into
                           two BF16 parts and keep three products (16
                           significand bits, relative error ~1e-5 per entry
                           of U); the per-row Gram and the contractions over
                           the points keep three fixed-point parts.  Plain
                           Vecchia: = VST_MIXED.  Single-dataset entry points
                           only. */
} vst_precision;

/* Native parameters of Eq. (2) plus the nugget of Eq. (1):
 *   c((s,t),(s',t')) = sigma1sq * psi^{-(delta+gamma)} * M_nu(c h psi^{-gamma/2}),
 *   psi = a |t-t'|^{2 alpha} + 1,  h = ||s - s'||,
 *   M_nu(x) = 2^{1-nu}/Gamma(nu) x^nu K_nu(x)   (d = 2),
 * response covariance Sigma~ = Sigma + nugget * I. */
typedef struct {
  double sigma1sq, c, a, gamma, nugget, alpha, delta, nu;
} vst_theta;

/* n space-time points in Vecchia order (device pointers). */
typedef struct {
  const double* xy;
  const double* t;
  int64_t n;
} vst_points;

/* k inducing points of the VIF model (Sect. 4.3), device pointers.  A NULL
 * pointer to this struct, or k == 0, selects the plain Vecchia model. */
typedef struct {
  const double* xy;
  const double* t;
  int64_t k;
} vst_inducing;

/* Device-side counters kept in the workspace header (see vst_workspace_status). */
typedef struct {
  int32_t status;        /* vst_status of the last call that used the workspace */
  int32_t reserved;
  int64_t bad_row;       /* first offending row, or -1 */
  int64_t n_fallback;    /* VST_MIXED: rows redone in FP64; vif_build_neighbors with
                            inducing points: rows searched by FP64 brute force */
  int64_t n_tie;         /* vif_build_neighbors: rows with a cut-off tie */
} vst_ws_info;

/* Host-only.  Map effective ranges to native parameters.  The effective
 * ranges are the distance (range_s) and lag (range_t) at which the
 * correlation decays to 0.05 (the convention of the paper's parameter tables,
 * Sect. 6 and Table A3):  M_nu(c range_s) = 0.05  and
 * (a range_t^{2 alpha} + 1)^{-(delta+gamma)} = 0.05.
 * Returns VST_EINVAL on non-positive ranges or an unsupported nu. */
vst_status vst_theta_from_ranges(double sigma1sq, double range_s, double range_t, double gamma,
                                 double nugget, double alpha, double delta, double nu,
                                 vst_theta* out);

/* Host-only.  Workspace bytes needed by any entry point below for n points,
 * m neighbours and k inducing points (k = 0: plain Vecchia). */
size_t vst_workspace_size(int64_t n, int m, int64_t k);
/* Workspace of vecchia_nll_grad with k > 0 inducing points (VIF). */
size_t vst_workspace_size_vif_grad(int64_t n, int m, int64_t k);

/* Correlation-based Vecchia neighbour selection (Sect. 4.4.1).
 * For every row i: the min(i, m) predecessors j < i with the largest
 * |rho_ij| = |Sigma_ij| / sqrt(Sigma_ii Sigma_jj) (latent covariance, no
 * nugget; equivalently the smallest d_c = sqrt(1 - |rho_ij|)), ranked in
 * FP64, ties broken by the smaller index, written to nn[i][0..] in decreasing
 * order of |rho|; nn_cnt[i] = min(i, m).
 * tie_rows (may be NULL): up to tie_cap rows (unordered) whose m-th and
 * (m+1)-th correlations differ by less than 1e-12 relative; their number is
 * vst_ws_info.n_tie.
 * The search is exact: a space-time bucket grid is pruned only by a rigorous
 * upper bound of the correlation over each bucket.
 * Synchronises `stream` once (to size the bucket grid from the point cloud's
 * bounding box).
 * VIF (ind != NULL, k > 0; Sect. 4.3 with the d_c metric of Sect. 4.4.1 on the
 * residual): the correlation is that of the latent residual
 * R = Sigma - U U^T (see vif_lowrank_u), |R_ij| / sqrt(R_ii R_jj), taken as 0
 * when R_ii or R_jj is at most 1e-12 sigma1sq; FP64 brute force over all
 * predecessors (O(n^2 k) work; for moderate n). */
vst_status vif_build_neighbors(const vst_points* pts, const vst_theta* theta, int m,
                               const vst_inducing* ind, int32_t* nn, int32_t* nn_cnt,
                               int64_t* tie_rows, int64_t tie_cap, void* workspace,
                               size_t ws_bytes, void* stream);

/* Vecchia factor of the response covariance Sigma~ (Sect. 4.1 with the nugget
 * of Sect. 3.1 on the diagonal): A_i = Sigma~_{i,N(i)} Sigma~_{N(i)}^{-1},
 * D_i = Sigma~_ii - A_i Sigma~_{i,N(i)}^T, N(i) = nn[i][0..nn_cnt[i]).
 * Entries q >= nn_cnt[i] of A[i] are set to 0.  Requires nn[i][q] < i.
 * VIF (ind != NULL, k > 0): the factor of the residual R + nugget I
 * (Sect. 4.3), R = Sigma - U U^T, so that
 * Sigma~_VIF = U U^T + B^{-1} diag(D) B^{-T}. */
vst_status vecchia_factor(const vst_points* pts, const vst_theta* theta, int m,
                          const vst_inducing* ind, const int32_t* nn, const int32_t* nn_cnt,
                          int precision, double* A, double* D, void* workspace,
                          size_t ws_bytes, void* stream);

/* Vecchia negative log-likelihood (Sect. 3.1 likelihood under the Vecchia
 * approximation of Sect. 4.1):
 *   nll = n/2 log(2 pi) + 1/2 sum_i log D_i + 1/2 sum_i (y_i - A_i y_N(i))^2 / D_i.
 * nll: one FP64 device scalar.  The sum is taken in a fixed order, so repeated
 * calls give the same bits.
 * VIF (ind != NULL, k > 0): -log N(y; 0, Sigma~_VIF) by the Woodbury identity
 * (the complexity remark of Sect. 4.3): with W = D^{-1/2} B U,
 * e = D^{-1/2} B y and M = I_k + W^T W,
 *   nll = n/2 log(2 pi) + 1/2 (sum_i log D_i + log det M)
 *         + 1/2 (e^T e - (W^T e)^T M^{-1} (W^T e)).
 * m = 0 gives the FITC likelihood (Sect. 4.2). */
vst_status vecchia_nll(const vst_points* pts, const vst_theta* theta, int m,
                       const vst_inducing* ind, const int32_t* nn, const int32_t* nn_cnt,
                       const double* y, int precision, double* nll, void* workspace,
                       size_t ws_bytes, void* stream);

/* NLL and its gradient with respect to the native parameters in the order
 * (sigma1sq, c, a, gamma, nugget); alpha, delta and nu are held fixed and the
 * neighbour sets are held fixed.  grad: 5 FP64 device values.  The factor is
 * recomputed, not stored.
 * VIF (ind != NULL, k > 0; the likelihood of Sect. 4.3 as in vecchia_nll,
 * inducing points held fixed): workspace vst_workspace_size_vif_grad(n, m, k)
 * bytes.  The gradient is the derivative of the VIF NLL, by an adjoint pass
 * through the Woodbury terms, the residual blocks and the low-rank part
 * U = Sigma_nk L^{-T} (L L^T = Sigma_kk); nll is the value vecchia_nll returns
 * for the same precision.  VST_FP64: FP64 throughout.  VST_MIXED /
 * VST_MIXED_BF16X3: the mixed NLL's FP32 low rank, W and residual Gram, the
 * dense products (n x k by k x k, and the k x k contraction over the points)
 * on split-BF16 tensor cores with FP32 accumulation, FP64 reductions over the
 * points and FP64 k x k algebra. */
vst_status vecchia_nll_grad(const vst_points* pts, const vst_theta* theta, int m,
                            const vst_inducing* ind, const int32_t* nn, const int32_t* nn_cnt,
                            const double* y, int precision, double* nll, double* grad,
                            void* workspace, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * Per-call options of the _ex entry points below.  A NULL pointer, or a
 * zero-initialised struct, selects every default.
 *  tau            VST_MIXED: a row is redone in FP64 when the condition
 *                 estimate of its local (|N(i)|+1)-block, (max_j L_jj /
 *                 min_j L_jj)^2 over the pivots of its FP32 Cholesky factor,
 *                 exceeds tau (rows whose FP32 Cholesky fails or whose D_i is
 *                 not positive are always redone).  <= 0: the default 1e4.
 *                 The number of such rows is vst_ws_info.n_fallback.
 *  row_begin,     plain Vecchia only: the sums run over the rows
 *  row_end        row_begin <= i < row_end (0 <= row_begin <= row_end <= n;
 *                 row_end == 0 means n).  The arrays keep their full length n
 *                 (a row may condition on any earlier point) and nll is
 *                 (row_end - row_begin)/2 log(2 pi) + the rows' terms, so
 *                 contiguous ranges that cover 0..n-1 give results that add up
 *                 to the full NLL and gradient (rows are independent given the
 *                 neighbour sets: ranges can be evaluated on separate GPUs and
 *                 summed, one reduction of six values).
 *  fallback_rows  optional uint8 DEVICE output indexed by row (length n, or
 *                 n_total for the batched call): 1 for a row the mixed form
 *                 redid in FP64, else 0.  Only rows in the range are written.
 *  wait_limit     vecchia_sample_ex: polls of a bounded device-side wait (on
 *                 a predecessor row) before it gives up and records
 *                 VST_ETIMEOUT (the row's value is then NaN); 0: the default
 *                 of about one second.
 * ------------------------------------------------------------------------ */
typedef struct {
  double tau;
  int64_t row_begin;
  int64_t row_end;
  uint8_t* fallback_rows;
  int64_t wait_limit;
} vst_options;

/* vecchia_nll_grad with options (plain Vecchia: ind must be NULL or k == 0;
 * otherwise VST_EINVAL).  opts: tau, row_begin/row_end, fallback_rows. */
vst_status vecchia_nll_grad_ex(const vst_points* pts, const vst_theta* theta, int m, const vst_inducing* ind,
                               const int32_t* nn, const int32_t* nn_cnt, const double* y, int precision,
                               const vst_options* opts, double* nll, double* grad, void* workspace,
                               size_t ws_bytes, void* stream);

/* Vecchia prediction at n_pred new points (the predictive distribution of
 * Sect. 3.1 under the Vecchia approximation of Sect. 4.1 with the
 * correlation-based neighbours of Sect. 4.4.1): every prediction point p
 * conditions on the min(m, n_train) training points of largest correlation
 * (all training points are candidates; ties to the smaller index), and
 *   mean[p] = A_p y_N(p),   var[p] = Sigma~_pp - A_p Sigma~_{N(p),p}
 * with A_p = Sigma~_{p,N(p)} Sigma~_{N(p)}^{-1}: the marginal predictive mean
 * and variance of the response (latent = 0) or, with latent != 0, of the
 * latent process (the nugget left out of var).  Prediction points do not
 * condition on one another.
 * train: n_train points (any order), y: their n_train responses; pred: n_pred
 * points; mean, var: n_pred FP64 device outputs; nn_out (may be NULL):
 * [n_pred][m] int32 training indices of the neighbours (-1 padded).
 * precision: VST_FP64 or VST_MIXED (VST_MIXED_BF16X3 = VST_MIXED here).
 * Workspace: vst_workspace_size_predict(n_train, n_pred, m) bytes.
 * Synchronises `stream` once (bounding box of the neighbour search). */
size_t vst_workspace_size_predict(int64_t n_train, int64_t n_pred, int m);
vst_status vecchia_predict(const vst_points* train, const vst_theta* theta, int m, const double* y,
                           const vst_points* pred, int precision, int latent, double* mean, double* var,
                           int32_t* nn_out, void* workspace, size_t ws_bytes, void* stream);

/* Space-time separated kMeans++ inducing points (Algorithm 3, Sect. 4.4.2):
 * m_s = round(sqrt(m n / |T|^2)) centres among the unique locations and
 * m_t = round(sqrt(m |T|^2 / n)) among the unique times (round = floor(x +
 * 1/2); clamped to [1, |S|], [1, |T|]), each by kMeans++ (first centre
 * uniform, then D^2 sampling) followed by lloyd_iters Lloyd steps; the k =
 * m_s m_t inducing points are the Cartesian product, point a m_t + b =
 * (location centre a, time centre b).  Draws: SplitMix64 from `seed` (times)
 * and seed ^ 0xD1B54A32D192ED03 (locations), u_j = (mix(x0 + (j+1) gamma)
 * >> 11) 2^-53.  D^2 weights and Lloyd sums are exact 64-bit integers
 * (2^32-scaled), so the result is deterministic and order-independent.
 * Unique locations are sorted lexicographically, unique times ascending.
 * xyk: [k_cap][2], tk: [k_cap] FP64 device outputs; k_out, ms_out, mt_out:
 * host outputs (ms_out, mt_out may be NULL).  VST_EINVAL if k > k_cap.
 * Synchronises `stream` several times.  Workspace:
 * vst_workspace_size_kmeans(n) bytes. */
size_t vst_workspace_size_kmeans(int64_t n);
vst_status vst_sts_kmeanspp(const vst_points* pts, int64_t m, uint64_t seed, int lloyd_iters, double* xyk,
                            double* tk, int64_t k_cap, int64_t* k_out, int64_t* ms_out, int64_t* mt_out,
                            void* workspace, size_t ws_bytes, void* stream);

/* VIF low-rank part (Sect. 4.3): Sigma_kk = L L^T (FP64 Cholesky of the
 * inducing-point covariance), U = Sigma_nk L^{-T} and the residual variances
 * r_i = sigma1sq - ||U_i||^2 (latent, no nugget).
 * U: [n][k] row-major FP64 device output; r: [n] FP64 device output.
 * precision: VST_FP64 (FP64 GEMM), VST_MIXED or VST_MIXED_BF16X3 (Sigma_nk
 * in FP32, U by the split-BF16 tensor-core GEMM, see vst_precision; U is
 * formed in FP32 and widened).  Workspace: vst_workspace_size(n, 0, k).
 * Sigma_kk not positive definite: VST_ENOTSPD in vst_workspace_status. */
vst_status vif_lowrank_u(const vst_points* pts, const vst_theta* theta, const vst_inducing* ind,
                         int precision, double* U, double* r, void* workspace, size_t ws_bytes,
                         void* stream);

/* The VIF's contraction over the points on the tensor cores (the products
 * W^T W, W^T e and e^T e of the Woodbury form in the complexity remark of
 * Sect. 4.3, and the gradient's k x k contractions): C = A^T B, or C = A^T A
 * when B is NULL (both triangles written).
 * A, B: [n][kc] FP32 device matrices, row strides lda, ldb >= kc (elements).
 * C: [kc][kc] row-major FP64 device output.  Column c of an operand gets,
 * in each block of 128 rows, the exponent E with max |A[i][c]| < 2^E over
 * the block, and each value is cut into three BF16 fixed-point parts of 9
 * bits (remainder at most 2^(E - 27)); six part products are kept, the
 * leading one summed exactly over each block, the corrections in FP32, the
 * blocks in double-float and FP64.  Values the parts hold exactly (integer
 * multiples of 2^(E - 8)) give C exactly while every partial sum stays below
 * 2^48 units of the product's leading power of two.
 * 1 <= kc <= 16384, 0 <= n < 2^31.  Workspace: vst_workspace_size_gram_tc(n,
 * kc) bytes, 256-byte aligned, caller-owned; a device wait that runs out is
 * reported as VST_ETIMEOUT by vst_workspace_status. */
size_t vst_workspace_size_gram_tc(int64_t n, int kc);
vst_status vif_gram_tc(int64_t n, int kc, const float* A, int64_t lda, const float* B, int64_t ldb, double* C,
                       void* workspace, size_t ws_bytes, void* stream);

/* Batched NLL and gradient of nsets independent datasets (one Vecchia model
 * each, Sect. 4.1 and 3.1) in one persistent launch.  Dataset d owns rows
 * offsets[d] .. offsets[d+1]-1 of the concatenated arrays xy, t, y, nn,
 * nn_cnt (layouts as above); its neighbour indices are local to the dataset
 * (0 = its first row).  offsets: nsets+1 int64 DEVICE values, offsets[0] = 0,
 * non-decreasing, offsets[nsets] = n_total.  thetas: nsets vst_theta in
 * DEVICE memory (so that a captured graph can be replayed after the caller
 * updates them in place); every dataset must use the same nu, passed as
 * `nu`.  nll: nsets FP64 device outputs; grad: [nsets][5] FP64 device
 * outputs (sigma1sq, c, a, gamma, nugget order).  Invalid offsets or
 * parameters are found on the device: vst_workspace_status then reports
 * VST_EINVAL with bad_row = the dataset index (or -2 for the offsets).
 * Workspace: vst_workspace_size_batched(nsets, n_total, m) bytes. */
size_t vst_workspace_size_batched(int nsets, int64_t n_total, int m);
vst_status vecchia_nll_grad_batched(int nsets, int64_t n_total, const int64_t* offsets,
                                    const vst_theta* thetas, double nu, const double* xy,
                                    const double* t, int m, const int32_t* nn, const int32_t* nn_cnt,
                                    const double* y, int precision, double* nll, double* grad,
                                    void* workspace, size_t ws_bytes, void* stream);

/* vecchia_nll_grad_batched with options: tau and fallback_rows (indexed by
 * the concatenated row index); row_begin and row_end must be 0. */
vst_status vecchia_nll_grad_batched_ex(int nsets, int64_t n_total, const int64_t* offsets,
                                       const vst_theta* thetas, double nu, const double* xy,
                                       const double* t, int m, const int32_t* nn, const int32_t* nn_cnt,
                                       const double* y, int precision, const vst_options* opts, double* nll,
                                       double* grad, void* workspace, size_t ws_bytes, void* stream);

/* A CUDA graph holding one vecchia_nll_grad_batched evaluation with the
 * given (device) buffers, captured once and replayed by vst_graph_launch on
 * any stream.  Replays read the buffers' current contents, so parameters,
 * responses or coordinates may be updated in place between replays; sizes,
 * pointers, m, nu and precision are fixed at capture.  The capture runs the
 * evaluation once (synchronously) before capturing it. */
typedef struct vst_graph_s* vst_graph;
vst_status vst_graph_capture_nll_grad_batched(int nsets, int64_t n_total, const int64_t* offsets,
                                              const vst_theta* thetas, double nu, const double* xy,
                                              const double* t, int m, const int32_t* nn,
                                              const int32_t* nn_cnt, const double* y, int precision,
                                              double* nll, double* grad, void* workspace,
                                              size_t ws_bytes, vst_graph* out);
vst_status vst_graph_launch(vst_graph graph, void* stream);
vst_status vst_graph_destroy(vst_graph graph);

/* Launch-shape autotuner.  Times the row kernel's launch shapes (resident
 * blocks per SM in {1, 2, 3, all that fit} x consecutive rows per warp in
 * {1, 4, 16, 64}) on the caller's inputs, keeps the fastest in the library's
 * tuned-shape cache (its only state across calls, keyed by batched/single,
 * precision, nu and the padded block size) and returns it.  Synchronises the
 * stream.  The environment variables VST_BLOCKS_PER_SM and VST_ROW_CHUNK
 * override the cache.  Results do not depend on the shape beyond rounding. */
typedef struct {
  int blocks_per_sm;  /* 0 = as many as fit */
  int row_chunk;
  float ms;           /* time of one evaluation with this shape */
} vst_tune_result;
vst_status vst_autotune_nll_grad(const vst_points* pts, const vst_theta* theta, int m,
                                 const int32_t* nn, const int32_t* nn_cnt, const double* y,
                                 int precision, void* workspace, size_t ws_bytes, void* stream,
                                 vst_tune_result* out);
vst_status vst_autotune_nll_grad_batched(int nsets, int64_t n_total, const int64_t* offsets,
                                         const vst_theta* thetas, double nu, const double* xy,
                                         const double* t, int m, const int32_t* nn,
                                         const int32_t* nn_cnt, const double* y, int precision,
                                         double* nll, double* grad, void* workspace, size_t ws_bytes,
                                         void* stream, vst_tune_result* out);
void vst_autotune_clear(void);

/* Draw y = B^{-1} D^{1/2} z, a sample of the Vecchia-approximated response
 * (y_i = A_i y_N(i) + sqrt(D_i) z_i in row order), with the FP64 factor of
 * (pts, theta, nn).  z: n FP64 device values; y: n FP64 device outputs. */
vst_status vecchia_sample(const vst_points* pts, const vst_theta* theta, int m,
                          const int32_t* nn, const int32_t* nn_cnt, const double* z, double* y,
                          void* workspace, size_t ws_bytes, void* stream);
/* vecchia_sample with options: wait_limit (the other fields must be 0). */
vst_status vecchia_sample_ex(const vst_points* pts, const vst_theta* theta, int m, const int32_t* nn,
                             const int32_t* nn_cnt, const double* z, double* y, const vst_options* opts,
                             void* workspace, size_t ws_bytes, void* stream);

/* Measurement hooks (not part of the method).  While enabled, the library
 * records a CUDA event pair on the launching stream around every launch of
 * its main kernels, by class: 0 = fused row kernel (NLL / gradient / factor),
 * 1 = FP64 fallback row kernel of the mixed form, 2 = neighbour query kernel,
 * 3 = Vecchia sampling kernel, 4 = VIF low-rank GEMM U = Sigma_nk L^{-T},
 * 5 = VIF per-row residual Gram, 6 = VIF [W e]^T [W e] product, 7 = VIF
 * residual-correlation candidate filter (tensor cores).
 * vst_profile_read() synchronises on the
 * recorded events and returns the number of launches of that class and their
 * summed device time (ms) since the last vst_profile_enable(1).  At most 4096
 * launches are recorded; later ones are counted but not timed (returns 1 if
 * any launch of the class was dropped, 0 otherwise, -1 on a bad class).
 * Not for use while a stream is being captured into a graph.  Host-only
 * bookkeeping, not thread-safe. */
void vst_profile_enable(int on);
int vst_profile_read(int kernel_class, int64_t* launches, double* total_ms);

/* ------------------------------------------------------------------------
 * No-allocation entry point.  The paper has no counterpart to this call: it
 * exists for callers that cannot call cudaMalloc at all -- code that runs
 * inside a host application which owns every device allocation (a fixed
 * memory pool, or a strict memory budget checked by its allocator), or code
 * on a latency-critical path, where cudaMalloc's implicit device-wide
 * synchronisation and possible failure are not acceptable.
 *
 * vecchia_nll_grad_noalloc computes what vecchia_nll_grad computes for plain
 * Vecchia (no inducing points: the call has no inducing-point argument), with
 * the same arguments minus the workspace, in any precision that call accepts
 * (VST_MIXED_BF16X3 is VST_MIXED here) and with the same launch shape (the
 * autotuner's cached shape, if any).  Its scratch memory is one file-scope
 * device array of 77,644,032 bytes (about 74 MiB; vst_noalloc_scratch_bytes()
 * returns the exact size) that every GPU loading the library holds until the
 * process exits: a 256-byte header, the FP64 and FP32 lag tables (32 KiB +
 * 16 KiB), two buffers of per-warp partial sums (2 x 4 MiB), one fallback flag
 * byte per point and one 32-byte mixed-form record per point (2^21 points
 * each).  It allocates nothing: no cudaMalloc/cudaFree and no allocating
 * library routine.
 *  - n may not exceed VST_NOALLOC_MAX_N (2^21 points); larger n returns
 *    VST_EINVAL with a message -- use vecchia_nll_grad with a workspace.
 *  - The first call on each device (and the first call after the device's
 *    context was reset) looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current); make that first call
 *    before capturing the stream into a CUDA graph.
 *  - Every call shares the one array and overwrites it (each call resets the
 *    parts that must start at zero).  Calls that may overlap on the GPU --
 *    on different streams, or from different host threads -- race on it and
 *    must not be issued concurrently; calls on one stream are ordered.
 *  - Device-side status of the last call: vst_noalloc_status().
 * ------------------------------------------------------------------------ */
#define VST_NOALLOC_MAX_N (1 << 21)
vst_status vecchia_nll_grad_noalloc(const vst_points* pts, const vst_theta* theta, int m,
                                    const int32_t* nn, const int32_t* nn_cnt, const double* y,
                                    int precision, double* nll, double* grad, void* stream);
/* Size in bytes of the static scratch array used by the call above. */
size_t vst_noalloc_scratch_bytes(void);
/* Like vst_workspace_status, for the static scratch of the no-allocation call
 * on the current device. */
vst_status vst_noalloc_status(void* stream, vst_ws_info* info);

/* Synchronise `stream` and copy the workspace header (device-side status and
 * counters of the last call on this workspace) into *info (may be NULL).
 * Returns info->status. */
vst_status vst_workspace_status(const void* workspace, void* stream, vst_ws_info* info);

/* Thread-local text of the last host-side error (empty if none). */
const char* vst_last_error(void);

/* Library version (major * 10000 + minor * 100 + patch). */
int vst_version(void);

#ifdef __cplusplus
}
#endif

#endif /* VST_H */
