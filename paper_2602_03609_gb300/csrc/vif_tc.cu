// The VIF's dense products on the tensor cores (mixed form), BF16 tcgen05
// GEMMs with split operands: the low rank U = Sigma_nk L^{-T} (Sect. 4.3), the
// gradient's n x k products Y = W M^{-1} and H = G_U L^{-1} (tc_product), and
// its contraction over the points J = H^T U (tc_gram, a warp-specialised
// split-K kernel described above gram_tc_kernel).
//
// Each FP32 operand value v is split into P BF16 parts, v ~ v_0 + v_1 + ...,
// v_0 = bf16(v), v_j = bf16(v - v_0 - ... - v_{j-1}).  The product of two
// split values keeps the terms whose part indices sum to at most P - 1:
//   P = 2: a0 b0 + a0 b1 + a1 b0                       (3 products)
//   P = 3: a0 b0 + a0 b1 + a1 b0 + a0 b2 + a1 b1 + a2 b0 (6 products)
// all accumulated in one FP32 accumulator in tensor memory.  Two parts carry
// 16 significand bits (relative error ~1e-5 per product), three parts carry
// 24 (the FP32 level).
//
// The contractions over the points (tc_gram, tc_syrk) use a fixed-point
// split instead, in 128-row blocks: column c of an operand gets, in each
// block, the exponent E with max |S[i][c]| < 2^E over the block's rows, and
// x = S[i][c] becomes
//   x 2^(8 - E) = s_0 + 2^-9 s_1 + 2^-18 s_2 + (a remainder below 2^-19)
// with integers |s_j| <= 256, each exact in BF16 (part j holds s_j 2^(-9 j)).
// The leading products s_0 s_0' are integers below 2^16 and the sum of one
// block's 128 of them an integer below 2^23, so the leading accumulator of
// one drain (one block) is exact whatever the tensor core's rounding: the
// rounding bias of the floating split (one sign for the positive sums on a
// Gram's diagonal) does not build up over n rows.  The other kept products,
// 2^-9 smaller and below, go to the correction accumulator.  The drain scales
// both by the block's power of two relative to the columns' largest exponents
// (exact) before adding them to its double-float sums, and the segment sum
// applies 2^(E_a + E_b - 16) of those largest exponents in FP64.  These
// contractions always take three parts (six products), which leave a
// remainder of at most 2^(E - 27) per value: the Woodbury form cancels two
// O(n) terms, and two parts (2^(E - 18)) moved the VIF NLL by ~1e-4 per point.
//
// Operands in HBM, K-major BF16 (K = inducing point index p, padded to kp):
//   A parts [P][n][kp]   A[i][p] = Sigma(x_i, z_p), FP32 evaluation
//   B parts [P][kp][kp]  B[c][p] = (L^{-1})[c][p]  (lower triangular)
// so that U[i][c] = sum_p A[i][p] B[c][p]; tile columns c0..c0+BN-1 need only
// p < c0 + BN.
//
// GEMM kernel: one CTA of 4 warps per 128 x BN output tile.  Warp 0 lane 0
// issues the TMA loads of 64-wide K blocks (128-byte swizzle) into a ring of
// STAGES shared-memory stages; warp 1 lane 0 issues tcgen05.mma (M = 128,
// N = BN, K = 16 per instruction) into two TMEM accumulators of BN columns,
// one for the leading product a0 b0 and one for the smaller correction
// products (the tensor core's FP32 accumulation is not round-to-nearest, and
// a separate accumulator keeps the corrections from adding rounding steps to
// the large sum; the two are added once in the epilogue), and
// frees each stage with tcgen05.commit (the other lanes of both warps follow
// their lane 0 through the waits); then all four warps read the
// accumulator (warp w owns TMEM lanes 32w..32w+31 = tile rows) and store U.
// Every wait is limited in time; a wait that runs out reports VST_ETIMEOUT and
// the CTA still frees its tensor memory.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "kernels.h"
#include "profile.h"
#include "umma.cuh"
#include "vif.h"
#include "workspace.h"

namespace vst {

vst_status fail(vst_status s, const char* fmt, ...);
vst_status cuda_fail(cudaError_t e, const char* where);
void launch_init_header(WsHeader* h, cudaStream_t st);

namespace {

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per wait

template <int P, int BN, int STAGES>
struct TcShape {
  static constexpr int BM = 128, BK = 64;
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = P * (A_BYTES + B_BYTES);
  static constexpr int BAR_BYTES = 256;
  static constexpr int SMEM = STAGES * STAGE_BYTES + BAR_BYTES + 1024;  // + alignment slack
  static_assert(STAGE_BYTES % 1024 == 0, "stage alignment");
  static_assert(BN % 32 == 0 && BN >= 32 && BN <= 256, "N tile");
};

// BF16 parts of an FP64 value (residuals exact in FP64)
template <int P>
__device__ __forceinline__ void split_parts(double v, __nv_bfloat16 (&o)[P]) {
#pragma unroll
  for (int j = 0; j < P; ++j) {
    o[j] = __double2bfloat16(v);
    v -= (double)__bfloat162float(o[j]);
  }
}
// ... of an FP32 value (residuals exact in FP32)
template <int P>
__device__ __forceinline__ void split_parts(float v, __nv_bfloat16 (&o)[P]) {
#pragma unroll
  for (int j = 0; j < P; ++j) {
    o[j] = __float2bfloat16_rn(v);
    v -= __bfloat162float(o[j]);
  }
}

// B parts from X = L^{-1} (FP64, row-major k x k, lower): [P][kp][kp], zero
// outside the lower triangle and the k x k block.
template <int P>
__global__ void split_x_kernel(const double* X, int k, int kp, __nv_bfloat16* B) {
  const int64_t total = (int64_t)kp * kp;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(id / kp), p = (int)(id % kp);
    const double v = (c < k && p <= c) ? X[(int64_t)c * k + p] : 0.0;
    __nv_bfloat16 o[P];
    split_parts<P>(v, o);
#pragma unroll
    for (int j = 0; j < P; ++j) B[(int64_t)j * total + id] = o[j];
  }
}

// A parts from an FP32 matrix (row stride lda): [P][n][kp], zero beyond k
template <int P>
__global__ void split_a_kernel(const float* A, int64_t lda, int64_t n, int k, int kp, __nv_bfloat16* Ap) {
  const int groups = kp / 8;
  const int64_t total = n * groups;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = id / groups;
    const int p0 = (int)(id % groups) * 8;
    __align__(16) __nv_bfloat16 o[P][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int p = p0 + q;
      __nv_bfloat16 s[P];
      split_parts<P>(p < k ? A[i * lda + p] : 0.0f, s);
#pragma unroll
      for (int j = 0; j < P; ++j) o[j][q] = s[j];
    }
#pragma unroll
    for (int j = 0; j < P; ++j)
      *reinterpret_cast<uint4*>(Ap + ((int64_t)j * n + i) * kp + p0) = *reinterpret_cast<const uint4*>(o[j]);
  }
}

// B parts [P][kp][kp] from an FP64 k x k matrix M: mode 1, B[c][p] = M[c][p];
// mode 2, B[c][p] = M[p][c] for p >= c (M lower triangular); zero elsewhere
template <int P>
__global__ void split_b_kernel(const double* M, int k, int kp, int mode, __nv_bfloat16* B) {
  const int64_t total = (int64_t)kp * kp;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(id / kp), p = (int)(id % kp);
    double v = 0.0;
    if (c < k && p < k) {
      if (mode == 1) v = M[(int64_t)c * k + p];
      else if (p >= c) v = M[(int64_t)p * k + c];
    }
    __nv_bfloat16 o[P];
    split_parts<P>(v, o);
#pragma unroll
    for (int j = 0; j < P; ++j) B[(int64_t)j * total + id] = o[j];
  }
}

// exponent E with |x| < 2^E for every x whose largest magnitude has the
// FP32 bit pattern bits (zero and subnormal maxima give E = -126)
__device__ __forceinline__ int fx_exp(unsigned bits) { return (int)((bits >> 23) & 0xffu) - 126; }

// fixed-point parts of x given the shift sh = 8 - E
template <int P>
__device__ __forceinline__ void split_fixed(float x, int sh, __nv_bfloat16 (&o)[P]) {
  float r = ldexpf(x, sh);  // |r| < 256
#pragma unroll
  for (int j = 0; j < P; ++j) {
    const float sj = rintf(r);  // an integer, |sj| <= 256
    o[j] = __float2bfloat16_rn(j == 0 ? sj : j == 1 ? sj * 0x1p-9f : sj * 0x1p-18f);
    r = (r - sj) * 512.0f;  // exact: |r - sj| <= 1/2 is a multiple of r's last place
  }
}

// column exponents are kept biased by kFxBias (positive, for atomicMax)
constexpr int kFxBias = 1024;

// Transposed fixed-point parts of an FP32 matrix S [n][k] (row stride lds):
// T[j][c][i] = part j of S[i][c], [P][kp][np], zero for i >= n or c >= k,
// with the exponent of column c over the 128-row block of row i, stored in
// eblk[i / 128][c]; eg[c] (zeroed beforehand) collects the largest block
// exponent of column c < k plus kFxBias.  One block of 256 threads per
// 128 x 64 tile, staged through shared memory so that both the reads (along
// c) and the writes (along i) are contiguous.  NaNs are passed over by the
// maxima and reach the products through the parts.
template <int P>
__global__ void __launch_bounds__(256) split_fx_t_kernel(const float* S, int64_t lds, int64_t n, int k, int kp,
                                                         int64_t np, __nv_bfloat16* T, int16_t* eblk, int* eg) {
  __shared__ float tile[128][65];
  __shared__ unsigned cmax[4][64];
  __shared__ int esh[64];
  const int64_t i0 = (int64_t)blockIdx.x * 128;
  const int c0 = blockIdx.y * 64;
  const int tc = threadIdx.x & 63, tr = threadIdx.x >> 6;
  float mx = 0.0f;
#pragma unroll 8
  for (int q = 0; q < 32; ++q) {
    const int r = tr + 4 * q;
    const int64_t i = i0 + r;
    const int c = c0 + tc;
    const float v = (i < n && c < k) ? S[i * lds + c] : 0.0f;
    tile[r][tc] = v;
    mx = fmaxf(mx, fabsf(v));
  }
  cmax[tr][tc] = __float_as_uint(mx);  // non-negative floats order as their bit patterns
  __syncthreads();
  if (threadIdx.x < 64) {
    const int t = threadIdx.x;
    const unsigned m = max(max(cmax[0][t], cmax[1][t]), max(cmax[2][t], cmax[3][t]));
    const int E = fx_exp(m);
    esh[t] = E;
    eblk[(int64_t)blockIdx.x * kp + c0 + t] = (int16_t)E;
    if (c0 + t < k) atomicMax(eg + c0 + t, E + kFxBias);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) {  // 64 columns x 16 groups of 8 rows
    const int item = threadIdx.x + 256 * q;
    const int cr = item >> 4, g = item & 15;
    const int sh = 8 - esh[cr];
    __align__(16) __nv_bfloat16 o[P][8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      __nv_bfloat16 sp[P];
      split_fixed<P>(tile[g * 8 + e][cr], sh, sp);
#pragma unroll
      for (int j = 0; j < P; ++j) o[j][e] = sp[j];
    }
#pragma unroll
    for (int j = 0; j < P; ++j)
      *reinterpret_cast<uint4*>(T + ((int64_t)j * kp + c0 + cr) * np + i0 + g * 8) =
          *reinterpret_cast<const uint4*>(o[j]);
  }
}

// the pieces of one operand in its tc_operand_bytes region
struct FxOperand {
  __nv_bfloat16* parts;
  int16_t* eblk;
  int* eg;
};
FxOperand fx_operand(char* p, int64_t n, int kc) {
  const size_t kp = (size_t)vif_kp(kc > 0 ? kc : 1);
  const size_t np = (size_t)((n > 0 ? n : 1) + 127) / 128 * 128;
  FxOperand o;
  o.parts = reinterpret_cast<__nv_bfloat16*>(p);
  o.eblk = reinterpret_cast<int16_t*>(p + align256(2 * (size_t)kVifMaxParts * kp * np));
  o.eg = reinterpret_cast<int*>(reinterpret_cast<char*>(o.eblk) + align256(2 * (np / 128) * kp));
  return o;
}

// double-float coordinates of the inducing points
__global__ void ind_coords_kernel(const double* xyk, int k, float4* zf) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= k) return;
  const double x = xyk[2 * p], y = xyk[2 * p + 1];
  const float xh = (float)x, yh = (float)y;
  zf[p] = make_float4(xh, (float)(x - (double)xh), yh, (float)(y - (double)yh));
}

// A parts: one thread per (row i, 8 consecutive inducing points); the
// covariance in FP32 as in the SIMT path (per-day lag factors rounded once
// from FP64, double-float coordinate differences), then split.
template <int NU, int P>
__global__ void snk_split_kernel(const double* xy, const double* t, int64_t n, const double* xyk, const double* tk,
                                 const float4* zf, int k, int kp, DevTheta th, const int64_t* dinfo,
                                 const float2* dtab, __nv_bfloat16* A) {
  const int groups = kp / 8;
  const int64_t total = n * groups;
  const bool use_tab = dinfo[2] != 0;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = id / groups;
    const int p0 = (int)(id % groups) * 8;
    const double xi = xy[2 * i], yi = xy[2 * i + 1], ti = t[i];
    const float xh = (float)xi, yh = (float)yi;
    const float4 a = make_float4(xh, (float)(xi - (double)xh), yh, (float)(yi - (double)yh));
    const int64_t day = use_tab ? (int64_t)ti - dinfo[0] : 0;
    __align__(16) __nv_bfloat16 o[P][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int p = p0 + q;
      float v = 0.0f;
      if (p < k) {
        if (use_tab) {
          const float2 pg = dtab[day * k + p];
          const float4 b = zf[p];
          const float dx = (a.x - b.x) + (a.y - b.y), dy = (a.z - b.z) + (a.w - b.w);
          const float x = pg.y * sqrtf(dx * dx + dy * dy);
          v = pg.x * matern_M<NU, float>(x, expf(-x));
        } else {
          v = cov32<NU>(th, (float)(xi - xyk[2 * p]), (float)(yi - xyk[2 * p + 1]), (float)(ti - tk[p]));
        }
      }
      __nv_bfloat16 s[P];
      split_parts<P>(v, s);
#pragma unroll
      for (int j = 0; j < P; ++j) o[j][q] = s[j];
    }
#pragma unroll
    for (int j = 0; j < P; ++j)
      *reinterpret_cast<uint4*>(A + ((int64_t)j * n + i) * kp + p0) = *reinterpret_cast<const uint4*>(o[j]);
  }
}

// part index pairs (a, b) of the kept products, a + b <= P - 1
template <int P>
struct SplitTerms;
template <>
struct SplitTerms<2> {
  static constexpr int N = 3;
  static __device__ __forceinline__ int a(int t) { return t == 2 ? 1 : 0; }
  static __device__ __forceinline__ int b(int t) { return t == 1 ? 1 : 0; }
};
template <>
struct SplitTerms<3> {
  static constexpr int N = 6;
  // (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
  static __device__ __forceinline__ int a(int t) { return t == 2 ? 1 : t == 4 ? 1 : t == 5 ? 2 : 0; }
  static __device__ __forceinline__ int b(int t) { return t == 1 ? 1 : t == 3 ? 2 : t == 4 ? 1 : 0; }
};

// K range of a column tile: KMODE 0, B[c][p] = 0 for p > c (K up to the
// tile's last column); 1, the whole K; 2, B[c][p] = 0 for p < c (K from the
// tile's first column).  RPART: also the row sums of the squared outputs.
template <int P, int BN, int STAGES, int KMODE = 0, bool RPART = true>
__global__ void __launch_bounds__(128, 1)
    ugemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t n,
                    int k, int kp, float* U, double* rpart, WsHeader* hdr) {
  using S = TcShape<P, BN, STAGES>;
  extern __shared__ unsigned char tc_smem[];
  const uint32_t raw = umma::smem_u32(tc_smem);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = tc_smem + (base - raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(gbase + STAGES * S::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accf + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // consecutive CTAs share the A tile (N tile fastest), so that its reads
  // across the kp / BN column tiles come from L2
  const int ntile = kp / BN;
  const int64_t m0 = (int64_t)(blockIdx.x / ntile) * S::BM;
  const int c0 = (int)(blockIdx.x % ntile) * BN;
  const int kend = KMODE == 0 ? (kp < c0 + BN ? kp : c0 + BN) : kp;
  const int kb0 = KMODE == 2 ? c0 / S::BK : 0;
  const int nkb = (kend + S::BK - 1) / S::BK - kb0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      umma::mbar_init(&full[s], 1);
      umma::mbar_init(&empty[s], 1);
    }
    umma::mbar_init(accf, 1);
    umma::fence_mbar_init();
  }
  if (warp == 0) {
    umma::tmem_alloc(umma::smem_u32(tslot), 2 * BN);
    umma::tmem_relinquish();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *tslot;
  bool ok = true;
  // lane 0 waits, the warp takes its answer (the warps stay converged)
  auto warp_wait = [&](uint64_t* bar, uint32_t parity) {
    bool done = true;
    if (lane == 0) done = umma::mbar_wait(bar, parity, kWaitLimitNs);
    return __shfl_sync(0xffffffffu, done ? 1 : 0, 0) != 0;
  };

  if (warp == 0) {
    // producer: TMA loads of the K blocks (lane 0 issues)
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES;
      const uint32_t use = (uint32_t)(kb / STAGES);
      if (use > 0 && !warp_wait(&empty[s], (use - 1) & 1u)) {
        ok = false;
        break;
      }
      if (lane == 0) {
        umma::mbar_arrive_expect_tx(&full[s], S::STAGE_BYTES);
        const uint32_t sa = base + s * S::STAGE_BYTES, sb = sa + P * S::A_BYTES;
#pragma unroll
        for (int j = 0; j < P; ++j) {
          umma::tma_load_2d(sa + j * S::A_BYTES, &tmA, (kb0 + kb) * S::BK, (int)(j * n + m0), &full[s]);
          umma::tma_load_2d(sb + j * S::B_BYTES, &tmB, (kb0 + kb) * S::BK, j * kp + c0, &full[s]);
        }
      }
      __syncwarp();
    }
  } else if (warp == 1) {
    // MMA issuer (lane 0 issues)
    constexpr uint32_t idesc = umma::idesc_bf16_f32(S::BM, BN);
    uint32_t acc_main = 0, acc_corr = 0;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES;
      const uint32_t use = (uint32_t)(kb / STAGES);
      if (!warp_wait(&full[s], use & 1u)) {
        ok = false;
        break;
      }
      umma::fence_after_sync();
      if (lane == 0) {
        const uint32_t sa = base + s * S::STAGE_BYTES, sb = sa + P * S::A_BYTES;
#pragma unroll
        for (int kk = 0; kk < S::BK / 16; ++kk) {
#pragma unroll
          for (int q = 0; q < SplitTerms<P>::N; ++q) {
            const uint64_t ad = umma::desc_kmajor_sw128(sa + SplitTerms<P>::a(q) * S::A_BYTES + kk * 32);
            const uint64_t bd = umma::desc_kmajor_sw128(sb + SplitTerms<P>::b(q) * S::B_BYTES + kk * 32);
            if (q == 0) {
              umma::mma_bf16(tmem, ad, bd, idesc, acc_main);
              acc_main = 1;
            } else {
              umma::mma_bf16(tmem + BN, ad, bd, idesc, acc_corr);
              acc_corr = 1;
            }
          }
        }
        umma::mma_commit(&empty[s]);
      }
      __syncwarp();
    }
    if (lane == 0) umma::mma_commit(accf);
    __syncwarp();
  }

  // epilogue: TMEM -> registers -> U (FP32, row-major [n][k])
  if (!warp_wait(accf, 0)) ok = false;
  umma::fence_after_sync();
  const int64_t i = m0 + warp * 32 + lane;
  const bool vec = (k & 3) == 0;
  df sq = {0.f, 0.f};  // this row's sum of U_ic^2 over the tile, double-float
#pragma unroll 1
  for (int cb = 0; cb < BN; cb += 32) {
    uint32_t v[32], w[32];
    const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb;
    umma::tmem_ld_32x32b_x32(ta, v);
    umma::tmem_ld_32x32b_x32(ta + BN, w);
    umma::tmem_wait_ld();
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = __float_as_uint(__uint_as_float(v[q]) + __uint_as_float(w[q]));
    const int cc = c0 + cb;
    if constexpr (RPART) {
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const float u = __uint_as_float(v[q]);
        if (cc + q < k) df_fma_acc(sq, u, df{u, 0.f});
      }
    }
    if (i < n && cc < k) {
      float* dst = U + i * k + cc;
      if (vec && cc + 32 <= k) {
#pragma unroll
        for (int q = 0; q < 32; q += 4)
          *reinterpret_cast<float4*>(dst + q) = make_float4(__uint_as_float(v[q]), __uint_as_float(v[q + 1]),
                                                            __uint_as_float(v[q + 2]), __uint_as_float(v[q + 3]));
      } else {
#pragma unroll
        for (int q = 0; q < 32; ++q)
          if (cc + q < k) dst[q] = __uint_as_float(v[q]);
      }
    }
  }
  if (RPART && i < n) rpart[i * ntile + c0 / BN] = df_to_double(sq);
  if (!ok) report_error(hdr, VST_ETIMEOUT, m0);
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tmem, 2 * BN);
}

// ---- C = A^T B over the rows of A and B (split K, warp-specialised) ----
//
// The operands come as transposed BF16 parts [P][kp][np] (split_fx_t_kernel):
// row c of part j holds part j of column c over the np rows (zero padded), so
// C[a][b] = sum_i At[a][i] Bt[b][i] is a K-major product with K = the row
// index.  A CTA computes one 128 x 128 output tile (of all T x T tiles, or of
// the lower triangle when tri) over one K segment of whole 128-row blocks.
// Warp 0 issues the TMA loads; warp 1 issues the MMAs into two TMEM buffers,
// each a main accumulator (a0 b0) and a correction accumulator (the other
// kept part products) of 128 columns; warps 4-11 drain a buffer every
// kGramDrainKb K blocks into double-float sums held in registers (warp w
// reads TMEM lanes 32 (w % 4) .. + 31 = tile rows, and columns
// 64 ((w - 4) / 4) .. + 63) while the MMAs fill the other buffer.  Warps 2-3
// only fill out the first warpgroup, which gives registers to the two
// draining warpgroups (384 threads launch with 168 registers each, 64,512 in
// all; 128 x 64 + 256 x 216 = 63,488).  One drain per 128-row block keeps
// the leading accumulator's fixed-point sum below 2^23, hence exact, and each
// correction run to 8 accumulation steps; the drain scales both by
// 2^(E_a - Eg_a + E_b - Eg_b) (the block's exponents against the columns'
// largest, at most 1, exact; below 2^-126 the block's terms are dropped) and
// the double-float sums carry ~48 bits over the whole segment.  Each CTA
// writes its tile (rows and columns < kc) in FP64 to out[segment];
// gram_sum_kernel adds the segments in a fixed order.
constexpr int kGramDrainKb = 2;
constexpr int kGramMaxSeg = 16;
static_assert(kGramDrainKb == 2, "one drain per 128-row exponent block");
static_assert(kGramDrainKb * 64 * 256 * 256 <= (1 << 23), "leading fixed-point sum of one drain exact in FP32");

template <int P, int STAGES>
struct GramTcShape {
  static constexpr int BM = 128, BN = 128, BK = 64;
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = P * (A_BYTES + B_BYTES);
  static constexpr int SMEM = STAGES * STAGE_BYTES + 256 + 1024 + 1024;  // + barriers, column exponents, slack
  static constexpr int THREADS = 384;
  static constexpr int REGS_LOW = 64, REGS_HIGH = 216;
  static_assert(128 * REGS_LOW + 256 * REGS_HIGH <= THREADS * 168, "register split");
  static_assert(STAGE_BYTES % 1024 == 0, "stage alignment");
  static_assert(SMEM <= 232448, "shared memory");
  static_assert(BM * (BN + 1) * 8 <= STAGES * STAGE_BYTES, "output tile staging");
};

template <int P, int STAGES>
__global__ void __launch_bounds__(384, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t np,
                   int kc, int kp, int nseg, int tri, const int16_t* ea_blk, const int* ea_g,
                   const int16_t* eb_blk, const int* eb_g, double* out, WsHeader* hdr) {
  using S = GramTcShape<P, STAGES>;
  extern __shared__ unsigned char tc_smem[];
  const uint32_t raw = umma::smem_u32(tc_smem);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = tc_smem + (base - raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(gbase + STAGES * S::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;  // [2] buffer filled
  uint64_t* acce = accf + 2;        // [2] buffer drained
  uint64_t* done = acce + 2;        // every MMA finished
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile uint32_t* drain_fail = tslot + 1;  // a drain warp's wait ran out
  int* egs = reinterpret_cast<int*>(gbase + STAGES * S::STAGE_BYTES + 256);  // [128 rows | 128 columns]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int T = kp / S::BM;
  const int ntiles = tri ? T * (T + 1) / 2 : T * T;
  const int tile = (int)(blockIdx.x % ntiles), seg = (int)(blockIdx.x / ntiles);
  int tm = tile / T, tn = tile % T;
  if (tri) {  // the lower triangle of tiles, tn <= tm
    tm = 0;
    while ((tm + 1) * (tm + 2) / 2 <= tile) ++tm;
    tn = tile - tm * (tm + 1) / 2;
  }
  // this segment's 128-row blocks (two K blocks each): the first (nb % nseg)
  // segments take one more
  const int64_t nb = np / 128;
  const int64_t per = nb / nseg, rem = nb % nseg;
  const int64_t b0 = seg * per + (seg < rem ? seg : rem);
  const int ndr = (int)(per + (seg < rem ? 1 : 0));
  const int64_t kb0 = 2 * b0;
  const int nkb = 2 * ndr;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      umma::mbar_init(&full[s], 1);
      umma::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      umma::mbar_init(&accf[b], 1);
      umma::mbar_init(&acce[b], 8);
    }
    umma::mbar_init(done, 1);
    *drain_fail = 0u;
    umma::fence_mbar_init();
  }
  for (int q = threadIdx.x; q < 256; q += S::THREADS)
    egs[q] = q < 128 ? ea_g[tm * S::BM + q] - kFxBias : eb_g[tn * S::BN + q - 128] - kFxBias;
  if (warp == 0) {
    umma::tmem_alloc(umma::smem_u32(tslot), 512);
    umma::tmem_relinquish();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *tslot;
  bool ok = true;
  auto warp_wait = [&](uint64_t* bar, uint32_t parity) {
    bool d = true;
    if (lane == 0) d = umma::mbar_wait(bar, parity, kWaitLimitNs);
    return __shfl_sync(0xffffffffu, d ? 1 : 0, 0) != 0;
  };

  if (warp < 4) {
    umma::regs_dec<S::REGS_LOW>();
    if (warp == 0) {
      // producer
      int issued = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % STAGES;
        const uint32_t use = (uint32_t)(kb / STAGES);
        if (use > 0 && !warp_wait(&empty[s], (use - 1) & 1u)) {
          ok = false;
          break;
        }
        if (lane == 0) {
          umma::mbar_arrive_expect_tx(&full[s], S::STAGE_BYTES);
          const uint32_t sa = base + s * S::STAGE_BYTES, sb = sa + P * S::A_BYTES;
          const int x = (int)((kb0 + kb) * S::BK);
#pragma unroll
          for (int j = 0; j < P; ++j) {
            umma::tma_load_2d(sa + j * S::A_BYTES, &tmA, x, j * kp + tm * S::BM, &full[s]);
            umma::tma_load_2d(sb + j * S::B_BYTES, &tmB, x, j * kp + tn * S::BN, &full[s]);
          }
        }
        __syncwarp();
        ++issued;
      }
      if (!ok) {
        // let the loads still in flight land before the CTA's shared memory goes
        for (int kb = issued - STAGES < 0 ? 0 : issued - STAGES; kb < issued; ++kb)
          warp_wait(&full[kb % STAGES], (uint32_t)(kb / STAGES) & 1u);
      }
    } else if (warp == 1) {
      // MMA issuer
      constexpr uint32_t idesc = umma::idesc_bf16_f32(S::BM, S::BN);
      int kb = 0;
      for (int d = 0; d < ndr && ok; ++d) {
        const int b = d & 1;
        const uint32_t u = (uint32_t)(d >> 1);
        if (u > 0 && !warp_wait(&acce[b], (u - 1) & 1u)) {
          ok = false;
          break;
        }
        umma::fence_after_sync();
        const uint32_t tb = tmem + (uint32_t)(b * 256);
        const int nk = nkb - d * kGramDrainKb < kGramDrainKb ? nkb - d * kGramDrainKb : kGramDrainKb;
        uint32_t acc_main = 0, acc_corr = 0;
        for (int j = 0; j < nk; ++j, ++kb) {
          const int s = kb % STAGES;
          const uint32_t use = (uint32_t)(kb / STAGES);
          if (!warp_wait(&full[s], use & 1u)) {
            ok = false;
            break;
          }
          umma::fence_after_sync();
          if (lane == 0) {
            const uint32_t sa = base + s * S::STAGE_BYTES, sb = sa + P * S::A_BYTES;
#pragma unroll
            for (int kk = 0; kk < S::BK / 16; ++kk) {
#pragma unroll
              for (int q = 0; q < SplitTerms<P>::N; ++q) {
                const uint64_t ad = umma::desc_kmajor_sw128(sa + SplitTerms<P>::a(q) * S::A_BYTES + kk * 32);
                const uint64_t bd = umma::desc_kmajor_sw128(sb + SplitTerms<P>::b(q) * S::B_BYTES + kk * 32);
                if (q == 0) {
                  umma::mma_bf16(tb, ad, bd, idesc, acc_main);
                  acc_main = 1;
                } else {
                  umma::mma_bf16(tb + S::BN, ad, bd, idesc, acc_corr);
                  acc_corr = 1;
                }
              }
            }
            umma::mma_commit(&empty[s]);
          }
          __syncwarp();
        }
        if (!ok) break;
        if (lane == 0) umma::mma_commit(&accf[b]);
        __syncwarp();
      }
      // every MMA this thread issued has finished before the tensor memory is freed
      if (lane == 0) umma::mma_commit(done);
      __syncwarp();
      if (!warp_wait(done, 0)) ok = false;
    }
  } else {
    umma::regs_inc<S::REGS_HIGH>();
    // drain warps
    const int q4 = warp & 3, half = (warp - 4) >> 2;
    float hi[64], lo[64];
#pragma unroll
    for (int c = 0; c < 64; ++c) hi[c] = lo[c] = 0.f;
    const int arow = q4 * 32 + lane;
    const int16_t* ea_row = ea_blk + tm * S::BM + arow;
    const int16_t* eb_col = eb_blk + tn * S::BN + half * 64;
    for (int d = 0; d < ndr; ++d) {
      const int b = d & 1;
      const int64_t blk = b0 + d;
      const int da = (int)ea_row[blk * kp] - egs[arow];
      if (!warp_wait(&accf[b], (uint32_t)(d >> 1) & 1u)) {
        ok = false;
        break;
      }
      umma::fence_after_sync();
      const uint32_t ta = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(b * 256 + half * 64);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        uint32_t v[8], w[8];
        umma::tmem_ld_32x32b_x8(ta + c * 8, v);
        umma::tmem_ld_32x32b_x8(ta + S::BN + c * 8, w);
        const uint4 e8 = __ldg(reinterpret_cast<const uint4*>(eb_col + blk * kp + c * 8));
        umma::tmem_wait_ld();
        if (c == 7) {
          // the buffer is free for the next MMAs once its last columns are read
          umma::fence_before_sync();
          __syncwarp();
          if (lane == 0) umma::mbar_arrive(&acce[b]);
        }
        const uint32_t ew[4] = {e8.x, e8.y, e8.z, e8.w};
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int eb = (int)(int16_t)(ew[e >> 1] >> (16 * (e & 1)));
          // 2^x for x = min(da + db, 0) (padding columns: zero products), 0 below 2^-126
          const int x = min(da + eb - egs[128 + half * 64 + c * 8 + e], 0);
          const float sc = x < -126 ? 0.0f : __int_as_float((127 + x) << 23);
          const df t = df_two_sum(hi[c * 8 + e], __uint_as_float(v[e]) * sc);
          hi[c * 8 + e] = t.hi;
          lo[c * 8 + e] += t.lo + __uint_as_float(w[e]) * sc;
        }
      }
    }
    // the tile through shared memory (the stages are idle once the last
    // buffer has been filled), then out to global memory row by row,
    // coalesced.  If any drain warp's wait ran out, loads or MMAs may still
    // be using the stages: the eight warps agree on that first and then skip
    // the staging and the store (the call reports VST_ETIMEOUT).
    if (!ok && lane == 0) *drain_fail = 1u;
    asm volatile("bar.sync 1, 256;" ::: "memory");  // the eight drain warps
    if (*drain_fail == 0u) {
      double* tsm = reinterpret_cast<double*>(gbase);
      const int r = q4 * 32 + lane;
#pragma unroll
      for (int c = 0; c < 64; ++c) tsm[r * (S::BN + 1) + half * 64 + c] = (double)hi[c] + (double)lo[c];
      asm volatile("bar.sync 1, 256;" ::: "memory");
      double* dst = out + (int64_t)seg * kc * kc;
      for (int e = threadIdx.x - 128; e < S::BM * S::BN; e += 256) {
        const int a = tm * S::BM + e / S::BN, bc = tn * S::BN + e % S::BN;
        if (a < kc && bc < kc) dst[(int64_t)a * kc + bc] = tsm[(e / S::BN) * (S::BN + 1) + e % S::BN];
      }
    }
  }
  if (!ok) report_error(hdr, VST_ETIMEOUT, (int64_t)blockIdx.x);
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tmem, 512);
}

// C[a][b] = 2^(Eg_a + Eg_b - 16) times the sum of the nseg FP64 partials
// (fixed order), Eg the columns' largest exponents (biased); sym: only
// b <= a was computed, mirrored into both triangles
__global__ void gram_sum_kernel(const double* part, int nseg, int kc, const int* ea, const int* eb, int sym,
                                double* C) {
  const int64_t kk = (int64_t)kc * kc;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < kk; id += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(id / kc), b = (int)(id % kc);
    if (sym && b > a) continue;
    double s = 0.0;
    for (int q = 0; q < nseg; ++q) s += part[q * kk + id];
    s = ldexp(s, ea[a] + eb[b] - 2 * kFxBias - 16);
    C[id] = s;
    if (sym) C[(int64_t)b * kc + a] = s;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2-D BF16 tensor map: rows x cols (cols contiguous), box 64 x box_rows, 128-byte swizzle
bool make_map(CUtensorMap* map, const void* ptr, uint64_t rows, uint64_t cols, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols * 2};
  const cuuint32_t box[2] = {64, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// r_i = sigma1^2 - sum_t part[i][t] over the GEMM's column tiles, in a fixed order
__global__ void rsum_kernel(const double* part, int64_t n, int nt, double s1, double* r) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < nt; ++q) s += part[i * nt + q];
    r[i] = s1 - s;
  }
}

template <int P, int BN, int STAGES>
cudaError_t launch_gemm(const __nv_bfloat16* A, const __nv_bfloat16* B, int64_t n, int k, int kp, float* U,
                        double* rpart, double s1, double* r, WsHeader* hdr, cudaStream_t st, bool* map_ok) {
  using S = TcShape<P, BN, STAGES>;
  CUtensorMap ta, tb;
  *map_ok = make_map(&ta, A, (uint64_t)P * n, (uint64_t)kp, S::BM) &&
            make_map(&tb, B, (uint64_t)P * kp, (uint64_t)kp, BN);
  if (!*map_ok) return cudaSuccess;
  auto kern = ugemm_tc_kernel<P, BN, STAGES>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (n + S::BM - 1) / S::BM * (kp / BN);
  if (tiles > 0x7fffffff) return cudaErrorInvalidConfiguration;
  const dim3 grid((unsigned)tiles);
  {
    ProfileScope ps(kProfVifGemm, st);
    kern<<<grid, 128, S::SMEM, st>>>(ta, tb, n, k, kp, U, rpart, hdr);
  }
  rsum_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 65535), 256, 0, st>>>(rpart, n, kp / BN, s1, r);
  return cudaGetLastError();
}

// C[i][c] = sum_p A[i][p] B[c][p] on the tensor cores (FP32 out [n][k]);
// bmode 1: B = M (full), bmode 2: B[c][p] = M[p][c], M lower triangular
template <int P, int BN, int KMODE>
vst_status tc_product_P(const float* A, int64_t lda, int64_t n, const double* M, int k, float* C, char* vbase,
                        const VifLayout& V, WsHeader* hdr, cudaStream_t st) {
  using S = TcShape<P, BN, 2>;
  const int kp = vif_kp(k);
  __nv_bfloat16* Ap = reinterpret_cast<__nv_bfloat16*>(vbase + V.Ap);
  __nv_bfloat16* Bp = reinterpret_cast<__nv_bfloat16*>(vbase + V.Bp);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::max(1, sms) * 8;
  split_a_kernel<P><<<grid, 256, 0, st>>>(A, lda, n, k, kp, Ap);
  split_b_kernel<P><<<grid, 256, 0, st>>>(M, k, kp, KMODE, Bp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "split kernels");
  CUtensorMap ta, tb;
  if (!make_map(&ta, Ap, (uint64_t)P * n, (uint64_t)kp, S::BM) || !make_map(&tb, Bp, (uint64_t)P * kp, (uint64_t)kp, BN))
    return fail(VST_ECUDA, "cuTensorMapEncodeTiled unavailable or rejected the operand layout");
  auto kern = ugemm_tc_kernel<P, BN, 2, KMODE, false>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core product attributes");
  const int64_t tiles = (n + S::BM - 1) / S::BM * (kp / BN);
  if (tiles > 0x7fffffff) return fail(VST_EINVAL, "too many tiles");
  kern<<<(unsigned)tiles, 128, S::SMEM, st>>>(ta, tb, n, k, kp, C, nullptr, hdr);
  e = cudaGetLastError();
  return e == cudaSuccess ? VST_OK : cuda_fail(e, "tensor-core product");
}

// segments of K for a grid of ntiles tiles: the count in 1..kGramMaxSeg
// (at most one per 128-row block) whose CTAs fill the SMs' waves best, the
// smallest such count on ties
int gram_nseg(int ntiles, int64_t kbt, int sms) {
  int best = 1;
  double best_eff = -1.0;
  for (int s = 1; s <= kGramMaxSeg && s <= kbt; ++s) {
    const int64_t c = (int64_t)ntiles * s;
    const int64_t waves = (c + sms - 1) / sms;
    const double eff = (double)c / (double)(waves * sms);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = s;
    }
  }
  return best;
}

// B == nullptr: the symmetric C = A^T A (one operand, the lower triangle of
// tiles, mirrored by the sum).  opa, opb: the operands' regions
// (tc_operand_bytes each; opb unused when symmetric).
template <int P, int STAGES>
vst_status tc_gram_P(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t n, int kc, double* C,
                     char* opa, char* opb, double* part, WsHeader* hdr, cudaStream_t st) {
  using S = GramTcShape<P, STAGES>;
  const bool sym = B == nullptr;
  const int kp = vif_kp(kc);
  const int64_t np = (n + 127) / 128 * 128;
  const FxOperand oa = fx_operand(opa, n, kc);
  const FxOperand ob = sym ? oa : fx_operand(opb, n, kc);
  const dim3 tgrid((unsigned)(np / 128), (unsigned)(kp / 64));
  if (np / 128 > 0x7fffffff) return fail(VST_EINVAL, "too many rows");
  cudaError_t e = cudaMemsetAsync(oa.eg, 0, sizeof(int) * kp, st);
  if (e == cudaSuccess && !sym) e = cudaMemsetAsync(ob.eg, 0, sizeof(int) * kp, st);
  if (e != cudaSuccess) return cuda_fail(e, "column exponents");
  split_fx_t_kernel<P><<<tgrid, 256, 0, st>>>(A, lda, n, kc, kp, np, oa.parts, oa.eblk, oa.eg);
  if (!sym) split_fx_t_kernel<P><<<tgrid, 256, 0, st>>>(B, ldb, n, kc, kp, np, ob.parts, ob.eblk, ob.eg);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "transposed split kernels");
  CUtensorMap ta, tb;
  if (!make_map(&ta, oa.parts, (uint64_t)P * kp, (uint64_t)np, S::BM) ||
      !make_map(&tb, ob.parts, (uint64_t)P * kp, (uint64_t)np, S::BN))
    return fail(VST_ECUDA, "cuTensorMapEncodeTiled unavailable or rejected the operand layout");
  auto kern = gram_tc_kernel<P, STAGES>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core Gram attributes");
  // the draining warpgroups' register increase is served from the registers
  // the block launches with: refuse a build whose launch count is too small
  cudaFuncAttributes fa{};
  e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core Gram attributes");
  if ((int64_t)fa.numRegs * S::THREADS < 128 * S::REGS_LOW + 256 * S::REGS_HIGH)
    return fail(VST_EINTERNAL, "tensor-core Gram: %d registers per thread at launch do not cover the split",
                fa.numRegs);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int T = kp / S::BM;
  const int ntiles = sym ? T * (T + 1) / 2 : T * T;
  const int nseg = gram_nseg(ntiles, np / 128, std::max(1, sms));
  kern<<<(unsigned)(ntiles * nseg), S::THREADS, S::SMEM, st>>>(ta, tb, np, kc, kp, nseg, sym ? 1 : 0, oa.eblk, oa.eg,
                                                               ob.eblk, ob.eg, part, hdr);
  const int64_t kk = (int64_t)kc * kc;
  gram_sum_kernel<<<(unsigned)std::min<int64_t>((kk + 255) / 256, 8192), 256, 0, st>>>(part, nseg, kc, oa.eg, ob.eg,
                                                                                       sym ? 1 : 0, C);
  e = cudaGetLastError();
  return e == cudaSuccess ? VST_OK : cuda_fail(e, "tensor-core Gram");
}

template <int P>
vst_status lowrank_tc_P(const vst_points* pts, const vst_theta* theta, const vst_inducing* ind, int nu,
                        char* vbase, const VifLayout& V, WsHeader* hdr, cudaStream_t st) {
  const int64_t n = pts->n;
  const int k = (int)ind->k, kp = vif_kp(k);
  const DevTheta th = dev_theta_vif(theta);
  const double* X = reinterpret_cast<const double*>(vbase + V.X);
  const int64_t* dinfo = reinterpret_cast<const int64_t*>(vbase + V.dinfo);
  const float2* dtab = reinterpret_cast<const float2*>(vbase + V.dtab);
  __nv_bfloat16* Ap = reinterpret_cast<__nv_bfloat16*>(vbase + V.Ap);
  __nv_bfloat16* Bp = reinterpret_cast<__nv_bfloat16*>(vbase + V.Bp);
  float4* zf = reinterpret_cast<float4*>(vbase + V.zf);
  float* U = reinterpret_cast<float*>(vbase + V.U);
  double* rpart = reinterpret_cast<double*>(vbase + V.rpart);
  double* r = reinterpret_cast<double*>(vbase + V.r);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::max(1, sms) * 8;
  split_x_kernel<P><<<grid, 256, 0, st>>>(X, k, kp, Bp);
  ind_coords_kernel<<<(k + 127) / 128, 128, 0, st>>>(ind->xy, k, zf);
  if (nu == 0)
    snk_split_kernel<0, P><<<grid, 256, 0, st>>>(pts->xy, pts->t, n, ind->xy, ind->t, zf, k, kp, th, dinfo, dtab, Ap);
  else if (nu == 1)
    snk_split_kernel<1, P><<<grid, 256, 0, st>>>(pts->xy, pts->t, n, ind->xy, ind->t, zf, k, kp, th, dinfo, dtab, Ap);
  else
    snk_split_kernel<2, P><<<grid, 256, 0, st>>>(pts->xy, pts->t, n, ind->xy, ind->t, zf, k, kp, th, dinfo, dtab, Ap);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "split kernels");
  bool map_ok = true;
  // two parts: 128 x 256 tiles; three parts: 128 x 128 tiles (two stages fit either way)
  if constexpr (P == 2) e = launch_gemm<2, 256, 2>(Ap, Bp, n, k, kp, U, rpart, theta->sigma1sq, r, hdr, st, &map_ok);
  else e = launch_gemm<3, 128, 2>(Ap, Bp, n, k, kp, U, rpart, theta->sigma1sq, r, hdr, st, &map_ok);
  if (!map_ok) return fail(VST_ECUDA, "cuTensorMapEncodeTiled unavailable or rejected the operand layout");
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core U GEMM");
  return VST_OK;
}

}  // namespace

// C = A B^T-shaped products of the mixed VIF gradient on the tensor cores:
// C[i][c] = sum_p A[i][p] B[c][p], A FP32 [n][k] (row stride lda), B from the
// FP64 k x k matrix M (bmode 1: M itself; 2: M^T of a lower-triangular M),
// split_terms = 3 or 6 as in the mixed NLL.  Uses the NLL's operand-part
// buffers, free once U is formed.
bool tc_make_map_bf16(CUtensorMap* map, const void* ptr, uint64_t rows, uint64_t cols, uint32_t box_rows) {
  return make_map(map, ptr, rows, cols, box_rows);
}

vst_status tc_product(const float* A, int64_t lda, int64_t n, const double* M, int bmode, int k, float* C,
                      int split_terms, char* vbase, const VifLayout& V, WsHeader* hdr, cudaStream_t st) {
  if (n <= 0) return VST_OK;
  if (bmode != 1 && bmode != 2) return fail(VST_EINVAL, "bad operand mode %d", bmode);
  if (split_terms == 3)
    return bmode == 1 ? tc_product_P<2, 256, 1>(A, lda, n, M, k, C, vbase, V, hdr, st)
                      : tc_product_P<2, 256, 2>(A, lda, n, M, k, C, vbase, V, hdr, st);
  return bmode == 1 ? tc_product_P<3, 128, 1>(A, lda, n, M, k, C, vbase, V, hdr, st)
                    : tc_product_P<3, 128, 2>(A, lda, n, M, k, C, vbase, V, hdr, st);
}

// FP64 partials of tc_gram / tc_syrk: up to kGramMaxSeg kc x kc segments
size_t tc_gram_part_bytes(int64_t kc) { return (size_t)8 * kGramMaxSeg * kc * kc; }

// C = A^T B (FP64 kc x kc) for FP32 A, B [n][kc] (row strides lda, ldb) on
// the tensor cores: transposed fixed-point parts, split-K tiles over the
// 128-row blocks with double-float drains of the tensor-memory accumulators,
// segments summed in FP64 in a fixed order.  opa, opb: tc_operand_bytes(n,
// kc) bytes each; part: tc_gram_part_bytes(kc) bytes.
vst_status tc_gram(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t n, int kc, double* C,
                   void* opa, void* opb, double* part, WsHeader* hdr, cudaStream_t st) {
  if (kc <= 0) return VST_OK;
  if (n <= 0) return cudaMemsetAsync(C, 0, sizeof(double) * kc * kc, st) == cudaSuccess ? VST_OK : VST_ECUDA;
  return tc_gram_P<3, 2>(A, lda, B, ldb, n, kc, C, static_cast<char*>(opa), static_cast<char*>(opb), part, hdr, st);
}

// C = A^T A (FP64 kc x kc, both triangles) for FP32 A [n][kc] (row stride
// lda): tc_gram's product on the lower triangle of tiles.  opa:
// tc_operand_bytes(n, kc) bytes; part: tc_gram_part_bytes(kc) bytes.
vst_status tc_syrk(const float* A, int64_t lda, int64_t n, int kc, double* C, void* opa, double* part,
                   WsHeader* hdr, cudaStream_t st) {
  if (kc <= 0) return VST_OK;
  if (n <= 0) return cudaMemsetAsync(C, 0, sizeof(double) * kc * kc, st) == cudaSuccess ? VST_OK : VST_ECUDA;
  return tc_gram_P<3, 2>(A, lda, nullptr, 0, n, kc, C, static_cast<char*>(opa), nullptr, part, hdr, st);
}

// U (FP32, [n][k]) of the mixed form on the tensor cores; split_terms = 3 or 6.
// Needs X = L^{-1}, the day range and the day lag table already in place.
vst_status lowrank_tc(const vst_points* pts, const vst_theta* theta, const vst_inducing* ind, int nu,
                      int split_terms, char* vbase, const VifLayout& V, WsHeader* hdr, cudaStream_t st) {
  if (pts->n <= 0) return VST_OK;
  return split_terms == 3 ? lowrank_tc_P<2>(pts, theta, ind, nu, vbase, V, hdr, st)
                          : lowrank_tc_P<3>(pts, theta, ind, nu, vbase, V, hdr, st);
}

}  // namespace vst

using namespace vst;

// workspace: the status header, the two operands' regions, the partials
extern "C" size_t vst_workspace_size_gram_tc(int64_t n, int kc) {
  if (n < 0 || kc <= 0) return 0;
  return 256 + 2 * tc_operand_bytes(n, kc) + align256(tc_gram_part_bytes(kc));
}

extern "C" vst_status vif_gram_tc(int64_t n, int kc, const float* A, int64_t lda, const float* B, int64_t ldb,
                                  double* C, void* ws, size_t ws_bytes, void* stream) {
  if (n < 0 || n >= (int64_t(1) << 31)) return fail(VST_EINVAL, "n=%lld out of range", (long long)n);
  if (kc <= 0 || kc > 16384) return fail(VST_EINVAL, "kc=%d out of range (1..16384)", kc);
  if (!C || (n > 0 && !A)) return fail(VST_EINVAL, "NULL array");
  if (lda < kc || (B && ldb < kc)) return fail(VST_EINVAL, "row strides below kc");
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256) return fail(VST_EINVAL, "workspace NULL or not 256-byte aligned");
  const size_t need = vst_workspace_size_gram_tc(n, kc);
  if (ws_bytes < need) return fail(VST_ENOMEM, "workspace has %zu bytes, %zu needed", ws_bytes, need);
  cudaStream_t st = (cudaStream_t)stream;
  char* base = static_cast<char*>(ws);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(base);
  launch_init_header(hdr, st);
  char* opa = base + 256;
  char* opb = opa + tc_operand_bytes(n, kc);
  double* part = reinterpret_cast<double*>(opb + tc_operand_bytes(n, kc));
  return B ? tc_gram(A, lda, B, ldb, n, kc, C, opa, opb, part, hdr, st) : tc_syrk(A, lda, n, kc, C, opa, part, hdr, st);
}
