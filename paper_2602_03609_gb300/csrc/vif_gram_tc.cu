// The mixed VIF's per-row residual Gram on the tensor cores (Sect. 4.3: the
// residual covariance C - U U^T of each local block): for row i and the
// positions p, q of its block (its neighbours, unused positions, and i
// itself at the last position L), gram[i][pair(p, q)] = U_p . U_q, for local
// blocks of 32 positions.
//
// usplit_kernel cuts every row of U once into three 9-bit fixed-point BF16
// parts per 64-column chunk: with E the exponent of the chunk's largest
// |U|, x = U 2^(8 - E) = s_0 + 2^-9 s_1 + 2^-18 s_2 + (below 2^-19), integers
// |s_j| <= 256 exact in BF16 (as the contractions over the points in
// vif_tc.cu); the parts go to [3][n][kp] and 2^(E - 8) to uscale[row][chunk].
//
// gram_tc_rows_kernel: four rows make one 128-row MMA operand (row 32 b + p =
// position p of row b); their blocks S = V V^T are the diagonal 32 x 32
// blocks of the 128 x 128 product, the rest is computed and not read.  Per
// chunk the leading part products are integers below 2^16 and the chunk's
// sum of 64 an integer below 2^22, exact in the FP32 accumulator whatever its
// rounding; the correction products go to a second accumulator.  Each chunk
// is drained on its own: the diagonal blocks are scaled by
// 2^(E_p + E_q - 16) (exact) and added to double-float sums in registers.
// (The SIMT kernel for other block sizes, gram_delta_kernel in vif.cu, works
// around the row's own vector, U_p - U_i; on the tensor cores the exponent
// per row and chunk keeps the direct form's error at |dNLL|/n ~1e-8 on the
// bench workload, with no bias.)
//
// CTA of 13 warps, persistent over groups of four rows:
//   warps 0-7  copy: warp w takes every other chunk (w / 4 the chunk parity);
//              eight lanes copy one position's 128-byte row of a part, 16
//              rows a pass, into a shared-memory stage in the 128-byte-
//              swizzled K-major layout the MMA reads, with the rows' scales
//   warps 8-11 drain TMEM lanes 32 b.. (row b = warp % 4) after each chunk;
//              at the end of a group they write gram[i][pair]
//   warp 12    TMEM allocation, tcgen05.mma issue (one lane), commits
// Stages are handed over with mbarriers (copiers -> MMA: full, count 4;
// MMA -> copiers: empty, by commit; MMA -> drains: accf, by commit;
// drains -> MMA: acce, count 4).  Every wait is limited in time; a wait that
// runs out reports VST_ETIMEOUT and the CTA still frees its tensor memory.
#include <cuda_bf16.h>

#include "kernels.h"
#include "umma.cuh"
#include "vif.h"

namespace vst {

vst_status fail(vst_status s, const char* fmt, ...);
vst_status cuda_fail(cudaError_t e, const char* where);

namespace {

constexpr int kGP = 32;                 // positions per row (PM)
constexpr int kGL = kGP - 1;            // the row's own position
constexpr int kGRows = 4;               // rows per group (MMA M = 128)
constexpr int kGKc = 64;                // columns per chunk
constexpr int kGStages = 3;
constexpr int kGPartBytes = 128 * kGKc * 2;        // one part of one stage: 128 rows x 128 bytes
constexpr int kGStageBytes = 3 * kGPartBytes;      // 49,152
constexpr int kGExpSlots = 8;                      // scale-factor ring (> stages + 2)
constexpr int kGSStride = kGP + 1;
constexpr int kGThreads = 416;
constexpr uint64_t kGWaitNs = 2000000000ull;
constexpr int kGSmem = kGStages * kGStageBytes + kGExpSlots * 128 * 4 + kGRows * kGP * kGSStride * 4 + 256 + 1024;
static_assert(kGSmem <= 232448, "shared memory");
static_assert(64 * 65536 <= (1 << 23), "a chunk's leading sum stays exact in FP32");

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// E with |x| < 2^E for the values whose largest magnitude has the biased
// FP32 exponent eb, clamped below at -100 so that 2^(8 - E) is a normal FP32
// value (smaller values keep less precision)
__device__ __forceinline__ int gexp_b(unsigned eb) {
  const int E = (int)eb - 126;
  return E < -100 ? -100 : E;
}

__device__ __forceinline__ float2 fsub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// three fixed-point parts of a packed pair x = v 2^(8 - E), |x| < 256:
// p0 = rint(x), p1 = the rest rounded to a multiple of 2^-9, p2 = what is
// left rounded to a multiple of 2^-18 (round to nearest even by adding and
// subtracting 1.5 2^23 at the grid's scale; the differences are exact)
__device__ __forceinline__ void gsplit2(float2 x, uint32_t& w0, uint32_t& w1, uint32_t& w2) {
  const float2 M0 = make_float2(12582912.0f, 12582912.0f);  // 1.5 2^23: unit grid
  const float2 M1 = make_float2(24576.0f, 24576.0f);        // 1.5 2^14: grid 2^-9
  const float2 M2 = make_float2(48.0f, 48.0f);              // 1.5 2^5:  grid 2^-18
  const float2 p0 = fsub2(__fadd2_rn(x, M0), M0);
  const float2 y = fsub2(x, p0);
  const float2 p1 = fsub2(__fadd2_rn(y, M1), M1);
  const float2 y2 = fsub2(y, p1);
  const float2 p2 = fsub2(__fadd2_rn(y2, M2), M2);
  const __nv_bfloat162 b0 = __floats2bfloat162_rn(p0.x, p0.y);  // each part exact in BF16
  const __nv_bfloat162 b1 = __floats2bfloat162_rn(p1.x, p1.y);
  const __nv_bfloat162 b2 = __floats2bfloat162_rn(p2.x, p2.y);
  w0 = *reinterpret_cast<const uint32_t*>(&b0);
  w1 = *reinterpret_cast<const uint32_t*>(&b1);
  w2 = *reinterpret_cast<const uint32_t*>(&b2);
}

// parts [3][n][kp] (BF16) and scales uscale[n][nchunk] of U [n][k]: one warp
// per row, lane l holds columns 2 l, 2 l + 1 of each 64-column chunk
__global__ void __launch_bounds__(256) usplit_kernel(const float* U, int64_t n, int k, int kp, int nchunk,
                                                     __nv_bfloat16* parts, float* uscale) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const bool vec = (k & 1) == 0;
  const int64_t pstride = n * (int64_t)kp;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    const float* u = U + i * (int64_t)k;
    for (int c = 0; c < nchunk; ++c) {
      const int col = c * kGKc + 2 * lane;
      float2 v = make_float2(0.f, 0.f);
      if (vec && col + 2 <= k) v = __ldg(reinterpret_cast<const float2*>(u + col));
      else {
        if (col < k) v.x = __ldg(u + col);
        if (col + 1 < k) v.y = __ldg(u + col + 1);
      }
      const unsigned mb = __reduce_max_sync(0xffffffffu, __float_as_uint(fmaxf(fabsf(v.x), fabsf(v.y))));
      const int E = gexp_b(mb >> 23);
      const float scale = __int_as_float((127 + 8 - E) << 23);
      uint32_t w0, w1, w2;
      gsplit2(__fmul2_rn(v, make_float2(scale, scale)), w0, w1, w2);
      uint32_t* dst = reinterpret_cast<uint32_t*>(parts + i * (int64_t)kp + col);
      dst[0] = w0;
      dst[pstride / 2] = w1;
      dst[pstride] = w2;
      if (lane == 0) uscale[i * nchunk + c] = __int_as_float((127 + E - 8) << 23);
    }
  }
}

// the six kept part products (a, b): (0,0) leading; (0,1) (1,0) (0,2) (1,1) (2,0)
__device__ __forceinline__ int gpa(int t) { return t == 2 ? 1 : t == 4 ? 1 : t == 5 ? 2 : 0; }
__device__ __forceinline__ int gpb(int t) { return t == 1 ? 1 : t == 3 ? 2 : t == 4 ? 1 : 0; }

__global__ void __launch_bounds__(kGThreads, 1)
    gram_tc_rows_kernel(const int32_t* nn, const int32_t* nn_cnt, int64_t n, int m, int k, int kp,
                        const __nv_bfloat16* parts, const float* uscale, float* gram, WsHeader* hdr) {
  extern __shared__ unsigned char g_smem[];
  const uint32_t raw = umma::smem_u32(g_smem);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  unsigned char* gb = g_smem + (sbase - raw);
  float* sfac = reinterpret_cast<float*>(gb + kGStages * kGStageBytes);  // [slot][128]: 2^(E - 8)
  float* Ssm = sfac + kGExpSlots * 128;                                      // [4][32][33]
  uint64_t* full = reinterpret_cast<uint64_t*>(Ssm + kGRows * kGP * kGSStride);
  uint64_t* empty = full + kGStages;
  uint64_t* accf = empty + kGStages;  // [2]
  uint64_t* acce = accf + 2;          // [2]
  uint64_t* done = acce + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ngroups = (n + kGRows - 1) / kGRows;
  const int nchunk = (k + kGKc - 1) / kGKc;
  const int64_t ng_cta = blockIdx.x < ngroups ? (ngroups - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t nt = ng_cta * nchunk;  // chunks this CTA processes

  if (threadIdx.x == 0) {
    for (int s = 0; s < kGStages; ++s) {
      umma::mbar_init(&full[s], 4);
      umma::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      umma::mbar_init(&accf[b], 1);
      umma::mbar_init(&acce[b], 4);
    }
    umma::mbar_init(done, 1);
    umma::fence_mbar_init();
  }
  if (warp == 12) {
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
    if (lane == 0) d = umma::mbar_wait(bar, parity, kGWaitNs);
    return __shfl_sync(0xffffffffu, d ? 1 : 0, 0) != 0;
  };

  if (warp < 8) {
    // ---- copiers: chunks t with t % 2 = warp / 4; set lane L = 32 (warp % 4)
    // + lane copies 16 bytes (unit L % 8) of rows 16 pass + L / 8, pass 0..7:
    // positions L / 8 and 16 + L / 8 of the four rows of the group
    const int par = warp >> 2;
    const int L = 32 * (warp & 3) + lane;
    const int unit = L & 7, rsub = L >> 3;
    const int64_t pstride = n * (int64_t)kp;
    int64_t cur_g = -1;
    int ridx[8];  // U row of tile row 16 pass + rsub (-1: zeros)
    for (int64_t t = par; t < nt; t += 2) {
      const int64_t gi = t / nchunk;
      const int c = (int)(t % nchunk);
      if (gi != cur_g) {
        cur_g = gi;
#pragma unroll
        for (int ps = 0; ps < 8; ++ps) {
          const int row = 16 * ps + rsub;
          const int b = row >> 5, pos = row & 31;
          const int64_t i = (blockIdx.x + gi * gridDim.x) * kGRows + b;
          int v = -1;
          if (i < n) {
            if (pos == kGL) {
              v = (int)i;
            } else {
              const int cnt = min(max(nn_cnt[i], 0), min(m, kGL));
              if (pos < cnt) v = nn[i * m + pos];
              if (v < 0 || v > i) v = -1;
            }
          }
          ridx[ps] = v;
        }
      }
      const int s = (int)(t % kGStages);
      const uint32_t use = (uint32_t)(t / kGStages);
      if (use > 0 && !warp_wait(&empty[s], (use - 1) & 1u)) {
        ok = false;
        break;
      }
      unsigned char* st = gb + s * kGStageBytes;
      const int slot = (int)(t % kGExpSlots);
      const int col = c * kGKc + 8 * unit;
      // all 24 loads of the lane (and the rows' scales) in flight before the stores
      uint4 d[3][8];
      float sc[8];
#pragma unroll
      for (int ps = 0; ps < 8; ++ps)
        sc[ps] = (unit == 0 && ridx[ps] >= 0) ? __ldg(uscale + (int64_t)ridx[ps] * nchunk + c) : 0.0f;
#pragma unroll
      for (int ps = 0; ps < 8; ++ps) {
        const __nv_bfloat16* src = parts + (int64_t)(ridx[ps] >= 0 ? ridx[ps] : 0) * kp + col;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          d[j][ps] = make_uint4(0u, 0u, 0u, 0u);
          if (ridx[ps] >= 0) d[j][ps] = __ldg(reinterpret_cast<const uint4*>(src + j * pstride));
        }
      }
#pragma unroll
      for (int ps = 0; ps < 8; ++ps) {
        const int row = 16 * ps + rsub;
        unsigned char* dst = st + (row >> 3) * 1024 + (row & 7) * 128 + ((unit ^ (row & 7)) << 4);
#pragma unroll
        for (int j = 0; j < 3; ++j) *reinterpret_cast<uint4*>(dst + j * kGPartBytes) = d[j][ps];
      }
      if (unit == 0) {
#pragma unroll
        for (int ps = 0; ps < 8; ++ps) sfac[slot * 128 + 16 * ps + rsub] = sc[ps];
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) umma::mbar_arrive(&full[s]);
    }
  } else if (warp < 12) {
    // ---- drains: row b = warp % 4 of each group, TMEM lanes 32 b ..
    const int b = warp & 3;
    float hi[kGP], lo[kGP];
    int64_t t = 0;
    for (int64_t gi = 0; gi < ng_cta && ok; ++gi) {
#pragma unroll
      for (int q = 0; q < kGP; ++q) hi[q] = lo[q] = 0.f;
      for (int c = 0; c < nchunk; ++c, ++t) {
        const int buf = (int)(t & 1);
        const uint32_t buse = (uint32_t)(t >> 1);
        if (!warp_wait(&accf[buf], buse & 1u)) {
          ok = false;
          break;
        }
        umma::fence_after_sync();
        const uint32_t ta = tmem + ((uint32_t)(b * 32) << 16) + (uint32_t)(buf * 256 + b * 32);
        const float* sf = sfac + (int)(t % kGExpSlots) * 128 + 32 * b;
        const float sp = sf[lane];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t mv[16], cv[16];
          umma::tmem_ld_32x32b_x16(ta + 16 * h, mv);
          umma::tmem_ld_32x32b_x16(ta + 128 + 16 * h, cv);
          umma::tmem_wait_ld();
          if (h == 1) {
            umma::fence_before_sync();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&acce[buf]);
          }
          const float2 sp2 = make_float2(sp, sp);
#pragma unroll
          for (int q4 = 0; q4 < 4; ++q4) {
            const float4 sq = *reinterpret_cast<const float4*>(sf + 16 * h + 4 * q4);
            const float2 sqv[2] = {make_float2(sq.x, sq.y), make_float2(sq.z, sq.w)};
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const int q = 16 * h + 4 * q4 + 2 * e;
              // 2^(E_p + E_q - 16), exact unless it leaves the FP32 range
              const float2 sc = __fmul2_rn(sp2, sqv[e]);
              const float2 mm = __fmul2_rn(make_float2(__uint_as_float(mv[4 * q4 + 2 * e]),
                                                       __uint_as_float(mv[4 * q4 + 2 * e + 1])), sc);
              const float2 cc = make_float2(__uint_as_float(cv[4 * q4 + 2 * e]), __uint_as_float(cv[4 * q4 + 2 * e + 1]));
              // two-sum of (hi, mm) on packed pairs
              const float2 h2 = make_float2(hi[q], hi[q + 1]);
              const float2 sm = __fadd2_rn(h2, mm);
              const float2 bb = fsub2(sm, h2);
              const float2 er = __fadd2_rn(fsub2(h2, fsub2(sm, bb)), fsub2(mm, bb));
              const float2 l2 = __fadd2_rn(make_float2(lo[q], lo[q + 1]), __ffma2_rn(cc, sc, er));
              hi[q] = sm.x;
              hi[q + 1] = sm.y;
              lo[q] = l2.x;
              lo[q + 1] = l2.y;
            }
          }
        }
      }
      if (!ok) break;
      // S of this row, then the E-step
      const int64_t i = (blockIdx.x + gi * gridDim.x) * kGRows + b;
      float* S = Ssm + b * kGP * kGSStride;
#pragma unroll
      for (int q = 0; q < kGP; ++q) S[lane * kGSStride + q] = hi[q] + lo[q];
      __syncwarp();
      if (i < n) {
        constexpr int NPAIR = kGP * (kGP + 1) / 2;
        for (int e = lane; e < NPAIR; e += 32) {
          int pa, pb;
          pair_of<kGP>(e, pa, pb);  // pa >= pb
          gram[i * NPAIR + e] = S[pa * kGSStride + pb];
        }
      }
      __syncwarp();
    }
  } else {
    // ---- MMA issue (warp 12)
    constexpr uint32_t idesc = umma::idesc_bf16_f32(128, 128);
    int64_t t = 0;
    for (; t < nt; ++t) {
      const int s = (int)(t % kGStages);
      const uint32_t use = (uint32_t)(t / kGStages);
      const int buf = (int)(t & 1);
      const uint32_t buse = (uint32_t)(t >> 1);
      if (!warp_wait(&full[s], use & 1u)) {
        ok = false;
        break;
      }
      if (buse > 0 && !warp_wait(&acce[buf], (buse - 1) & 1u)) {
        ok = false;
        break;
      }
      umma::fence_after_sync();
      if (lane == 0) {
        const uint32_t sa = sbase + s * kGStageBytes;
        const uint32_t tb = tmem + (uint32_t)(buf * 256);
#pragma unroll
        for (int kk = 0; kk < kGKc / 16; ++kk) {
#pragma unroll
          for (int q = 0; q < 6; ++q) {
            const uint64_t ad = umma::desc_kmajor_sw128(sa + gpa(q) * kGPartBytes + kk * 32);
            const uint64_t bd = umma::desc_kmajor_sw128(sa + gpb(q) * kGPartBytes + kk * 32);
            if (q == 0) umma::mma_bf16(tb, ad, bd, idesc, kk > 0 ? 1u : 0u);
            else umma::mma_bf16(tb + 128, ad, bd, idesc, (kk > 0 || q > 1) ? 1u : 0u);
          }
        }
        umma::mma_commit(&empty[s]);
        umma::mma_commit(&accf[buf]);
      }
      __syncwarp();
    }
    // every MMA this thread issued has finished before the tensor memory is freed
    if (lane == 0) umma::mma_commit(done);
    __syncwarp();
    if (!warp_wait(done, 0)) ok = false;
  }
  if (!ok) report_error(hdr, VST_ETIMEOUT, (int64_t)blockIdx.x);
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 12) umma::tmem_dealloc(tmem, 512);
}

}  // namespace

// gram[i][e] (FP32, [n][32 * 33 / 2]) of the mixed VIF for local blocks of 32
// positions (m + 1 <= 32 rounded up to 32), on the tensor cores.  parts:
// 3 n kp BF16 values (kp = k rounded up to 256); uscale: n ceil(k / 64) floats.
vst_status gram_tc_rows(const int32_t* nn, const int32_t* nn_cnt, int64_t n, int m, int k, const float* U,
                        __nv_bfloat16* parts, float* uscale, float* gram, WsHeader* hdr, cudaStream_t st) {
  if (n <= 0 || k <= 0) return VST_OK;
  const int kp = vif_kp(k);
  const int nchunk = (k + kGKc - 1) / kGKc;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  usplit_kernel<<<(unsigned)std::min<int64_t>((n + 7) / 8, (int64_t)std::max(1, sms) * 32), 256, 0, st>>>(
      U, n, k, kp, nchunk, parts, uscale);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "fixed-point split of U");
  e = cudaFuncSetAttribute(gram_tc_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kGSmem);
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core row Gram attributes");
  const int64_t ngroups = (n + kGRows - 1) / kGRows;
  const int grid = (int)std::min<int64_t>(ngroups, std::max(1, sms));
  gram_tc_rows_kernel<<<grid, kGThreads, kGSmem, st>>>(nn, nn_cnt, n, m, k, kp, parts, uscale, gram, hdr);
  e = cudaGetLastError();
  return e == cudaSuccess ? VST_OK : cuda_fail(e, "tensor-core row Gram");
}

}  // namespace vst
