// The mixed VIF's per-row residual Gram on the tensor cores (Sect. 4.3: the
// residual covariance C - U U^T of each local block).  For row i with
// positions p (its neighbours, unused positions, and i itself at the last
// position L), V_p = U_p - U_i for the neighbours and V_L = U_i; the block
// S = V V^T (32 x 32) gives
//   U_p . U_q = |U_i|^2 + w_p + w_q + S_pq,  w_p = S_Lp,  |U_i|^2 = sigma1^2 - r_i,
// formed in double-float and rounded once, as in the SIMT kernel
// (gram_delta_kernel, vif.cu), whose accumulation this replaces for PM = 32.
//
// Four rows make one 128-row MMA operand (row 32 b + p = position p of row
// b); S of the four rows are the diagonal 32 x 32 blocks of the 128 x 128
// product, the rest is computed and not read.  The columns (the k inducing
// points) go in chunks of 64.  Per chunk each position gets the exponent E
// of its largest |V| there and its 64 values become three 9-bit fixed-point
// BF16 parts of 2^(E - 8) (as the contractions over the points in
// vif_tc.cu): the leading part products are integers below 2^16, a chunk's
// sum of 64 an integer below 2^22, exact in the FP32 accumulator whatever
// its rounding.  The correction products go to a second accumulator.  Each
// chunk is drained on its own: the diagonal blocks are scaled by
// 2^(E_p + E_q - 16) (exact) and added to double-float sums in registers.
//
// CTA of 13 warps, persistent over groups of four rows:
//   warps 0-7  convert: warp w takes row w % 4 of every other chunk (w / 4
//              the chunk parity); each load instruction reads two of the 32
//              U rows 256 bytes at a time (coalesced), a position's maximum
//              is reduced over the 16 lanes holding it, and the parts go to
//              a shared-memory stage in the 128-byte-swizzled K-major
//              layout the MMA reads
//   warps 8-11 drain TMEM lanes 32 b.. (row b = warp % 4) after each chunk;
//              at the end of a group the E-step above, writing gram[i][pair]
//   warp 12    TMEM allocation, tcgen05.mma issue (one lane), commits
// Stages are handed over with mbarriers (converters -> MMA: full, count 4;
// MMA -> converters: empty, by commit; MMA -> drains: accf, by commit;
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

// the six kept part products (a, b): (0,0) leading; (0,1) (1,0) (0,2) (1,1) (2,0)
__device__ __forceinline__ int gpa(int t) { return t == 2 ? 1 : t == 4 ? 1 : t == 5 ? 2 : 0; }
__device__ __forceinline__ int gpb(int t) { return t == 1 ? 1 : t == 3 ? 2 : t == 4 ? 1 : 0; }

__global__ void __launch_bounds__(kGThreads, 1)
    gram_tc_rows_kernel(const int32_t* nn, const int32_t* nn_cnt, int64_t n, int m, int k, const float* U,
                        const double* r, double s1, float* gram, WsHeader* hdr) {
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
    // ---- converters: row b = warp % 4, chunks t with t % 2 = warp / 4.
    // Load instruction j reads positions 2 j (lanes 0-15) and 2 j + 1 (lanes
    // 16-31), four columns per lane; position p's maximum is reduced over its
    // 16 lanes.
    const int b = warp & 3, par = warp >> 2;
    const int half = lane >> 4, cl = lane & 15;  // position parity, column quad
    const bool vec = (k & 3) == 0;
    int64_t cur_g = -1;
    int myidx = -1;  // U row of position `lane` (-1: unused)
    int64_t i = 0;
    for (int64_t t = par; t < nt; t += 2) {
      const int64_t gi = t / nchunk;
      const int c = (int)(t % nchunk);
      if (gi != cur_g) {
        cur_g = gi;
        i = (blockIdx.x + gi * gridDim.x) * kGRows + b;
        myidx = -1;
        if (i < n) {
          const int cnt = min(max(nn_cnt[i], 0), min(m, kGL));
          if (lane < cnt) myidx = nn[i * m + lane];
          if (lane == kGL) myidx = (int)i;
          if (myidx < 0 || myidx > i) myidx = -1;
        }
      }
      const int s = (int)(t % kGStages);
      const uint32_t use = (uint32_t)(t / kGStages);
      if (use > 0 && !warp_wait(&empty[s], (use - 1) & 1u)) {
        ok = false;
        break;
      }
      const int col = c * kGKc + 4 * cl;
      // U_i at this lane's four columns (unused positions and the row's own
      // position subtract nothing)
      float4 ui = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i < n) {
        const float* pu = U + i * (int64_t)k + col;
        if (vec && col + 4 <= k) ui = __ldg(reinterpret_cast<const float4*>(pu));
        else if (col < k) {
          ui.x = __ldg(pu);
          if (col + 1 < k) ui.y = __ldg(pu + 1);
          if (col + 2 < k) ui.z = __ldg(pu + 2);
          if (col + 3 < k) ui.w = __ldg(pu + 3);
        }
      }
      unsigned char* st = gb + s * kGStageBytes;
      // all 16 loads of the chunk in flight before any is used
      float4 av[16];
      unsigned sub = 0u;  // bit j: position 2 j + half is a neighbour (V = U_p - U_i)
      const bool fast = vec && c * kGKc + kGKc <= k;  // the whole chunk inside the k columns
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int ridx = __shfl_sync(0xffffffffu, myidx, 2 * j + half);
        av[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ridx >= 0 && 2 * j + half != kGL) sub |= 1u << j;
        if (ridx >= 0) {
          const float* pa = U + (int64_t)ridx * k + col;
          if (fast) {
            av[j] = __ldg(reinterpret_cast<const float4*>(pa));
          } else if (col < k) {
            av[j].x = __ldg(pa);
            if (col + 1 < k) av[j].y = __ldg(pa + 1);
            if (col + 2 < k) av[j].z = __ldg(pa + 2);
            if (col + 3 < k) av[j].w = __ldg(pa + 3);
          }
        }
      }
      // V, and each position's largest magnitude as its biased exponent:
      // four positions per word (one byte each), reduced over the 16 lanes
      // of a position with per-byte maxima
      unsigned ebw[4] = {0u, 0u, 0u, 0u};
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        float4 a = av[j];
        if (sub & (1u << j)) {  // (unused positions stay zero, the row's own is U_i)
          const float2 d0 = fsub2(make_float2(a.x, a.y), make_float2(ui.x, ui.y));
          const float2 d1 = fsub2(make_float2(a.z, a.w), make_float2(ui.z, ui.w));
          a = make_float4(d0.x, d0.y, d1.x, d1.y);
          av[j] = a;
        }
        const float lm = fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w)));
        ebw[j >> 2] |= (__float_as_uint(lm) >> 23) << (8 * (j & 3));
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) ebw[q] = __vmaxu4(ebw[q], __shfl_xor_sync(0xffffffffu, ebw[q], o));
      const int slot = (int)(t % kGExpSlots);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int pos = 2 * j + half;
        const int E = gexp_b((ebw[j >> 2] >> (8 * (j & 3))) & 0xffu);
        const float scale = __int_as_float((127 + 8 - E) << 23);
        const float2 sc2 = make_float2(scale, scale);
        uint2 o0, o1, o2;
        gsplit2(__fmul2_rn(make_float2(av[j].x, av[j].y), sc2), o0.x, o1.x, o2.x);
        gsplit2(__fmul2_rn(make_float2(av[j].z, av[j].w), sc2), o0.y, o1.y, o2.y);
        const int row = 32 * b + pos;
        // this lane's 8 bytes: 16-byte chunk cl / 2 of the row, half cl % 2
        const int off = (row >> 3) * 1024 + (row & 7) * 128 + (((cl >> 1) ^ (row & 7)) << 4) + ((cl & 1) << 3);
        *reinterpret_cast<uint2*>(st + off) = o0;
        *reinterpret_cast<uint2*>(st + kGPartBytes + off) = o1;
        *reinterpret_cast<uint2*>(st + 2 * kGPartBytes + off) = o2;
        if (cl == 0) sfac[slot * 128 + row] = __int_as_float((127 + E - 8) << 23);
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
        const df s1m = df_split(s1 - r[i]);  // |U_i|^2 = sigma1^2 - r_i
        for (int e = lane; e < NPAIR; e += 32) {
          int pa, pb;
          pair_of<kGP>(e, pa, pb);  // pa >= pb
          df v = {0.f, 0.f};
          if (pa != kGL) {
            v = df_two_sum(S[kGL * kGSStride + pa], S[kGL * kGSStride + pb]);
            const df tt = df_two_sum(v.hi, S[pa * kGSStride + pb]);
            v = df{tt.hi, v.lo + tt.lo};
          } else if (pb != kGL) {
            v = df{S[kGL * kGSStride + pb], 0.f};
          }
          const df tt = df_two_sum(v.hi, s1m.hi);
          gram[i * NPAIR + e] = tt.hi + (tt.lo + (v.lo + s1m.lo));
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
// positions (m + 1 <= 32 rounded up to 32), on the tensor cores.
vst_status gram_tc_rows(const int32_t* nn, const int32_t* nn_cnt, int64_t n, int m, int k, const float* U,
                        const double* r, double s1, float* gram, WsHeader* hdr, cudaStream_t st) {
  if (n <= 0 || k <= 0) return VST_OK;
  cudaError_t e = cudaFuncSetAttribute(gram_tc_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kGSmem);
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core row Gram attributes");
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ngroups = (n + kGRows - 1) / kGRows;
  const int grid = (int)std::min<int64_t>(ngroups, std::max(1, sms));
  gram_tc_rows_kernel<<<grid, kGThreads, kGSmem, st>>>(nn, nn_cnt, n, m, k, U, r, s1, gram, hdr);
  e = cudaGetLastError();
  return e == cudaSuccess ? VST_OK : cuda_fail(e, "tensor-core row Gram");
}

}  // namespace vst
