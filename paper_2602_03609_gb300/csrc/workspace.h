// Layout of the caller-provided workspace.  Every region starts on a 256-byte
// boundary; the layout depends only on (n, m, k), so vst_workspace_size() and
// the entry points agree.
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>

#include "common.cuh"

namespace vst {

constexpr int64_t kMaxTimeBins = 1 << 16;   // neighbour search: time bins
constexpr int kBBoxBlocks = 512;            // neighbour search: bounding-box partials

inline int64_t max_buckets(int64_t n) { return 2 * n + 4096; }

// VIF scratch (only when k > 0), sized for FP64 buffers
constexpr int64_t kVifMaxWarps = 1 << 16;
constexpr int kVifSyrkChunks = 16;
constexpr int64_t kVifMaxK = 4096;
constexpr int64_t kVifMaxDays = 4096;  // data-day x inducing-point lag table
constexpr int kVifDayBlocks = 256;     // day-range reduction blocks

struct VifLayout {
  size_t S, X, U, r, gram, WE, logd, syrk, G, M, v, z, dinfo, dtab;
  size_t uscale;  // mixed: per (U row, 64-column chunk) scale of its fixed-point parts
  size_t Ap, Bp, zf;  // tensor-core low rank: BF16 operand parts, inducing coordinates
  size_t rpart;       // per (row, column tile) sums of U_ic^2 from the GEMM epilogue
  size_t dpart;       // day-range partials
  size_t lagdf;       // per-lag (P, G) as double-floats (mixed residual covariance)
  // residual-correlation neighbour search: per-row threshold, candidate
  // lists and counts, rows left to the brute-force search and their count
  size_t tau, cand, ccount, fbrows, fbcount;
  size_t gath;  // BF16 U rows of the rows re-screened after a candidate overflow
  size_t kscr;  // knn_scratch_bytes
  size_t total;
};

// inducing-point dimension padded for the tensor-core GEMM (N tiles of 256)
inline int64_t vif_kp(int64_t k) { return (k + 255) / 256 * 256; }
constexpr int kVifMaxParts = 3;  // BF16 parts per operand value
constexpr int kVifCand = 1024;   // candidate slots per row of the filtered neighbour search
constexpr int64_t kVifGather = 8192;  // rows per batch of the search's second (gathered) round
// tensor-core candidate filter of the residual search: row and column tile
// sizes, row tiles per group
constexpr int kKnnTileRows = 128, kKnnTileCols = 256, kKnnGroup = 16;

// scratch of that filter: item counts per group, per-tile time ranges, the
// times flag, counters, the row lists of its later rounds and their |rho|
// histograms (256 bins)
inline size_t knn_scratch_bytes(int64_t n) {
  auto a = [](size_t v) { return (v + 255) & ~size_t(255); };
  const size_t nn = n > 0 ? (size_t)n : 1;
  const size_t T = (nn + kKnnTileRows - 1) / kKnnTileRows, T2 = (nn + kKnnTileCols - 1) / kKnnTileCols;
  const size_t ng = (T + kKnnGroup - 1) / kKnnGroup;
  const size_t tg = (size_t)std::min<int64_t>((int64_t)nn, kVifGather) / kKnnTileRows + 1;
  const size_t ng2 = (size_t)std::min<int64_t>((int64_t)nn, kVifGather);
  return a(8 * (ng + 1)) + a(16 * T) + a(16 * T2) + a(16 * tg) + a(4) + a(64) + 4 * a(4 * nn) + a(4 * ng2 * 256) +
         a(4 * ng2);
}

inline size_t align256(size_t v);

// one operand of the tensor-core contractions over the points: its
// transposed BF16 parts [kVifMaxParts][kp][np] (np = n rounded up to 128),
// the exponent of each column over each 128-row block [np / 128][kp] (int16)
// and over all rows [kp] (int32)
inline size_t tc_operand_bytes(int64_t n, int64_t kc) {
  const size_t kp = (size_t)vif_kp(kc > 0 ? kc : 1);
  const size_t np = (size_t)((n > 0 ? n : 1) + 127) / 128 * 128;
  return align256(2 * (size_t)kVifMaxParts * kp * np) + align256(2 * (np / 128) * kp) + align256(4 * kp);
}
// scratch of the symmetric product A^T A: one operand
inline size_t tc_syrk_tmp_bytes(int64_t n, int64_t kc) { return tc_operand_bytes(n, kc); }

inline VifLayout vif_layout(int64_t n, int m, int64_t k) {
  VifLayout L{};
  size_t off = 0;
  auto take = [&off](size_t b) {
    const size_t at = off;
    off = (off + b + 255) & ~size_t(255);
    return at;
  };
  const size_t nn = n > 0 ? (size_t)n : 1, kk = k > 0 ? (size_t)k : 1;
  const int pm = padded_pm(m + 1);
  const size_t npair = (size_t)pm * (pm + 1) / 2;
  L.S = take(sizeof(double) * kk * kk);
  L.X = take(sizeof(double) * kk * kk);
  L.U = take(sizeof(double) * nn * kk);
  L.r = take(sizeof(double) * nn);
  L.gram = take(sizeof(double) * nn * npair);
  L.WE = take(sizeof(double) * nn * (kk + 1));
  L.logd = take(sizeof(double) * kVifMaxWarps);
  L.syrk = take(sizeof(double) * (kk + 1) * (kk + 1) * kVifSyrkChunks);
  L.G = take(sizeof(double) * (kk + 1) * (kk + 1));
  L.M = take(sizeof(double) * kk * kk);
  L.v = take(sizeof(double) * (kk + 1));
  L.z = take(sizeof(double) * (kk + 2));
  L.dinfo = take(sizeof(int64_t) * 4);
  L.dtab = take(sizeof(float) * 2 * kk * (size_t)kVifMaxDays);
  L.uscale = take(sizeof(float) * nn * ((kk + 63) / 64));
  const size_t kp = (size_t)vif_kp((int64_t)kk);
  // (the residual neighbour search keeps U in FP32 and then in BF16 [n][k
  // rounded up to 64] here; the 1 KiB covers the alignment between the two)
  // (also the scratch of the tensor-core [W e]^T [W e], kk + 1 columns)
  L.Ap = take(std::max(2 * (size_t)kVifMaxParts * nn * kp + 1024, tc_syrk_tmp_bytes((int64_t)nn, (int64_t)kk + 1)));
  L.Bp = take(2 * (size_t)kVifMaxParts * kp * kp);
  L.zf = take(16 * kk);
  L.rpart = take(sizeof(double) * nn * (kp / 128));
  L.dpart = take(sizeof(double) * 3 * kVifDayBlocks);
  L.lagdf = take(16 * (size_t)kLagTab);
  L.tau = take(16 * nn);
  L.cand = take(sizeof(int32_t) * nn * kVifCand);
  L.ccount = take(sizeof(int32_t) * nn);
  L.fbrows = take(sizeof(int32_t) * nn);
  L.fbcount = take(256);
  L.gath = take(2 * (size_t)std::min<int64_t>((int64_t)nn, kVifGather) * (size_t)((kk + 63) / 64 * 64));
  L.kscr = take(knn_scratch_bytes((int64_t)nn));
  L.total = off;
  return L;
}

struct WsLayout {
  size_t hdr, lagd, lagf, partial, flag, prep;
  size_t vif;  // VIF scratch (k > 0 only)
  // neighbour search
  size_t bbox_part, bbox, binmin, offsets, cursor, blocksums, sidx, sx, sy, pbucket;
  // Vecchia sampling
  size_t sA, sD, ready, counter;
  size_t total;
};

inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

inline WsLayout ws_layout(int64_t n, int m, int64_t k) {
  WsLayout L{};
  size_t off = 0;
  auto take = [&off](size_t bytes) {
    const size_t at = off;
    off = align256(off + bytes);
    return at;
  };
  const int64_t nb = max_buckets(n);
  const int64_t nn = n > 0 ? n : 1;
  L.hdr = take(256);
  L.lagd = take(sizeof(LagD) * kLagTab);
  L.lagf = take(sizeof(LagF) * kLagTab);
  L.partial = take(sizeof(double) * 8 * (size_t)(1 << 16) * 2);
  L.flag = take((size_t)nn);
  L.prep = take(sizeof(PrepPt) * (size_t)nn);
  L.bbox_part = take(sizeof(double) * 8 * kBBoxBlocks);
  L.bbox = take(sizeof(double) * 8);
  L.binmin = take(sizeof(int32_t) * kMaxTimeBins);
  L.offsets = take(sizeof(int32_t) * (size_t)(nb + 1));
  L.cursor = take(sizeof(int32_t) * (size_t)nb);
  L.blocksums = take(sizeof(int32_t) * (size_t)(nb / 1024 + 2));
  L.sidx = take(sizeof(int32_t) * (size_t)nn);
  L.sx = take(sizeof(float) * (size_t)nn);
  L.sy = take(sizeof(float) * (size_t)nn);
  L.pbucket = take(sizeof(int32_t) * (size_t)nn);
  L.sA = take(sizeof(double) * (size_t)nn * (size_t)(m > 0 ? m : 1));
  L.sD = take(sizeof(double) * (size_t)nn);
  L.ready = take(sizeof(int32_t) * (size_t)nn);
  L.counter = take(sizeof(unsigned long long) * 2);
  L.vif = take(k > 0 ? vif_layout(n, m, k).total : 0);
  L.total = off;
  return L;
}

}  // namespace vst
