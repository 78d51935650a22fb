// Optional CUDA-event timing of the library's main kernels (see vst.h).
#include <cuda_runtime.h>

#include <vector>

#include "profile.h"

namespace vst {

namespace {
constexpr int kMaxRecords = 4096;
constexpr int kClasses = kProfClasses;
struct Rec {
  int cls;
  cudaEvent_t a, b;
};
bool g_on = false;
std::vector<Rec> g_recs;
int64_t g_count[kClasses] = {};
int64_t g_dropped[kClasses] = {};

void clear() {
  for (auto& r : g_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_recs.clear();
  for (int c = 0; c < kClasses; ++c) g_count[c] = g_dropped[c] = 0;
}
}  // namespace

ProfileScope::ProfileScope(int cls, cudaStream_t st) : cls_(cls), st_(st), rec_(-1) {
  if (!g_on || cls < 0 || cls >= kClasses) return;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return;
  ++g_count[cls];
  if ((int)g_recs.size() >= kMaxRecords) {
    ++g_dropped[cls];
    return;
  }
  Rec r{cls, nullptr, nullptr};
  if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return;
  cudaEventRecord(r.a, st);
  g_recs.push_back(r);
  rec_ = (int)g_recs.size() - 1;
}

ProfileScope::~ProfileScope() {
  if (rec_ >= 0 && rec_ < (int)g_recs.size()) cudaEventRecord(g_recs[rec_].b, st_);
}

}  // namespace vst

extern "C" void vst_profile_enable(int on) {
  vst::clear();
  vst::g_on = on != 0;
}

extern "C" int vst_profile_read(int cls, int64_t* launches, double* total_ms) {
  using namespace vst;
  if (cls < 0 || cls >= kClasses) return -1;
  double ms = 0.0;
  for (auto& r : g_recs) {
    if (r.cls != cls) continue;
    cudaEventSynchronize(r.b);
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms += t;
  }
  if (launches) *launches = g_count[cls];
  if (total_ms) *total_ms = ms;
  return g_dropped[cls] ? 1 : 0;
}
