// Stage timing with CUDA events (a measurement aid of the C ABI).
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "api_internal.h"

namespace gmi {
namespace {

struct Pending {
  int stage;
  cudaEvent_t a, b;
};

std::mutex g_mu;
bool g_on = false;
std::vector<cudaEvent_t> g_free;
std::vector<Pending> g_pending;
constexpr int kPool = 8192;

}  // namespace

bool profile_on() { return g_on; }

// Records the opening event of a stage (stage -1 in the mark when off or exhausted).
ProfileMark profile_begin(int stage, cudaStream_t s) {
  static const char* const kRange[GMI_STAGE_COUNT] = {"gmi.bin", "gmi.near", "gmi.far", "gmi.backward"};
  ProfileMark m{-1, nullptr, nullptr, false};
  if (stage >= 0 && stage < GMI_STAGE_COUNT) {
    nvtxRangePushA(kRange[stage]);
    m.range = true;
  }
  if (!g_on) return m;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return m;  // not inside graphs
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_free.size() < 2) return m;
  m.stage = stage;
  m.a = g_free.back(); g_free.pop_back();
  m.b = g_free.back(); g_free.pop_back();
  cudaEventRecord(m.a, s);
  return m;
}

void profile_end(const ProfileMark& m, cudaStream_t s) {
  if (m.range) nvtxRangePop();
  if (m.stage < 0) return;
  cudaEventRecord(m.b, s);
  std::lock_guard<std::mutex> lk(g_mu);
  g_pending.push_back(Pending{m.stage, m.a, m.b});
}

}  // namespace gmi

using namespace gmi;

extern "C" gmi_status gmi_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (on && g_free.empty() && g_pending.empty()) {
    for (int i = 0; i < kPool; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return GMI_ERR_CUDA;
      g_free.push_back(e);
    }
  }
  g_on = on != 0;
  return GMI_OK;
}

extern "C" gmi_status gmi_profile_read(double* ms, int* launches, int reset) {
  std::vector<Pending> todo;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    todo = g_pending;
    if (reset) g_pending.clear();
  }
  double acc[GMI_STAGE_COUNT] = {0, 0, 0, 0};
  int cnt[GMI_STAGE_COUNT] = {0, 0, 0, 0};
  gmi_status st = GMI_OK;
  for (const Pending& p : todo) {
    float t = 0.f;
    if (cudaEventSynchronize(p.b) != cudaSuccess || cudaEventElapsedTime(&t, p.a, p.b) != cudaSuccess) {
      st = GMI_ERR_CUDA;
      continue;
    }
    if (p.stage >= 0 && p.stage < GMI_STAGE_COUNT) {
      acc[p.stage] += t;
      cnt[p.stage] += 1;
    }
  }
  if (reset) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (const Pending& p : todo) {
      g_free.push_back(p.a);
      g_free.push_back(p.b);
    }
  }
  for (int k = 0; k < GMI_STAGE_COUNT; ++k) {
    if (ms) ms[k] += acc[k];
    if (launches) launches[k] += cnt[k];
  }
  return st;
}
