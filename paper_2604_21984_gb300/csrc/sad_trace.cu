// Stage tracing of libsad.so: CUDA events around kernel launches, recorded
// only while switched on (sad_trace_enable) and never on a capturing stream.
// The host-side bookkeeping is a mutex-protected list; collection waits for
// the recorded events and returns per-stage launch counts and device times.
#include <cstring>
#include <mutex>
#include <vector>

#include "sad_host.h"

namespace sad {

namespace {

struct TraceRec {
  const char* name;
  cudaEvent_t e0, e1;
};

std::mutex g_mu;
bool g_on = false;
std::vector<cudaEvent_t> g_pool;
std::vector<TraceRec> g_recs;
constexpr size_t kMaxRecs = 1 << 16;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

}  // namespace

TraceScope::TraceScope(cudaStream_t st, const char* nm) : s(st), name(nm), e0(nullptr), e1(nullptr) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on || g_recs.size() >= kMaxRecs) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;
  }
  e0 = take_event();
  e1 = take_event();
  if (!e0 || !e1 || cudaEventRecord(e0, s) != cudaSuccess) {
    if (e0) g_pool.push_back(e0);
    if (e1) g_pool.push_back(e1);
    e0 = e1 = nullptr;
    cudaGetLastError();
  }
}

TraceScope::~TraceScope() {
  if (!e0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (cudaEventRecord(e1, s) != cudaSuccess) {
    cudaGetLastError();
    g_pool.push_back(e0);
    g_pool.push_back(e1);
    return;
  }
  g_recs.push_back(TraceRec{name, e0, e1});
}

}  // namespace sad

using namespace sad;

extern "C" {

int sad_trace_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  const int prev = g_on ? 1 : 0;
  g_on = on != 0;
  return prev;
}

int sad_trace_collect(sad_trace_entry* out, int32_t max_entries, int32_t* n_out) {
  if (!n_out || max_entries < 0 || (max_entries > 0 && !out))
    return einval("sad_trace_collect: bad output arguments");
  std::vector<TraceRec> recs;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    recs.swap(g_recs);
  }
  std::vector<sad_trace_entry> agg;
  int status = SAD_OK;
  for (const TraceRec& r : recs) {
    float ms = 0.f;
    if (status == SAD_OK) {
      cudaError_t e = cudaEventSynchronize(r.e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.e0, r.e1);
      if (e != cudaSuccess) {
        set_error("sad_trace_collect: %s", cudaGetErrorString(e));
        status = SAD_ECUDA;
      }
    }
    if (status == SAD_OK) {
      size_t k = 0;
      while (k < agg.size() && std::strncmp(agg[k].name, r.name, sizeof(agg[k].name) - 1) != 0) ++k;
      if (k == agg.size()) {
        sad_trace_entry t{};
        std::strncpy(t.name, r.name, sizeof(t.name) - 1);
        agg.push_back(t);
      }
      agg[k].launches += 1;
      agg[k].total_ms += ms;
    }
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (const TraceRec& r : recs) {
      g_pool.push_back(r.e0);
      g_pool.push_back(r.e1);
    }
  }
  *n_out = static_cast<int32_t>(agg.size());
  for (size_t k = 0; k < agg.size() && static_cast<int32_t>(k) < max_entries; ++k) out[k] = agg[k];
  return status;
}

}  // extern "C"
