// Tracing aids: a count of the library's kernel launches and, when enabled,
// CUDA-event timings of the tensor-core GEMM kernels recorded on the stream
// each kernel is launched on.
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace rsvd {

namespace {
std::atomic<long long> g_launches{0};
std::mutex g_mu;
bool g_on = false;
struct Rec {
  int cls;
  cudaEvent_t a, b;
};
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t get_event() {
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

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int trace_begin(int cls, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return -1;
  Rec r{cls, get_event(), get_event()};
  if (!r.a || !r.b) return -1;
  if (cudaEventRecord(r.a, s) != cudaSuccess) return -1;
  g_recs.push_back(r);
  return (int)g_recs.size() - 1;
}

void trace_end(int idx, cudaStream_t s) {
  if (idx < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (idx < (int)g_recs.size()) cudaEventRecord(g_recs[idx].b, s);
}

}  // namespace rsvd

extern "C" {

rsvd_status rsvd_trace_enable(int enable) {
  std::lock_guard<std::mutex> lk(rsvd::g_mu);
  rsvd::g_on = enable != 0;
  return RSVD_OK;
}

int64_t rsvd_kernel_launch_count(void) { return rsvd::g_launches.load(); }

int rsvd_trace_read(double* ms, int64_t* launches, int nclass) {
  std::lock_guard<std::mutex> lk(rsvd::g_mu);
  if (!ms || !launches || nclass < 1) return -1;
  for (int c = 0; c < nclass; ++c) {
    ms[c] = 0.0;
    launches[c] = 0;
  }
  for (auto& r : rsvd::g_recs) {
    float t = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess &&
        r.cls >= 0 && r.cls < nclass) {
      ms[r.cls] += t;
      launches[r.cls] += 1;
    }
    rsvd::g_pool.push_back(r.a);
    rsvd::g_pool.push_back(r.b);
  }
  rsvd::g_recs.clear();
  return RSVD_TRACE_CLASSES;
}

}  // extern "C"
