// Phase profiler: when enabled, each instrumented launch is bracketed by two
// CUDA events on its own stream and tagged with the algorithmic flops and
// bytes of that launch.  tk_profile_collect() turns the records into per-phase
// totals (time from the events, so only device time is counted).
#include <atomic>
#include <mutex>
#include <vector>

#include "tk_internal.cuh"

namespace tk {
namespace {

struct Rec {
  int phase;
  cudaEvent_t a, b;
  double flops, bytes, impl_bytes;
  bool closed;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

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

std::atomic<unsigned long long> g_launches{0};

}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(size_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

bool prof_enabled() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_on;
}

int prof_begin(int phase, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return -1;
  Rec r{phase, take_event(), take_event(), 0.0, 0.0, 0.0, false};
  if (!r.a || !r.b) return -1;
  cudaEventRecord(r.a, st);
  g_recs.push_back(r);
  return (int)g_recs.size() - 1;
}

void prof_end(int tok, cudaStream_t st, double flops, double bytes, double impl_bytes) {
  if (tok < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (tok >= (int)g_recs.size()) return;
  Rec& r = g_recs[tok];
  cudaEventRecord(r.b, st);
  r.flops = flops;
  r.bytes = bytes;
  r.impl_bytes = impl_bytes < 0.0 ? bytes : impl_bytes;
  r.closed = true;
}

}  // namespace tk

using namespace tk;

extern "C" {

TK_API const char* tk_phase_name(int phase) {
  static const char* names[TK_PHASE_COUNT] = {"sketch", "gram",        "cholesky",     "svd",
                                              "precond_apply", "A_times_W", "At_times_U", "refine_residual64",
                                              "refine_normal64", "precond_inverse", "A_times_W_digits",
                                              "At_times_U_digits", "slice_A", "cholesky_update",
                                              "lsqr_step_fused"};
  if (phase < 0 || phase >= TK_PHASE_COUNT) return "unknown";
  return names[phase];
}

TK_API unsigned long long tk_launch_count(void) { return g_launches.load(); }

TK_API tk_status tk_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = on != 0;
  return TK_OK;
}

TK_API tk_status tk_profile_collect(tk_phase_stats* out) {
  std::vector<Rec> recs;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    recs.swap(g_recs);
  }
  if (out)
    for (int p = 0; p < TK_PHASE_COUNT; ++p) out[p] = tk_phase_stats{0.0, 0.0, 0.0, 0, 0.0};
  tk_status st = TK_OK;
  for (auto& r : recs) {
    if (r.closed) {
      if (cudaEventSynchronize(r.b) != cudaSuccess) st = TK_ECUDA;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) st = TK_ECUDA;
      if (out && r.phase >= 0 && r.phase < TK_PHASE_COUNT) {
        out[r.phase].ms += ms;
        out[r.phase].flops += r.flops;
        out[r.phase].bytes += r.bytes;
        out[r.phase].impl_bytes += r.impl_bytes;
        out[r.phase].launches += 1;
      }
    }
  }
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& r : recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  return st;
}

}  // extern "C"
