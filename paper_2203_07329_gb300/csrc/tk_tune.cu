// Measured tile choices for the GEMMs of the LSQR and refinement passes.
//
// tk_autotune() runs, on the caller's workspace, every candidate tile shape
// (and, for split-K products, every candidate split count) of the products a
// solve of that problem will issue, for the active-lambda counts 1, 2, 4, ...
// up to N, times each on the stream with CUDA events, and records the
// fastest here.  The GEMM dispatch and the split-K callers consult this table
// on every launch; shapes that were never tuned keep the fixed rules.
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <mutex>
#include <tuple>

#include "tk_internal.cuh"

namespace tk {
namespace {

using Key = std::tuple<int, int, int, int, int, int, int64_t, int64_t, int64_t>;
std::mutex g_tune_mu;
std::map<Key, TuneChoice> g_tune;

Key make_key(const GemmKey& k) {
  return Key(k.ta, k.tb, k.tc, k.transA, k.transB, k.split, k.M, k.N, k.K);
}

}  // namespace

int64_t tune_bucket(int64_t M) {
  int64_t b = 1;
  while (b < M) b <<= 1;
  return b;
}

bool tune_lookup(GemmKey k, TuneChoice* out) {
  k.M = tune_bucket(k.M);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(make_key(k));
  if (it == g_tune.end()) return false;
  *out = it->second;
  return true;
}

void tune_store(GemmKey k, TuneChoice c) {
  k.M = tune_bucket(k.M);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[make_key(k)] = c;
}

size_t tune_size() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return g_tune.size();
}

size_t tune_describe(char* buf, size_t len) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::string out;
  char line[160];
  for (const auto& kv : g_tune) {
    const Key& k = kv.first;
    snprintf(line, sizeof line, "types %d%d%d trans %d%d split %d M %lld N %lld K %lld -> cfg %d splits %d\n",
             std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k), std::get<4>(k), std::get<5>(k),
             (long long)std::get<6>(k), (long long)std::get<7>(k), (long long)std::get<8>(k), kv.second.cfg,
             kv.second.splits);
    out += line;
  }
  if (buf && len > 0) {
    const size_t n = std::min(len - 1, out.size());
    memcpy(buf, out.data(), n);
    buf[n] = 0;
  }
  return out.size() + 1;
}

void tune_clear() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
}

}  // namespace tk
