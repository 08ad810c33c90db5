// Per-launcher timing with CUDA events on the launching stream (off by default).
#include <atomic>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "tachiom_internal.cuh"

namespace tachiom {

namespace {
struct Rec {
  const char *name;
  cudaEvent_t a, b;
};
std::atomic<int> g_on{0};
std::mutex g_mu;
std::map<cudaStream_t, std::vector<Rec>> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

ProfScope::ProfScope(const char *name, cudaStream_t s) : name_(name), s_(s), a_(nullptr) {
  if (!g_on.load(std::memory_order_relaxed)) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;
  }
  std::lock_guard<std::mutex> g(g_mu);
  a_ = take_event();
  cudaEventRecord((cudaEvent_t)a_, s);
}

ProfScope::~ProfScope() {
  if (!a_) return;
  std::lock_guard<std::mutex> g(g_mu);
  cudaEvent_t b = take_event();
  cudaEventRecord(b, s_);
  g_recs[s_].push_back({name_, (cudaEvent_t)a_, b});
}

}  // namespace tachiom

using namespace tachiom;

extern "C" tachiom_status tachiom_profile_enable(int on) {
  g_on.store(on ? 1 : 0);
  return TACHIOM_OK;
}

extern "C" tachiom_status tachiom_profile_read(void *stream, tachiom_profile_entry *out, int32_t cap,
                                               int32_t *n_out) {
  if (!n_out || (cap > 0 && !out)) return fail(TACHIOM_ERR_INVALID, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  TCUDA(cudaStreamSynchronize(s));
  std::vector<Rec> recs;
  {
    std::lock_guard<std::mutex> g(g_mu);
    recs.swap(g_recs[s]);
  }
  std::vector<std::string> order;
  std::map<std::string, std::pair<int, double>> agg;
  for (auto &r : recs) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    std::string k(r.name);
    if (!agg.count(k)) order.push_back(k);
    agg[k].first += 1;
    agg[k].second += ms;
  }
  {
    std::lock_guard<std::mutex> g(g_mu);
    for (auto &r : recs) {
      g_pool.push_back(r.a);
      g_pool.push_back(r.b);
    }
  }
  int n = 0;
  for (auto &k : order) {
    if (n >= cap) break;
    memset(out[n].name, 0, sizeof out[n].name);
    strncpy(out[n].name, k.c_str(), sizeof out[n].name - 1);
    out[n].launches = agg[k].first;
    out[n].total_ms = agg[k].second;
    n++;
  }
  *n_out = n;
  return TACHIOM_OK;
}
