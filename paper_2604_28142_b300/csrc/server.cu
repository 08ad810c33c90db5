// Continuous-batching request loop over tachiom_search.
//
// Requests (one query each, 1..32 tokens, its own k) are submitted from any
// host thread and queued. A scheduler thread owns `n_slots` slots; a slot is a
// CUDA stream with pinned staging and device buffers for one batch. Whenever a
// slot is free it takes the queued requests in arrival order (up to the batch
// limits), copies them in, runs the search on its stream and copies the
// results out, so batches admitted while others run overlap on the device.
// Admission also respects a device scratch budget: a batch is only launched
// when the scratch that all in-flight batches may hold stays within it.
// A finished batch hands each request its own results and latency
// (submission to completion on the host clock).
//
// A query's result does not depend on what it is batched with: every step of
// the search treats queries independently and in a fixed order, so a request
// gets the same bits alone and in any mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tachiom_internal.cuh"

namespace tachiom {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  int ntok = 0, k = 0;
  std::vector<float> q;
  std::vector<int32_t> ids;
  std::vector<float> scores;
  Clock::time_point t_submit, t_done;
  bool done = false;
  tachiom_status status = TACHIOM_OK;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  float *h_q = nullptr, *d_q = nullptr;
  int32_t *h_ids = nullptr, *d_ids = nullptr;
  float *h_s = nullptr, *d_s = nullptr;
  std::vector<int32_t> ntok, k;
  std::vector<uint64_t> reqs;
  int64_t scratch = 0;
  bool busy = false;
};

}  // namespace

struct Server {
  Index *ix = nullptr;
  tachiom_search_params params{};
  tachiom_server_config cfg{};
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> pending;
  std::unordered_map<uint64_t, Request> reqs;
  uint64_t next_id = 1;
  std::atomic<bool> stop{false};
  std::thread th;
  int64_t scratch_in_flight = 0;
  // stats
  std::vector<double> lat_ms;
  int64_t batches = 0, batched_queries = 0;
  Clock::time_point t_first, t_last;
  bool any = false;
  tachiom_status fatal = TACHIOM_OK;
  char fatal_msg[256] = {0};
};

namespace {

// scratch a batch may hold: the step (a) survivors per row, the gather's candidate parts and the
// refine's per-candidate buffers
int64_t batch_scratch(const Index &ix, int nq, int rows, int kd, int kc) {
  return (int64_t)rows * (kc * 8 + 4096 * 8) + (int64_t)gather_pool_elems(ix, nq, kd) * 8 + (int64_t)nq * kd * 64;
}

void finish_slot(Server *S, Slot &sl) {
  // results are in the slot's pinned buffers: hand them to the requests
  const auto now = Clock::now();
  int64_t off = 0;
  std::lock_guard<std::mutex> g(S->mu);
  for (size_t u = 0; u < sl.reqs.size(); u++) {
    Request &r = S->reqs[sl.reqs[u]];
    r.ids.assign(sl.h_ids + off, sl.h_ids + off + r.k);
    r.scores.assign(sl.h_s + off, sl.h_s + off + r.k);
    off += r.k;
    r.t_done = now;
    r.done = true;
    S->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r.t_submit).count());
  }
  S->t_last = now;
  S->batches++;
  S->batched_queries += (int64_t)sl.reqs.size();
  S->scratch_in_flight -= sl.scratch;
  sl.reqs.clear();
  sl.busy = false;
  S->cv_done.notify_all();
}

// launch one batch on a free slot; the caller holds no lock
bool launch_batch(Server *S, Slot &sl) {
  std::vector<uint64_t> take;
  int rows = 0, maxk = 0;
  int64_t need = 0;
  {
    std::lock_guard<std::mutex> g(S->mu);
    if (S->pending.empty()) return false;
    const int kd_cap = S->params.kappa_d;
    while (!S->pending.empty() && (int)take.size() < S->cfg.max_batch_queries) {
      const Request &r = S->reqs[S->pending.front()];
      if (rows + r.ntok > S->cfg.max_batch_rows) break;
      if (kd_cap == 0 && std::max(maxk, r.k) * 4 > MAX_KD && !take.empty()) break;
      take.push_back(r.id);
      rows += r.ntok;
      maxk = std::max(maxk, r.k);
      S->pending.pop_front();
    }
    if (take.empty()) return false;
    const int kd = S->params.kappa_d > 0 ? S->params.kappa_d : std::min(MAX_KD, std::max(1000, 4 * maxk));
    need = batch_scratch(*S->ix, (int)take.size(), rows, kd, S->params.kappa_c);
    if (S->cfg.scratch_budget_bytes > 0 && S->scratch_in_flight > 0 &&
        S->scratch_in_flight + need > S->cfg.scratch_budget_bytes) {
      // not enough scratch while others run: put the requests back, in order
      for (auto it = take.rbegin(); it != take.rend(); ++it) S->pending.push_front(*it);
      return false;
    }
    S->scratch_in_flight += need;
    sl.ntok.clear();
    sl.k.clear();
    int64_t qo = 0;
    for (uint64_t id : take) {
      const Request &r = S->reqs[id];
      memcpy(sl.h_q + qo, r.q.data(), (size_t)r.ntok * DIM * 4);
      qo += (int64_t)r.ntok * DIM;
      sl.ntok.push_back(r.ntok);
      sl.k.push_back(r.k);
    }
  }
  sl.reqs = take;
  sl.scratch = need;
  int64_t tk = 0;
  for (int k : sl.k) tk += k;
  tachiom_status st = TACHIOM_OK;
  if (cudaMemcpyAsync(sl.d_q, sl.h_q, (size_t)rows * DIM * 4, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
    st = fail(TACHIOM_ERR_CUDA, "server: query copy failed");
  if (!st)
    st = tachiom_search(reinterpret_cast<tachiom_index *>(S->ix), &S->params, sl.d_q, sl.ntok.data(), sl.k.data(),
                        (int32_t)sl.ntok.size(), sl.d_ids, sl.d_s, sl.stream);
  if (!st && (cudaMemcpyAsync(sl.h_ids, sl.d_ids, (size_t)tk * 4, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
              cudaMemcpyAsync(sl.h_s, sl.d_s, (size_t)tk * 4, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
              cudaEventRecord(sl.done, sl.stream) != cudaSuccess))
    st = fail(TACHIOM_ERR_CUDA, "server: result copy failed");
  if (st) {
    std::lock_guard<std::mutex> g(S->mu);
    for (uint64_t id : take) {
      Request &r = S->reqs[id];
      r.status = st;
      r.done = true;
    }
    S->scratch_in_flight -= need;
    S->fatal = st;
    snprintf(S->fatal_msg, sizeof S->fatal_msg, "%s", tachiom_last_error());
    sl.reqs.clear();
    S->cv_done.notify_all();
    return false;
  }
  sl.busy = true;
  return true;
}

void scheduler(Server *S) {
  cudaSetDevice(S->ix->device);
  while (true) {
    bool did = false;
    // completions
    for (Slot &sl : S->slots) {
      if (sl.busy && cudaEventQuery(sl.done) == cudaSuccess) {
        finish_slot(S, sl);
        did = true;
      }
    }
    // admissions: a free slot takes the queue's head once the batch is full, the
    // oldest request has waited max_wait_us, or the device is otherwise idle
    bool any_busy = false;
    for (Slot &sl : S->slots) any_busy |= sl.busy;
    for (Slot &sl : S->slots) {
      if (sl.busy) continue;
      bool go = false;
      {
        std::lock_guard<std::mutex> g(S->mu);
        if (!S->pending.empty()) {
          const Request &head = S->reqs[S->pending.front()];
          const double waited = std::chrono::duration<double, std::micro>(Clock::now() - head.t_submit).count();
          go = !any_busy || (int)S->pending.size() >= S->cfg.max_batch_queries || waited >= S->cfg.max_wait_us;
        }
      }
      if (go && launch_batch(S, sl)) {
        did = true;
        any_busy = true;
      }
    }
    if (S->stop.load()) {
      bool busy = false;
      for (Slot &sl : S->slots) busy |= sl.busy;
      std::lock_guard<std::mutex> g(S->mu);
      if (!busy && S->pending.empty()) break;
    }
    if (!did) {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait_for(lk, std::chrono::microseconds(20));
    }
  }
}

void destroy_slots(Server *S) {
  for (Slot &sl : S->slots) {
    if (sl.stream) {
      cudaStreamSynchronize(sl.stream);
      ws_release(S->ix, sl.stream);
    }
    if (sl.h_q) cudaFreeHost(sl.h_q);
    if (sl.h_ids) cudaFreeHost(sl.h_ids);
    if (sl.h_s) cudaFreeHost(sl.h_s);
    if (sl.d_q) cudaFree(sl.d_q);
    if (sl.d_ids) cudaFree(sl.d_ids);
    if (sl.d_s) cudaFree(sl.d_s);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  S->slots.clear();
}

}  // namespace
}  // namespace tachiom

using namespace tachiom;

extern "C" tachiom_status tachiom_server_create(tachiom_index *index, const tachiom_search_params *params,
                                                const tachiom_server_config *cfg, tachiom_server **out) {
  if (!index || !params || !cfg || !out) return fail(TACHIOM_ERR_INVALID, "NULL argument");
  *out = nullptr;
  if (params->kappa_c < 1 || params->kappa_c > MAX_KC || params->kappa_d < 0 || params->kappa_d > MAX_KD)
    return fail(TACHIOM_ERR_INVALID, "bad search parameters");
  if (cfg->n_slots < 1 || cfg->n_slots > 64 || cfg->max_batch_queries < 1 || cfg->max_batch_rows < MAX_NTOK ||
      cfg->max_wait_us < 0)
    return fail(TACHIOM_ERR_INVALID, "bad server configuration");
  Index *ix = reinterpret_cast<Index *>(index);
  Server *S = new Server();
  S->ix = ix;
  S->params = *params;
  S->cfg = *cfg;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ix->device);
  S->slots.resize(cfg->n_slots);
  const int64_t maxk_total = (int64_t)cfg->max_batch_queries * MAX_KD;
  for (Slot &sl : S->slots) {
    bool ok = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess &&
              cudaMallocHost((void **)&sl.h_q, (size_t)cfg->max_batch_rows * DIM * 4) == cudaSuccess &&
              cudaMallocHost((void **)&sl.h_ids, (size_t)maxk_total * 4) == cudaSuccess &&
              cudaMallocHost((void **)&sl.h_s, (size_t)maxk_total * 4) == cudaSuccess &&
              cudaMalloc((void **)&sl.d_q, (size_t)cfg->max_batch_rows * DIM * 4) == cudaSuccess &&
              cudaMalloc((void **)&sl.d_ids, (size_t)maxk_total * 4) == cudaSuccess &&
              cudaMalloc((void **)&sl.d_s, (size_t)maxk_total * 4) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      destroy_slots(S);
      delete S;
      cudaSetDevice(prev);
      return fail(TACHIOM_ERR_OOM, "server: slot allocation failed");
    }
  }
  cudaSetDevice(prev);
  S->th = std::thread(scheduler, S);
  *out = reinterpret_cast<tachiom_server *>(S);
  return TACHIOM_OK;
}

extern "C" tachiom_status tachiom_server_submit(tachiom_server *server, const float *h_query, int32_t ntok,
                                                int32_t k, uint64_t *id_out) {
  Server *S = reinterpret_cast<Server *>(server);
  if (!S || !h_query || !id_out) return fail(TACHIOM_ERR_INVALID, "NULL argument");
  if (ntok < 1 || ntok > MAX_NTOK) return fail(TACHIOM_ERR_INVALID, "ntok = %d out of [1, %d]", ntok, MAX_NTOK);
  const int kd = S->params.kappa_d > 0 ? S->params.kappa_d : MAX_KD;
  if (k < 1 || k > kd) return fail(TACHIOM_ERR_INVALID, "k = %d out of [1, kappa_d]", k);
  if (S->stop.load()) return fail(TACHIOM_ERR_BUSY, "server is shutting down");
  Request r;
  r.ntok = ntok;
  r.k = k;
  r.q.assign(h_query, h_query + (size_t)ntok * DIM);
  r.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> g(S->mu);
    if (S->fatal) return fail(S->fatal, "server stopped after an error: %s", S->fatal_msg);
    r.id = S->next_id++;
    if (!S->any) {
      S->any = true;
      S->t_first = r.t_submit;
    }
    *id_out = r.id;
    S->pending.push_back(r.id);
    S->reqs.emplace(r.id, std::move(r));
  }
  S->cv_work.notify_one();
  return TACHIOM_OK;
}

extern "C" tachiom_status tachiom_server_wait(tachiom_server *server, uint64_t id, int32_t timeout_ms,
                                              int32_t *h_ids, float *h_scores, double *latency_ms) {
  Server *S = reinterpret_cast<Server *>(server);
  if (!S) return fail(TACHIOM_ERR_INVALID, "NULL server");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return fail(TACHIOM_ERR_INVALID, "unknown request id %llu", (unsigned long long)id);
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
  while (!it->second.done) {
    if (timeout_ms >= 0 && Clock::now() >= deadline) return fail(TACHIOM_ERR_TIMEOUT, "request not finished");
    S->cv_done.wait_for(lk, std::chrono::milliseconds(1));
    it = S->reqs.find(id);
  }
  Request &r = it->second;
  tachiom_status st = r.status;
  if (!st) {
    if (h_ids) memcpy(h_ids, r.ids.data(), (size_t)r.k * 4);
    if (h_scores) memcpy(h_scores, r.scores.data(), (size_t)r.k * 4);
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
  }
  S->reqs.erase(it);
  if (st) return fail(st, "request failed: %s", S->fatal_msg);
  return TACHIOM_OK;
}

extern "C" tachiom_status tachiom_server_read_stats(tachiom_server *server, tachiom_server_stats *out) {
  Server *S = reinterpret_cast<Server *>(server);
  if (!S || !out) return fail(TACHIOM_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> g(S->mu);
  memset(out, 0, sizeof *out);
  out->completed = (int64_t)S->lat_ms.size();
  out->batches = S->batches;
  out->mean_batch = S->batches ? (double)S->batched_queries / S->batches : 0.0;
  if (!S->lat_ms.empty()) {
    std::vector<double> v = S->lat_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
    out->p50_ms = pct(0.50);
    out->p95_ms = pct(0.95);
    out->p99_ms = pct(0.99);
    const double span = std::chrono::duration<double>(S->t_last - S->t_first).count();
    out->qps = span > 0 ? out->completed / span : 0.0;
  }
  return TACHIOM_OK;
}

extern "C" tachiom_status tachiom_server_destroy(tachiom_server *server) {
  Server *S = reinterpret_cast<Server *>(server);
  if (!S) return TACHIOM_OK;
  S->stop.store(true);
  S->cv_work.notify_all();
  if (S->th.joinable()) S->th.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(S->ix->device);
  destroy_slots(S);
  cudaSetDevice(prev);
  delete S;
  return TACHIOM_OK;
}
