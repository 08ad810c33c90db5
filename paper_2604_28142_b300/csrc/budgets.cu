// Candidate budgets (kappa_c, kappa_d) picked by measurement, and the exhaustive
// reference they are judged against.
//
// tachiom_exhaustive_topk: the k best documents of the whole collection by the
// refined score S(q, d) = sum_i max_t (<q_i, c_a(t)> + rho_t <q_i, r^_t>) of Sec. 2.2
// (the cascade with kappa_c = C and kappa_d = D, "exhaustive PQ-MaxSim"). Every
// document is scored by the refine of step (c) in chunks of 4,096 consecutive
// document ids per query; a running top-k per query is merged on the host by
// (score desc, doc asc).
//
// tachiom_autotune_budgets: the paper tunes kappa_c and kappa_d on a grid
// (Sec. 3). On a tuning split of queries, every (kappa_c, kappa_d) of the grid is
// timed (CUDA events, median of 3 runs) and its recall@k against the exhaustive
// top-k is measured; the fastest point with recall >= min_recall wins (none: the
// point of highest recall, the faster on a tie).
#include <algorithm>
#include <cstring>
#include <vector>

#include "tachiom_internal.cuh"

namespace tachiom {
namespace {

constexpr int kChunk = 4096;  // documents scored per query and refine call

// cand[q][i] = d0 + i, or -1 past the last document
__global__ void k_iota_rows(int32_t *__restrict__ cand, int nq, int64_t d0, int64_t D) {
  const int64_t n = (int64_t)nq * kChunk;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = d0 + (x % kChunk);
    cand[x] = d < D ? (int32_t)d : -1;
  }
}

struct DevBufs {
  std::vector<void *> p;
  ~DevBufs() {
    for (void *q : p) cudaFree(q);
  }
  template <typename T>
  tachiom_status alloc(T **out, size_t n) {
    if (cudaMalloc((void **)out, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      return fail(TACHIOM_ERR_OOM, "autotune buffers");
    }
    p.push_back(*out);
    return TACHIOM_OK;
  }
};

// (score desc, doc asc)
bool better(float sa, int32_t da, float sb, int32_t db) { return sa > sb || (sa == sb && da < db); }

}  // namespace
}  // namespace tachiom

using namespace tachiom;

extern "C" tachiom_status tachiom_exhaustive_topk(tachiom_index *index, int32_t precision, const float *d_queries,
                                                  const int32_t *h_ntok, int32_t nq, int32_t k, int32_t *h_ids,
                                                  float *h_scores, void *stream) {
  Index *ix = reinterpret_cast<Index *>(index);
  if (!ix || !d_queries || !h_ntok || !h_ids || !h_scores) return fail(TACHIOM_ERR_INVALID, "NULL argument");
  if (nq < 0 || nq > 4096) return fail(TACHIOM_ERR_INVALID, "nq out of [0, 4096]");
  if (k < 1 || k > 1000) return fail(TACHIOM_ERR_INVALID, "k out of [1, 1000]");
  if (nq == 0) return TACHIOM_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ix->device) cudaSetDevice(ix->device);
  tachiom_status st = TACHIOM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  {
    DevBufs B;
    int32_t *cand = nullptr, *oi = nullptr;
    float *os = nullptr;
    if (!(st = B.alloc(&cand, (size_t)nq * kChunk)) && !(st = B.alloc(&oi, (size_t)nq * k)) &&
        !(st = B.alloc(&os, (size_t)nq * k))) {
      tachiom_search_params p{};
      p.kappa_c = 1;
      p.kappa_d = kChunk;
      p.precision = precision;
      p.plan_id = -1;
      std::vector<int32_t> kk((size_t)nq, k);
      std::vector<int32_t> ci((size_t)nq * k);
      std::vector<float> cs((size_t)nq * k);
      // running top-k per query
      std::vector<int32_t> bi((size_t)nq * k, -1);
      std::vector<float> bs((size_t)nq * k, -INFINITY);
      std::vector<std::pair<float, int32_t>> tmp;
      for (int64_t d0 = 0; d0 < ix->D && !st; d0 += kChunk) {
        k_iota_rows<<<256, 256, 0, s>>>(cand, nq, d0, ix->D);
        if (cudaGetLastError() != cudaSuccess) {
          st = fail(TACHIOM_ERR_CUDA, "exhaustive top-k: launch failed");
          break;
        }
        if ((st = tachiom_refine(index, &p, d_queries, h_ntok, kk.data(), nq, cand, oi, os, stream))) break;
        if (cudaMemcpyAsync(ci.data(), oi, ci.size() * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(cs.data(), os, cs.size() * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
          st = fail(TACHIOM_ERR_CUDA, "exhaustive top-k: copy failed");
          break;
        }
        for (int q = 0; q < nq; q++) {
          tmp.clear();
          for (int u = 0; u < k; u++) {
            const size_t a = (size_t)q * k + u;
            if (bi[a] >= 0) tmp.emplace_back(bs[a], bi[a]);
            if (ci[a] >= 0) tmp.emplace_back(cs[a], ci[a]);
          }
          std::sort(tmp.begin(), tmp.end(), [](const std::pair<float, int32_t> &x, const std::pair<float, int32_t> &y) {
            return better(x.first, x.second, y.first, y.second);
          });
          for (int u = 0; u < k; u++) {
            const size_t a = (size_t)q * k + u;
            if (u < (int)tmp.size()) {
              bs[a] = tmp[u].first;
              bi[a] = tmp[u].second;
            } else {
              bs[a] = -INFINITY;
              bi[a] = -1;
            }
          }
        }
      }
      if (!st) {
        memcpy(h_ids, bi.data(), bi.size() * 4);
        memcpy(h_scores, bs.data(), bs.size() * 4);
      }
    }
  }
  if (prev >= 0 && prev != ix->device) cudaSetDevice(prev);
  return st;
}

extern "C" tachiom_status tachiom_autotune_budgets(tachiom_index *index, int32_t precision, const float *d_queries,
                                                   const int32_t *h_ntok, int32_t nq, int32_t k,
                                                   const int32_t *h_grid_kc, int32_t n_kc, const int32_t *h_grid_kd,
                                                   int32_t n_kd, float min_recall, int32_t *best_kc, int32_t *best_kd,
                                                   float *best_recall, float *best_ms, float *h_table,
                                                   void *stream) {
  Index *ix = reinterpret_cast<Index *>(index);
  if (!ix || !d_queries || !h_ntok || !h_grid_kc || !h_grid_kd || !best_kc || !best_kd)
    return fail(TACHIOM_ERR_INVALID, "NULL argument");
  if (nq < 1 || nq > 4096 || k < 1 || k > 1000 || n_kc < 1 || n_kd < 1 || n_kc * n_kd > 256)
    return fail(TACHIOM_ERR_INVALID, "bad sizes");
  for (int i = 0; i < n_kc; i++)
    if (h_grid_kc[i] < 1 || h_grid_kc[i] > MAX_KC) return fail(TACHIOM_ERR_INVALID, "kappa_c grid value out of range");
  for (int i = 0; i < n_kd; i++)
    if (h_grid_kd[i] < k || h_grid_kd[i] > MAX_KD) return fail(TACHIOM_ERR_INVALID, "kappa_d grid value out of [k, 4096]");
  tachiom_status st;
  // the exhaustive reference
  std::vector<int32_t> ref((size_t)nq * k);
  std::vector<float> refs((size_t)nq * k);
  if ((st = tachiom_exhaustive_topk(index, precision, d_queries, h_ntok, nq, k, ref.data(), refs.data(), stream)))
    return st;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ix->device) cudaSetDevice(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  {
    DevBufs B;
    int32_t *oi = nullptr;
    float *os = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    st = B.alloc(&oi, (size_t)nq * k);
    if (!st) st = B.alloc(&os, (size_t)nq * k);
    if (!st && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
      st = fail(TACHIOM_ERR_CUDA, "autotune events");
    std::vector<int32_t> kk((size_t)nq, k), got((size_t)nq * k);
    int bkc = -1, bkd = -1;
    float brec = -1.f, bms = 0.f;
    bool bok = false;
    for (int a = 0; a < n_kc && !st; a++)
      for (int b = 0; b < n_kd && !st; b++) {
        tachiom_search_params p{};
        p.kappa_c = h_grid_kc[a];
        p.kappa_d = h_grid_kd[b];
        p.precision = precision;
        p.plan_id = -1;
        // one run sizes the scratch and gives the result, three are timed
        if ((st = tachiom_search(index, &p, d_queries, h_ntok, kk.data(), nq, oi, os, stream))) break;
        if (cudaMemcpyAsync(got.data(), oi, got.size() * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
          st = fail(TACHIOM_ERR_CUDA, "autotune copy");
          break;
        }
        float ms[3];
        for (int r = 0; r < 3 && !st; r++) {
          cudaEventRecord(e0, s);
          st = tachiom_search(index, &p, d_queries, h_ntok, kk.data(), nq, oi, os, stream);
          cudaEventRecord(e1, s);
          if (!st && cudaEventSynchronize(e1) != cudaSuccess) st = fail(TACHIOM_ERR_CUDA, "autotune timing");
          if (!st) cudaEventElapsedTime(&ms[r], e0, e1);
        }
        if (st) break;
        std::sort(ms, ms + 3);
        // recall@k: the share of the exhaustive top-k found
        int64_t hit = 0, tot = 0;
        for (int q = 0; q < nq; q++) {
          const int32_t *rq = ref.data() + (size_t)q * k, *gq = got.data() + (size_t)q * k;
          for (int u = 0; u < k; u++) {
            if (rq[u] < 0) continue;
            tot++;
            for (int v = 0; v < k; v++)
              if (gq[v] == rq[u]) {
                hit++;
                break;
              }
          }
        }
        const float rec = tot ? (float)hit / (float)tot : 1.f;
        if (h_table) {
          float *row = h_table + (size_t)(a * n_kd + b) * 4;
          row[0] = (float)p.kappa_c;
          row[1] = (float)p.kappa_d;
          row[2] = rec;
          row[3] = ms[1];
        }
        const bool ok = rec >= min_recall;
        bool take;
        if (bkc < 0) take = true;
        else if (ok != bok) take = ok;
        else if (ok) take = ms[1] < bms;
        else take = rec > brec || (rec == brec && ms[1] < bms);
        if (take) {
          bkc = p.kappa_c;
          bkd = p.kappa_d;
          brec = rec;
          bms = ms[1];
          bok = ok;
        }
      }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (!st) {
      *best_kc = bkc;
      *best_kd = bkd;
      if (best_recall) *best_recall = brec;
      if (best_ms) *best_ms = bms;
    }
  }
  if (prev >= 0 && prev != ix->device) cudaSetDevice(prev);
  return st;
}
