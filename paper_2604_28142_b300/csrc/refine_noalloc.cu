// Steps (c)-(d) on caller-given candidates without any allocation.
//
// Who needs this: callers that must not allocate device memory while they
// run, e.g. a host process whose device memory is carved up in advance by a
// fixed-budget allocator, a plug-in that runs inside another framework's
// memory pool, or a real-time thread that may not block in cudaMalloc (which
// can synchronise the device). tachiom_refine takes its scratch (per-query
// metadata and per-group partial sums) from a per-stream workspace that the
// library grows with cudaMalloc; this variant takes it from one file-scope
// device array instead, so a call allocates nothing: no cudaMalloc, no
// cudaFree, no pinned host buffer, no heap.
//
// The array holds at most kMaxQueries queries of kMaxKd candidates each (the
// partial sums of up to 8 query-token groups per candidate) plus the query
// metadata: 2 MiB + 4 KiB, resident on every device that loads the library
// until the process exits. Every call uses the same array; nothing in it has
// to start at zero (each call writes every entry it later reads), and calls
// whose work overlaps on the GPU (different streams, or different host
// threads) race on it.
#include <mutex>

#include "tachiom_internal.cuh"

namespace tachiom {
namespace {

constexpr int kMaxQueries = 64;
constexpr int kMaxKd = 1024;
constexpr int kMaxGroups = 8;  // query-token groups of k_refine at pq_m = 32
constexpr size_t kPartBytes = (size_t)kMaxQueries * kMaxGroups * kMaxKd * sizeof(float);
constexpr size_t kMetaBytes = 4096;  // >= (4 * kMaxQueries + 2) int32 + the status word
constexpr size_t kScratchBytes = kPartBytes + kMetaBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// device address of g_noalloc_scratch, looked up once per device
std::mutex g_mu;
void *g_addr[64] = {nullptr};

tachiom_status scratch_address(int dev, unsigned char **out) {
  if (dev < 0 || dev >= 64) return fail(TACHIOM_ERR_INVALID, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // the device is current here
    if (e != cudaSuccess || !p)
      return fail(TACHIOM_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                  cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = static_cast<unsigned char *>(g_addr[dev]);
  return TACHIOM_OK;
}

}  // namespace
}  // namespace tachiom

using namespace tachiom;

extern "C" tachiom_status tachiom_refine_noalloc(tachiom_index *index, const tachiom_search_params *params,
                                                 const float *d_queries, const int32_t *h_ntok,
                                                 const int32_t *h_k, int32_t nq, const int32_t *d_cand_ids,
                                                 int32_t *d_out_ids, float *d_out_scores, void *stream) {
  Index *ix = reinterpret_cast<Index *>(index);
  if (!ix) return fail(TACHIOM_ERR_INVALID, "index is NULL");
  if (!params) return fail(TACHIOM_ERR_INVALID, "params is NULL");
  if (nq < 0) return fail(TACHIOM_ERR_INVALID, "nq < 0");
  if (nq == 0) return TACHIOM_OK;
  if (nq > kMaxQueries)
    return fail(TACHIOM_ERR_CAPACITY, "tachiom_refine_noalloc: nq = %d exceeds the static maximum of %d queries",
                nq, kMaxQueries);
  if (params->kappa_d < 1 || params->kappa_d > kMaxKd)
    return fail(TACHIOM_ERR_CAPACITY,
                "tachiom_refine_noalloc: kappa_d = %d must be given explicitly, 1..%d (static maximum)",
                params->kappa_d, kMaxKd);
  if (!h_ntok || !h_k || !d_queries || !d_cand_ids || !d_out_ids || !d_out_scores)
    return fail(TACHIOM_ERR_INVALID, "NULL argument");
  const int kd = params->kappa_d;
  // per-query metadata in a fixed-size host array (no heap): qoff | koff | k | ntok
  int32_t meta[4 * kMaxQueries + 2];
  meta[0] = 0;
  meta[nq + 1] = 0;
  for (int i = 0; i < nq; i++) {
    if (h_ntok[i] < 1 || h_ntok[i] > MAX_NTOK)
      return fail(TACHIOM_ERR_INVALID, "ntok[%d] = %d out of [1, %d]", i, h_ntok[i], MAX_NTOK);
    if (h_k[i] < 1 || h_k[i] > kd) return fail(TACHIOM_ERR_INVALID, "k[%d] = %d out of [1, kappa_d]", i, h_k[i]);
    meta[i + 1] = meta[i] + h_ntok[i];
    meta[nq + 2 + i] = meta[nq + 1 + i] + h_k[i];
    meta[2 * nq + 2 + i] = h_k[i];
    meta[3 * nq + 2 + i] = h_ntok[i];
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ix->device && cudaSetDevice(ix->device) != cudaSuccess)
    return fail(TACHIOM_ERR_CUDA, "cudaSetDevice(%d) failed", ix->device);
  tachiom_status st = TACHIOM_OK;
  unsigned char *base = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  if (!(st = scratch_address(ix->device, &base))) {
    float *part = reinterpret_cast<float *>(base);
    int32_t *dmeta = reinterpret_cast<int32_t *>(base + kPartBytes);
    uint32_t *dflags = reinterpret_cast<uint32_t *>(base + kPartBytes + kMetaBytes - 256);
    // pageable source: the call returns once `meta` has been staged, so the stack array may go
    cudaError_t e = cudaMemcpyAsync(dmeta, meta, (size_t)(4 * nq + 2) * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      st = fail(TACHIOM_ERR_CUDA, "metadata copy failed: %s", cudaGetErrorString(e));
    } else if (!(st = launch_refine(*ix, d_queries, dmeta, nq, d_cand_ids, kd, part, dflags, s))) {
      st = launch_final_topk(*ix, dmeta, nq, d_cand_ids, kd, part, d_out_ids, d_out_scores, s);
    }
  }
  if (prev >= 0 && prev != ix->device) cudaSetDevice(prev);
  return st;
}
