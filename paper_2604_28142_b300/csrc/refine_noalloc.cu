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
// metadata and a status word: 2 MiB + 4 KiB, resident on every device that
// loads the library until the process exits. Every call uses the same array;
// nothing in it has to start at zero (each call writes every entry it later
// reads) except the status word, which is zero at load and cleared by
// tachiom_refine_noalloc_status. The per-query metadata is staged on the host
// in one file-scope array (no heap, no stack buffer handed to the copy engine).
// Calls whose work overlaps on the GPU (different streams, or different host
// threads) race on both arrays. The refine always scores in FP32 (the FP32
// lookup-table kernel), whatever params->precision says.
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
constexpr int kMetaInts = 4 * kMaxQueries + 2;  // qoff [nq+1] | koff [nq+1] | k [nq] | ntok [nq]
// the group count of the FP32 refine at the widest pq_m (32) and the longest query
static_assert(kMaxGroups >= (MAX_NTOK + 3) / 4, "partial-sum region too small for pq_m = 32");
// the metadata ends below the status word at kMetaBytes - 256
static_assert((size_t)kMetaInts * sizeof(int32_t) <= kMetaBytes - 256, "metadata overlaps the status word");

static int32_t g_meta_host[kMetaInts];  // host staging of the metadata (shared by every call)

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
  if (params->precision != TACHIOM_PREC_FP32 && params->precision != TACHIOM_PREC_BF16 &&
      params->precision != TACHIOM_PREC_FP8)
    return fail(TACHIOM_ERR_INVALID, "unknown precision %d", params->precision);
  if (refine_groups(ix->M) > kMaxGroups)
    return fail(TACHIOM_ERR_CAPACITY, "tachiom_refine_noalloc: pq_m = %d needs more partial sums than the static array",
                ix->M);
  const int kd = params->kappa_d;
  // per-query metadata in the file-scope host array (no heap): qoff | koff | k | ntok
  int32_t *meta = g_meta_host;
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
    // pageable source: the copy is staged before the call returns
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

extern "C" tachiom_status tachiom_refine_noalloc_status(tachiom_index *index, void *stream, uint32_t *h_flags) {
  Index *ix = reinterpret_cast<Index *>(index);
  if (!ix || !h_flags) return fail(TACHIOM_ERR_INVALID, "NULL argument");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ix->device && cudaSetDevice(ix->device) != cudaSuccess)
    return fail(TACHIOM_ERR_CUDA, "cudaSetDevice(%d) failed", ix->device);
  tachiom_status st = TACHIOM_OK;
  unsigned char *base = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  if (!(st = scratch_address(ix->device, &base))) {
    uint32_t *dflags = reinterpret_cast<uint32_t *>(base + kPartBytes + kMetaBytes - 256);
    uint32_t v = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&v, dflags, sizeof(v), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dflags, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = fail(TACHIOM_ERR_CUDA, "status word read failed: %s", cudaGetErrorString(e));
    else *h_flags = v;
  }
  if (prev >= 0 && prev != ix->device) cudaSetDevice(prev);
  return st;
}
