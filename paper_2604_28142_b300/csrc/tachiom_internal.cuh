// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "../../include/tachiom.h"

namespace tachiom {

constexpr int DIM = 128;
constexpr int MAX_NTOK = 32;   // query tokens per query
constexpr int MAX_KC = 128;    // kappa_c
constexpr int MAX_KD = 4096;   // kappa_d
constexpr int SEL_CAP = 16384; // candidates a query's exact kappa_d selection takes at once

// ---- errors -----------------------------------------------------------------
void set_error(const char *fmt, ...);
tachiom_status fail(tachiom_status st, const char *fmt, ...);

#define TCUDA(call)                                                                    \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return ::tachiom::fail(TACHIOM_ERR_CUDA, "%s failed: %s (%s:%d)", #call,         \
                             cudaGetErrorString(e_), __FILE__, __LINE__);              \
  } while (0)

#define TLAUNCH()                                                                      \
  do {                                                                                 \
    cudaError_t e_ = cudaGetLastError();                                               \
    if (e_ != cudaSuccess)                                                             \
      return ::tachiom::fail(TACHIOM_ERR_CUDA, "kernel launch failed: %s (%s:%d)",     \
                             cudaGetErrorString(e_), __FILE__, __LINE__);              \
  } while (0)

// ---- ordered keys --------------------------------------------------------------
// fkey maps float order onto uint32 order (0 is never produced: it marks "empty").
__device__ __forceinline__ uint32_t fkey(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float funkey(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(u);
}
// (score desc, id asc) as one descending uint64; 0 sorts after every real entry.
__device__ __forceinline__ uint64_t comp_key(float s, int32_t id) {
  return ((uint64_t)fkey(s) << 32) | (uint32_t)(~(uint32_t)id);
}
__device__ __forceinline__ int32_t comp_id(uint64_t c) { return (int32_t)(~(uint32_t)(c & 0xffffffffu)); }
__device__ __forceinline__ float comp_score(uint64_t c) { return funkey((uint32_t)(c >> 32)); }

// Descending bitonic sort of n (power of two) uint64 in shared memory by the whole block.
__device__ __forceinline__ void block_sort_desc(uint64_t *a, int n) {
  for (int k = 2; k <= n; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int l = i ^ j;
        if (l > i) {
          uint64_t x = a[i], y = a[l];
          bool desc = (i & k) == 0;
          if (desc ? (x < y) : (x > y)) { a[i] = y; a[l] = x; }
        }
      }
      __syncthreads();
    }
}

// Same, by one warp (lane stride), for n <= a few hundred.
__device__ __forceinline__ void warp_sort_desc(uint64_t *a, int n) {
  const int lane = threadIdx.x & 31;
  for (int k = 2; k <= n; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < n; i += 32) {
        int l = i ^ j;
        if (l > i) {
          uint64_t x = a[i], y = a[l];
          bool desc = (i & k) == 0;
          if (desc ? (x < y) : (x > y)) { a[i] = y; a[l] = x; }
        }
      }
      __syncwarp();
    }
}

// The kappa-th largest of the n distinct keys a[0..n) (1 <= kappa <= n), to every thread:
// a radix select over 11-bit digits from the top (bits 63..53, 52..42, ...); once the digit
// holding the cut has at most 64 keys, one warp sorts those. The bins are scanned from the top
// by the whole block (thread t owns a contiguous run of bins). Uses hist[2048], small[64],
// wsum[32] and sh[8]; ends with a barrier.
constexpr int KSEL_BITS = 11;
__device__ __forceinline__ uint64_t block_kth_largest(const uint64_t *a, int n, int kappa, uint32_t *hist, uint64_t *small,
                                   uint32_t *wsum, uint32_t *sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  uint64_t prefix = 0ull, mask = 0ull;
  uint32_t need = (uint32_t)kappa;
  for (int top = 64; top > 0; top -= KSEL_BITS) {
    const int shift = max(0, top - KSEL_BITS), bits = top - shift, nbin = 1 << bits;
    const uint64_t dmask = (uint64_t)(nbin - 1);
    for (int i = tid; i < nbin; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    for (int i0 = 0; i0 < n; i0 += blockDim.x) {
      const int i = i0 + tid;
      int dg = -1;
      if (i < n) {
        const uint64_t k = a[i];
        if ((k & mask) == prefix) dg = (int)((k >> shift) & dmask);
      }
      const unsigned peers = __match_any_sync(0xffffffffu, dg);
      if (dg >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[dg], (uint32_t)__popc(peers));
    }
    __syncthreads();
    // thread t: bins [hi - w, hi), hi = nbin - t w, counted from the top
    const int w = (nbin + blockDim.x - 1) / blockDim.x;
    const int bhi = max(0, nbin - tid * w), blo = max(0, bhi - w);
    uint32_t c = 0;
    for (int d = blo; d < bhi; d++) c += hist[d];
    uint32_t inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    uint32_t before = 0;
    for (int u = 0; u < warp; u++) before += wsum[u];
    (void)nw;
    const uint32_t excl = before + inc - c;
    inc += before;
    if (c > 0 && excl < need && need <= inc) {
      uint32_t cum = excl;
      int d = bhi - 1;
      for (; d > blo; d--) {
        if (cum + hist[d] >= need) break;
        cum += hist[d];
      }
      sh[0] = (uint32_t)d;
      sh[1] = need - cum;
      sh[2] = hist[d];
      sh[3] = 0u;
    }
    __syncthreads();
    prefix |= (uint64_t)sh[0] << shift;
    mask |= dmask << shift;
    need = sh[1];
    const uint32_t inbin = sh[2];
    if (inbin <= 64u) {
      // gather the bin's keys and pick the need-th largest
      for (int i0 = 0; i0 < n; i0 += blockDim.x) {
        const int i = i0 + tid;
        if (i < n && (a[i] & mask) == prefix) {
          const uint32_t d = atomicAdd(&sh[3], 1u);
          if (d < 64u) small[d] = a[i];
        }
      }
      __syncthreads();
      if (warp == 0) {
        for (int i = (int)inbin + lane; i < 64; i += 32) small[i] = 0ull;
        __syncwarp();
        warp_sort_desc(small, 64);
      }
      __syncthreads();
      const uint64_t r = small[need - 1];
      __syncthreads();  // small, wsum and sh are free again when this returns
      return r;
    }
    __syncthreads();  // sh and wsum are read by every thread before the next pass rewrites them
  }
  return prefix;  // not reached: distinct keys leave a single key in the last digit's bin
}

__host__ __device__ inline int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// ---- index ------------------------------------------------------------------------
struct Workspace;

struct Index {
  int device = 0;
  int64_t C = 0, D = 0, T = 0;
  int M = 16, ds = 8;
  int cdtype = TACHIOM_DTYPE_F32;
  float *cent_f32 = nullptr;            // [C x 128] FP32 values of the stored centroids
  __nv_bfloat16 *cent_bf16 = nullptr;   // [C x 128] BF16 operand of the tensor-core path
  float cnorm_max = 0.f;                // max_j ||c_j|| (error bound of the BF16 path)
  float cerr_max = 0.f;                 // max_j ||bf16(c_j) - c_j|| (0 for a BF16-stored table)
  uint8_t *cent_e4m3 = nullptr;         // [C x 128] E4M3 operand: c_j * 2^k_j rounded (power-of-two row scale)
  float *cent_inv_sc = nullptr;         // [C] 2^-k_j
  float cerr8_max = 0.f;                // max_j ||e4m3(c_j) 2^-k_j - c_j||
  int32_t *cent_type = nullptr;         // [C] or null
  int64_t *doc_off = nullptr;           // [D+1]
  int32_t *tok_cid = nullptr;           // [T]
  uint8_t *codes = nullptr;             // [T x M]
  uint16_t *rnorm = nullptr;            // [T] fp16 bits (1.0 everywhere when absent)
  float *codebooks = nullptr;           // [M x 256 x ds]
  float2 *doc_xe = nullptr;             // [D] per document, max over its tokens of the decode pass's
                                        // ||h(x~_t)|| and ||e_x,t|| bounds (k_doc_decode_norms)
  uint16_t *cbk_h16 = nullptr;          // [M x 256 x ds] fp16 codewords in the decode pass's layout
  float *cbk_err2 = nullptr;            // [M x 256] squared norm of each codeword's fp16 rounding error
  int64_t *list_off = nullptr;          // [C+1]
  int32_t *list_doc = nullptr;          // [n_list]
  int64_t n_list = 0;
  int range_docs = 0;                   // documents per gather range (<= 2^20)
  int n_ranges = 0;
  int32_t *list_roff = nullptr;         // [C x (n_ranges+1)] offset in L_j of the first doc
                                        // of each range
  size_t device_bytes = 0;
  std::mutex mu;
  std::unordered_map<cudaStream_t, Workspace *> ws;
};

// scratch of one stream, grown on demand
struct Workspace {
  cudaStream_t stream = nullptr;
  int device = 0;
  std::vector<void *> blocks;          // device allocations, freed with the workspace
  // capacities
  int64_t cap_rows = 0, cap_q = 0, cap_kc = 0, cap_kd = 0, cap_split_entries = 0;
  int64_t cap_pool = 0;
  // device buffers
  int32_t *d_meta = nullptr;           // qoff [B+1] | koff [B+1] | k [B] | ntok [B]
  float *d_rows_f32 = nullptr;         // staging of host queries (search_host)
  __nv_bfloat16 *d_rows_bf16 = nullptr;// [rows x 128]
  uint8_t *d_rows_f8 = nullptr;        // [rows x 128] E4M3 rows (power-of-two row scale)
  float *d_inv_sq = nullptr;           // [rows] their scales 2^-k
  uint64_t *d_split = nullptr;         // [rows x splits x capout] candidates of step (a)
  uint32_t *d_gmax = nullptr;          // tensor-core path: the sample pass's per-stream top group maxima
  uint32_t *d_tau = nullptr;           // tensor-core path: per-row lower bound of the cut
  float *d_margin = nullptr;           // tensor-core path: per-row repair window (twice the error bound)
  int32_t *d_glist = nullptr;          // tensor-core path: candidate centroids per row, then per-row thresholds
  int32_t *d_gcount = nullptr;         // tensor-core path: number of candidates per row
  int32_t *d_lossy = nullptr;          // rows recomputed by the full FP32 scan
  int64_t cap_gmax = 0;
  int32_t *d_split_cnt = nullptr;      // [rows x splits]
  int32_t *d_top_ids = nullptr;        // [rows x kc]
  float *d_top_s = nullptr;            // [rows x kc]
  uint64_t *d_pool = nullptr;          // [B x groups x kd] each range group's top-kappa_d (S~, doc) keys
  int32_t *d_pool_n = nullptr;         // [B x groups] their counts
  int32_t *d_cand = nullptr;           // [B x kd]
  float *d_cand_s = nullptr;           // [B x kd]
  int32_t *d_ncand = nullptr;          // [B]
  float *d_part = nullptr;             // [B x groups x kd] refine partial sums
  int32_t *d_win = nullptr;            // [B x kd] FP32 rescoring window of the tensor-core refine
  int32_t *d_win_slot = nullptr;       // [B x kd] each window entry's candidate slot
  float *d_thr = nullptr;              // [B x kd x 32] per (slot, query token) thresholds of the window pass
  int2 *d_wl = nullptr;                // [B x WL_PER_QUERY] candidate pairs of the window pass
  unsigned long long *d_wl_n = nullptr;  // pairs offered to the list (64-bit: it keeps counting past the cap)
  uint32_t *d_emx = nullptr;           // [B x kd x 32] their exact maxima
  int32_t *d_wovf = nullptr;           // [B x kd] documents left to the all-pairs FP32 kernel
  int32_t *d_out_ids = nullptr;        // staging for search_host
  float *d_out_s = nullptr;
  uint32_t *d_flags = nullptr;         // status word
  // host pinned staging
  int32_t *h_meta = nullptr;
  int64_t cap_meta = 0;
  float *h_rows = nullptr;
  int64_t cap_h_rows = 0;
  int32_t *h_out_ids = nullptr;
  float *h_out_s = nullptr;
  int64_t cap_h_out = 0;
  cudaEvent_t meta_done = nullptr;     // host staging reusable once this fires
};

// lifecycle helpers (search.cu)
tachiom_status ws_get(Index *ix, cudaStream_t stream, Workspace **out);
void ws_destroy(Workspace *w);
void ws_release(Index *ix, cudaStream_t stream);  // free a stream's scratch (the stream is idle)

// ---- per-launcher timing (tachiom_profile_enable) -----------------------------------
class ProfScope {
 public:
  ProfScope(const char *name, cudaStream_t s);
  ~ProfScope();

 private:
  const char *name_;
  cudaStream_t s_;
  void *a_;
};
#define TPROF_CAT2(a, b) a##b
#define TPROF_CAT(a, b) TPROF_CAT2(a, b)
#define TPROF(name, s) ::tachiom::ProfScope TPROF_CAT(prof_scope_, __LINE__)(name, s)

// ---- kernel launchers (one per translation unit) -----------------------------------
// step (a)
tachiom_status launch_quantize_bf16(const float *rows, __nv_bfloat16 *out, int64_t n, cudaStream_t s);
tachiom_status launch_topc_f32(const Index &ix, const float *rows, int nrows, int kc, int splits,
                               int capout, uint64_t *split, int32_t *split_cnt, uint32_t *flags,
                               cudaStream_t s);
tachiom_status launch_topc_merge(const Index &ix, const float *rows, int nrows, int kc, int splits,
                                 int capout, const uint64_t *split, const int32_t *split_cnt,
                                 const float *margins, int rescore, int32_t *top_ids, float *top_s,
                                 uint32_t *flags, cudaStream_t s);
tachiom_status launch_quantize_rows(const Index &ix, const float *rows, __nv_bfloat16 *out, int nrows,
                                    float *margins, cudaStream_t s);
// E4M3 rows with a power-of-two scale per row, and per row 2 lambda times the rigorous bound of
// the E4M3 score error (the repair window of the E4M3 step (a))
tachiom_status launch_quantize_e4m3(const Index &ix, const float *rows, int nrows, uint8_t *out, float *inv,
                                    float lambda, float *margins, cudaStream_t s);
// the index's E4M3 centroid copy (index load)
tachiom_status launch_cent_e4m3(Index &ix, cudaStream_t s);
// tensor-core step (a): rows_q BF16 (f8 false: group selection) or E4M3 with inv_sq (sample,
// emission); gmax_tops, glist and gcount are scratch (topc_tc_gmax_elems, topc_tc_glist_elems,
// rows); gcount receives the kept groups (BF16) or the candidates (E4M3) of every row
tachiom_status launch_topc_tc(const Index &ix, const void *rows_q, const float *inv_sq, bool f8, const float *rows,
                              int nrows, int kc, const float *margins, float *gmax_tops, int32_t *glist, int32_t *gcount,
                              int32_t *lossy_rows, int32_t *top_ids, float *top_s, uint32_t *flags, cudaStream_t s);
tachiom_status launch_topc_rescue(const Index &ix, const float *rows, int nrows, int kc, const int32_t *lossy_rows,
                                  int32_t *top_ids, float *top_s, cudaStream_t s);
size_t topc_tc_glist_elems(int rows);
int topc_tc_supported();
tachiom_status launch_topc_tc_raw(const Index &ix, const void *rows_q, const float *inv_sq, bool f8, int nrows,
                                  float *out, uint32_t *flags, cudaStream_t s);
// diagnostics: a tensor-core pass whose producer withholds every copy, waits limited to wait_ns
tachiom_status launch_topc_tc_wait_test(const Index &ix, const void *rows_q, uint64_t wait_ns, float *tops,
                                        uint32_t *flags, cudaStream_t s);
tachiom_status launch_topc_tc1(const Index &ix, const __nv_bfloat16 *rows, int nrows, int kc, const float *margins,
                               uint64_t *split_out, int32_t *split_cnt, uint32_t *flags, cudaStream_t s);
int topc_tc1_capout();
int topc_tc1_max_kc();
int topc_tc1_splits(const Index &ix, int nrows);
size_t topc_tc_gmax_elems(const Index &ix, int rows);
tachiom_status launch_score_pairs(const Index &ix, const float *rows, int nrows, const int32_t *ids,
                                  int kc, int32_t *out_ids, float *scores, uint32_t *flags, cudaStream_t s);
// step (b): per (query, range group) the group's top-kappa_d keys into pool, then per query the
// exact top-kappa_d of its groups' parts
// range groups per query of step (b); groups > 0 (a plan's choice) asks for 2 x groups
int gather_groups(const Index &ix, int nq, int kd, int groups);
size_t gather_pool_elems(const Index &ix, int nq, int kd);
tachiom_status launch_gather(const Index &ix, const int32_t *meta, int nq, const int32_t *top_ids, const float *top_s,
                             int kc, int kd, uint64_t *pool, int32_t *pool_n, bool force_split, int groups,
                             uint32_t *flags, cudaStream_t s);
tachiom_status launch_select_kd(const Index &ix, const int32_t *meta, int nq, int kd, const uint64_t *pool,
                                const int32_t *pool_n, int groups, int32_t *cand, float *cand_s, int32_t *ncand,
                                cudaStream_t s);
// steps (c), (d)
tachiom_status launch_refine_win(const Index &ix, const float *queries, const int32_t *meta, int nq,
                                 const int32_t *cand, int kd, float *part, uint32_t *flags, cudaStream_t s);
// centroid_only: every residual norm taken as 0, so the partial sums are the full centroid
// interaction sum_i max_{t in d} <q_i, c_a(t)>
tachiom_status launch_refine(const Index &ix, const float *queries, const int32_t *meta, int nq,
                             const int32_t *cand, int kd, float *part, uint32_t *flags,
                             cudaStream_t s, bool centroid_only = false);
tachiom_status launch_final_topk(const Index &ix, const int32_t *meta, int nq, const int32_t *cand,
                                 int kd, const float *part, int32_t *out_ids, float *out_s,
                                 cudaStream_t s);
int refine_groups(int M);
tachiom_status launch_refine_tc(const Index &ix, const float *queries, const int32_t *meta, int nq,
                                const int32_t *cand, int kd, float *part, uint32_t *flags, cudaStream_t s);
tachiom_status launch_refine_dec(const Index &ix, const float *queries, const int32_t *meta, int nq,
                                 const int32_t *cand, int kd, float *sa, float *da, float *thr, uint32_t *flags,
                                 cudaStream_t s);
// fills ix.cbk_h16, ix.cbk_err2 and ix.doc_xe (allocated by the caller) from the index's codebooks,
// codes, norms and BF16 centroids: the tables of the decode pass of step (c)
tachiom_status launch_decode_tables(const Index &ix, cudaStream_t s);
// scratch of the window pass: the candidate pairs, their exact maxima, the overflowed documents
constexpr int WL_PER_QUERY = 8192;  // candidate pairs a query's window may list
struct WinScratch {
  int2 *wl;
  unsigned long long *wl_n;
  int wl_cap;
  uint32_t *emx;   // [B x kd x 32]
  int32_t *wovf;   // [B x kd]
};
tachiom_status launch_refine_dec_win(const Index &ix, const float *queries, const int32_t *meta, int nq,
                                     const int32_t *win, const int32_t *win_slot, int kd, float *thr, float *part,
                                     const WinScratch &ws, uint32_t *flags, cudaStream_t s);
tachiom_status launch_refine_win_only(const Index &ix, const float *queries, const int32_t *meta, int nq,
                                      const int32_t *cand, int kd, const int32_t *only, float *part,
                                      uint32_t *flags, cudaStream_t s);
tachiom_status launch_refine_window_b(const Index &ix, const int32_t *meta, int nq, const int32_t *cand, int kd,
                                      const float *sa, const float *da, int32_t *win, int32_t *win_slot,
                                      cudaStream_t s);
tachiom_status launch_refine_sum(const Index &ix, const int32_t *meta, int nq, const int32_t *cand, int kd,
                                 const float *part, float *out, cudaStream_t s);
tachiom_status launch_refine_window(const Index &ix, const int32_t *meta, int nq, const int32_t *cand, int kd,
                                    const float *part, float delta_per_token, int32_t *win, cudaStream_t s);

}  // namespace tachiom
