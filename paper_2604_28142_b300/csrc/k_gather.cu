// Step (b): inverted-list gather and centroid-only late interaction
// (Sec. 2.2, Gather steps 2-4), then the kappa_d truncation.
//
// The documents are cut into ranges of R consecutive ids, and a per-(list,
// range) offset table locates the slice of every L_j that starts at a range
// boundary. k_gather_pool runs one CTA per (group of consecutive ranges,
// query). It walks its group's documents in pieces [d0, d1): a piece's slice
// of every list L_{Top_i[u]} comes from the table (binary search inside a range
// for an unaligned bound), and a piece with more list entries than the key
// buffers hold is cut into up to 8 pieces, recursively, so the pieces follow
// the density of the query's entries (a piece spans at most 2^20 ids; one
// document always fits, with at most one entry per list). For each piece it
//   1. turns each list entry into the 32-bit key
//          (d - d0) << 12 | i << 7 | u            (d - d0 < 2^20, i < 32, u < 128);
//   2. sorts the keys by document in shared memory: a counting sort on the
//      document bits (a few keys per bucket), then every key takes its place
//      in its bucket by counting the bucket's smaller keys, so a document's
//      keys are one run ordered by (token, rank);
//   3. for every reached document forms
//          S~(q, d) = sum over the run's tokens, ascending i, of the score of
//                     the token's first (best-ranked) key,
//      the FP32 sums of the token-serial definition, since Top_i is sorted by
//      (score desc, id asc), and keeps (S~, d) if it beats the group's
//      running cut.
// The group's candidates live in a shared-memory buffer. When the next piece
// could overflow it, an exact block-wide radix select finds the kappa_d-th
// largest key, the buffer keeps the kappa_d keys at or above it, and that key
// becomes the running cut (keys are unique: the document id is part of them).
// A group thus ends with its exact top-kappa_d by (S~ desc, doc asc), and the
// union of a query's groups holds the query's top-kappa_d. The scratch is one
// kappa_d-sized part per (query, group): it follows the hits, not the number
// of documents.
//
// k_pool_select: per query, the exact top-kappa_d of the union of its parts.
#include <algorithm>

#include "tachiom_internal.cuh"

namespace tachiom {

constexpr int GP_THREADS = 512;
constexpr int GP_NB_BITS = 11;                 // at most 2^11 buckets per piece
constexpr int GP_NB_MAX = 1 << GP_NB_BITS;
constexpr int GP_ECAP_MIN = 2048;              // key buffers always hold a whole document and
                                               // the compaction's slot list (kappa_d <= 2 * ecap)
constexpr int GP_ECAP_MAX = 8192;
constexpr int GP_SMEM_TWO_PER_SM = 106 * 1024; // two CTAs per SM when the layout fits this (with
                                               // the static shared memory and the 1 KB per CTA
                                               // the hardware reserves: 228 KB per SM)
constexpr int GP_SMEM_MAX = 227 * 1024;
constexpr int GP_STACK = 64;                   // pending pieces of a split chunk (<= 7 levels x 7 + 1)
constexpr int GP_SPT = 8;                      // segments per thread: 32 tokens x 128 ranks / 512
constexpr int GP_XMAX = 1 << 20;               // documents a piece may span (20-bit offsets in the keys)
constexpr int GP_SPLIT_FORCED = 256;           // piece size when every range is split (test plan)

__device__ __forceinline__ int ceil_log2(uint32_t v) { return v <= 1 ? 0 : 32 - __clz(v - 1); }

struct GpSmem {
  int32_t *j;       // [nseg] centroid of segment (i, u), -1 if none
  int32_t *base;    // [nseg] position of L_j in list_doc
  float *sc;        // [nseg] <q_i, c_j>
  int32_t *start;   // [nseg] first list position of the current piece
  uint32_t *pref;   // [nseg] piece length, then its exclusive prefix
  uint32_t *cnt;    // [GP_NB_MAX] bucket counts, then cursors
  uint32_t *kin;    // [ecap]
  uint32_t *kout;   // [ecap]
  uint64_t *lbuf;   // [lbcap] the group's candidates
};

__host__ __device__ inline size_t gp_smem_bytes(int nseg_max, int ecap, int lbcap) {
  return (size_t)nseg_max * 20 + (size_t)GP_NB_MAX * 4 + (size_t)ecap * 8 + (size_t)lbcap * 8;
}

// Exclusive scan of v[0..n) in place by the whole block (thread t owns a contiguous chunk);
// returns the total to every thread. Ends with a barrier.
__device__ uint32_t gp_block_scan(uint32_t *v, int n, uint32_t *wsum) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int s0 = min(n, tid * per), s1 = min(n, s0 + per);
  uint32_t mine = 0;
  for (int e = s0; e < s1; e++) mine += v[e];
  uint32_t inc = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  uint32_t base = 0, total = 0;
  for (int w = 0; w < nw; w++) {
    if (w < warp) base += wsum[w];
    total += wsum[w];
  }
  base += inc - mine;
  for (int e = s0; e < s1; e++) {
    const uint32_t x = v[e];
    v[e] = base;
    base += x;
  }
  __syncthreads();
  return total;
}

// Running maximum of v[0..n) in place (the segment of each list entry from the marks
// its segments left at their first entry). Ends with a barrier.
__device__ void gp_block_runmax(uint32_t *v, int n, uint32_t *wsum) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int e0 = min(n, tid * per), e1 = min(n, e0 + per);
  uint32_t run = 0;
  for (int e = e0; e < e1; e++) run = max(run, v[e]);
  uint32_t inc = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc = max(inc, y);
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  uint32_t before = __shfl_up_sync(0xffffffffu, inc, 1);
  if (lane == 0) before = 0;
  for (int w = 0; w < warp; w++) before = max(before, wsum[w]);
  for (int e = e0; e < e1; e++) {
    before = max(before, v[e]);
    v[e] = before;
  }
  __syncthreads();
}

// Keep the kappa keys of lbuf[0..n) at or above the kappa-th largest T (n > kappa): the kept
// keys found beyond position kappa move into the dropped slots below it (their numbers are
// equal). slots: >= kappa words of scratch. Returns T; ends with a barrier.
__device__ uint64_t gp_compact(uint64_t *lbuf, int n, int kappa, uint32_t *slots, uint32_t *hist,
                               uint64_t *small, uint32_t *wsum, uint32_t *sh, uint32_t *flags) {
  const uint64_t T = block_kth_largest(lbuf, n, kappa, hist, small, wsum, sh);
  if (threadIdx.x == 0) {
    sh[4] = 0u;
    sh[5] = 0u;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kappa; i += blockDim.x)
    if (lbuf[i] < T) {
      const uint32_t d = atomicAdd(&sh[4], 1u);
      if (d < (uint32_t)kappa) slots[d] = (uint32_t)i;
      else atomicOr(flags, TACHIOM_FLAG_CAPACITY);  // not reachable with distinct keys
    }
  __syncthreads();
  for (int i = kappa + threadIdx.x; i < n; i += blockDim.x) {
    const uint64_t k = lbuf[i];
    if (k >= T) {
      const uint32_t d = atomicAdd(&sh[5], 1u);
      if (d < min(sh[4], (uint32_t)kappa)) lbuf[slots[d]] = k;
      else atomicOr(flags, TACHIOM_FLAG_CAPACITY);  // not reachable with distinct keys
    }
  }
  __syncthreads();
  return T;
}

// first position p in [lo, hi) with list_doc[p] >= v (hi if none)
__device__ __forceinline__ int32_t gp_lower_bound(const int32_t *__restrict__ list_doc, int32_t lo, int32_t hi,
                                                  int32_t v) {
  while (lo < hi) {
    const int32_t mid = lo + ((hi - lo) >> 1);
    if (__ldg(list_doc + mid) < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

struct GpArgs {
  const int32_t *meta;  // qoff [nq+1] | koff [nq+1] | k [nq] | ntok [nq] | kappa_d [nq]
  int nq;
  const int32_t *top_ids;
  const float *top_s;
  int kc;
  const int64_t *list_off;
  const int32_t *list_doc;
  const int32_t *list_roff;
  int nr;          // ranges
  int64_t D;
  int RD;          // documents per range
  int64_t C;
  int ng;          // range groups per query
  int kd;          // pool stride (the batch's largest kappa_d)
  int ecap;        // key buffer capacity
  int lbcap;       // candidate buffer capacity (>= kd + ecap)
  int split_cap;   // a piece with more entries is halved (ecap, or small to test the split path)
  uint64_t *pool;  // [nq x ng x kd]
  int32_t *pool_n; // [nq x ng]
  int64_t nlist;   // list entries
  uint32_t *flags;
};

__global__ void __launch_bounds__(GP_THREADS)
k_gather_pool(const GpArgs A) {
  extern __shared__ __align__(16) unsigned char gp_raw[];
  __shared__ uint32_t wsum[GP_THREADS / 32];
  __shared__ uint64_t small[64];
  __shared__ uint32_t sh[8];
  __shared__ int s_lcount;
  __shared__ int2 stack[GP_STACK];
  __shared__ int s_sp;
  const int g = blockIdx.x, q = blockIdx.y, tid = threadIdx.x, lane = tid & 31;
  const int kc = A.kc;
  const int nseg_max = MAX_NTOK * kc;
  GpSmem S;
  {
    unsigned char *p = gp_raw;
    S.lbuf = reinterpret_cast<uint64_t *>(p);
    p += (size_t)A.lbcap * 8;
    S.j = reinterpret_cast<int32_t *>(p);
    p += (size_t)nseg_max * 4;
    S.base = reinterpret_cast<int32_t *>(p);
    p += (size_t)nseg_max * 4;
    S.sc = reinterpret_cast<float *>(p);
    p += (size_t)nseg_max * 4;
    S.start = reinterpret_cast<int32_t *>(p);
    p += (size_t)nseg_max * 4;
    S.pref = reinterpret_cast<uint32_t *>(p);
    p += (size_t)nseg_max * 4;
    S.cnt = reinterpret_cast<uint32_t *>(p);
    p += (size_t)GP_NB_MAX * 4;
    S.kin = reinterpret_cast<uint32_t *>(p);
    p += (size_t)A.ecap * 4;
    S.kout = reinterpret_cast<uint32_t *>(p);
  }
  const int nq = A.nq;
  const int row_b = A.meta[q], ntok = A.meta[q + 1] - row_b;
  const int kdq = min(A.kd, A.meta[4 * nq + 2 + q]);
  const int nseg = ntok * kc;
  const int nr1 = A.nr + 1;
  const int rlo = (int)((int64_t)g * A.nr / A.ng), rhi = (int)((int64_t)(g + 1) * A.nr / A.ng);
  // the query's segments: centroid, list position, score (thread tid owns segments tid + u * 512,
  // u < 8: every load of a phase is issued before any is used)
  {
    int32_t jj[GP_SPT];
#pragma unroll
    for (int u = 0; u < GP_SPT; u++) {
      const int e = tid + u * GP_THREADS;
      jj[u] = e < nseg ? A.top_ids[(int64_t)row_b * kc + e] : -1;
      if (e < nseg) S.sc[e] = A.top_s[(int64_t)row_b * kc + e];
    }
    int64_t lb[GP_SPT];
#pragma unroll
    for (int u = 0; u < GP_SPT; u++) {
      if (jj[u] >= A.C) {
        atomicOr(A.flags, TACHIOM_FLAG_BAD_INPUT);
        jj[u] = -1;
      }
      lb[u] = jj[u] >= 0 ? __ldg(A.list_off + jj[u]) : 0;
    }
#pragma unroll
    for (int u = 0; u < GP_SPT; u++) {
      const int e = tid + u * GP_THREADS;
      if (e < nseg) {
        S.j[e] = jj[u];
        S.base[e] = (int32_t)lb[u];
      }
    }
  }
  if (tid == 0) s_lcount = 0;
  uint64_t thr = 0ull;  // the running cut: a key is kept if above it (real keys are > 0)
  // Position (relative to L_j) of the first document >= d in list j: the table's entry at a range
  // boundary, else a binary search inside the range's slice. r and aligned are the same for every
  // segment of a piece (computed once per piece).
  auto bound = [&](int32_t jj, int32_t base, int64_t d, int r, bool aligned) -> int32_t {
    const int32_t lo = __ldg(A.list_roff + (int64_t)jj * nr1 + r);
    if (aligned) return lo;
    const int32_t hi = __ldg(A.list_roff + (int64_t)jj * nr1 + r + 1);
    return gp_lower_bound(A.list_doc, base + lo, base + hi, (int32_t)d) - base;
  };
  // segment index -> (token, rank) by a multiplication: floor(e / kc) = umulhi(e, 2^32 / kc + 1)
  // for e < 2^12 and kc <= 2^7 (the rounding error e * kc stays below 2^32 / kc)
  const uint32_t kc_magic = 0xffffffffu / (uint32_t)kc + 1u;
  // The group's documents in chunks of at most 2^20 ids starting on range boundaries; a chunk
  // whose entries exceed the key buffers is cut into up to 8 pieces (on range boundaries where
  // possible), recursively, until every piece fits.
  const int64_t g_d0 = (int64_t)rlo * A.RD, g_d1 = min(A.D, (int64_t)rhi * A.RD);
  const int64_t chunk = max((int64_t)1, (int64_t)GP_XMAX / A.RD) * A.RD;
  __syncthreads();

  for (int64_t c0 = g_d0; c0 < g_d1; c0 += chunk) {
    if (tid == 0) {
      stack[0] = make_int2((int)c0, (int)min(g_d1, c0 + chunk));
      s_sp = 1;
    }
    __syncthreads();
    while (s_sp > 0) {
      const int2 piece = stack[s_sp - 1];
      const int64_t d0 = piece.x, d1 = piece.y;
      __syncthreads();  // every thread has read the top of the stack
      if (tid == 0) s_sp--;
      // the piece's slice of every list
      const int ra = (int)((uint32_t)d0 / (uint32_t)A.RD), rb_ = d1 >= A.D ? A.nr : (int)((uint32_t)d1 / (uint32_t)A.RD);
      const bool al_a = d0 == (int64_t)ra * A.RD, al_b = d1 >= A.D || d1 == (int64_t)rb_ * A.RD;
      if (al_a && al_b) {
        // both ends on range boundaries (the usual case): two table reads per segment, all in flight
        int32_t ta[GP_SPT], tb[GP_SPT];
#pragma unroll
        for (int u = 0; u < GP_SPT; u++) {
          const int e = tid + u * GP_THREADS;
          const int32_t jj = e < nseg ? S.j[e] : -1;
          ta[u] = jj >= 0 ? __ldg(A.list_roff + (int64_t)jj * nr1 + ra) : 0;
          tb[u] = jj >= 0 ? __ldg(A.list_roff + (int64_t)jj * nr1 + rb_) : 0;
        }
#pragma unroll
        for (int u = 0; u < GP_SPT; u++) {
          const int e = tid + u * GP_THREADS;
          if (e < nseg) {
            S.start[e] = S.base[e] + ta[u];
            S.pref[e] = (uint32_t)(tb[u] - ta[u]);
          }
        }
      } else {
        for (int e = tid; e < nseg; e += GP_THREADS) {
          const int32_t jj = S.j[e];
          int32_t a = 0, b = 0;
          if (jj >= 0) {
            a = bound(jj, S.base[e], d0, ra, al_a);
            b = bound(jj, S.base[e], d1, rb_, al_b);
          }
          S.start[e] = S.base[e] + a;
          S.pref[e] = (uint32_t)(b - a);
        }
      }
      __syncthreads();
      const int E = (int)gp_block_scan(S.pref, nseg, wsum);
      if (E == 0) continue;
      if (E > A.split_cap && d1 - d0 > 1) {
        // too many entries for one pass: k pieces, the lowest on top of the stack
        if (tid == 0) {
          int k = min(8, max(2, (int)((2 * (int64_t)E + A.split_cap - 1) / A.split_cap)));
          k = (int)min((int64_t)k, d1 - d0);
          // a piece over several ranges is cut on range boundaries only (table reads, no search)
          const int64_t nrp = (d1 + A.RD - 1) / A.RD - d0 / A.RD;
          if (nrp >= 2) k = (int)min((int64_t)k, nrp);
          if (s_sp + k <= GP_STACK) {
            int64_t hi = d1;
            for (int i = k - 1; i >= 1; i--) {
              int64_t p = d0 + (d1 - d0) * i / k;
              const int64_t rb = (p + A.RD / 2) / A.RD * A.RD;  // nearest range boundary
              if (rb > d0 && rb < hi) p = rb;
              if (p <= d0 || p >= hi) continue;
              stack[s_sp++] = make_int2((int)p, (int)hi);
              hi = p;
            }
            stack[s_sp++] = make_int2((int)d0, (int)hi);
          } else {
            atomicOr(A.flags, TACHIOM_FLAG_CAPACITY);  // not reachable: depth <= 7 levels of 8
          }
        }
        __syncthreads();
        continue;
      }
      // keys are taken relative to the piece's first document
      const int64_t r0 = d0;
      const int x0 = 0, x1 = (int)(d1 - d0);
      // room in the candidate buffer for every document of this piece
      if (s_lcount + E > A.lbcap) {
        const int n = s_lcount;
        thr = gp_compact(S.lbuf, n, kdq, S.kin, S.cnt, small, wsum, sh, A.flags);
        if (tid == 0) s_lcount = kdq;
        __syncthreads();
      }
      // buckets over the piece's documents: about one key per bucket
      const int nbb = min(GP_NB_BITS, max(5, ceil_log2((uint32_t)E)));
      const int bsh = max(0, ceil_log2((uint32_t)(x1 - x0)) - nbb);
      const int nb = ((x1 - x0 - 1) >> bsh) + 1;
      for (int x = tid; x < E; x += GP_THREADS) S.kout[x] = 0u;
      for (int b = tid; b < nb; b += GP_THREADS) S.cnt[b] = 0u;
      __syncthreads();
      // each segment marks its first entry with its index; a running maximum then gives every
      // entry its segment (the marks increase with the position)
      for (int e = tid; e < nseg; e += GP_THREADS) {
        const uint32_t p = S.pref[e];
        const uint32_t len = (e + 1 < nseg ? S.pref[e + 1] : (uint32_t)E) - p;
        if (len > 0) S.kout[p] = (uint32_t)e;
      }
      __syncthreads();
      gp_block_runmax(S.kout, E, wsum);
      // the keys, four list entries per thread in flight, and the bucket counts
      for (int e0 = 0; e0 < E; e0 += 4 * GP_THREADS) {
        int32_t pos[4];
        uint32_t sg[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const int e = e0 + u * GP_THREADS + tid;
          pos[u] = 0;
          sg[u] = 0u;
          if (e < E) {
            sg[u] = S.kout[e];
            pos[u] = S.start[sg[u]] + (e - (int)S.pref[sg[u]]);
          }
        }
        int32_t dv[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
          if ((uint32_t)pos[u] >= (uint32_t)A.nlist) {  // a piece bound outside the lists: skipped
            atomicOr(A.flags, TACHIOM_FLAG_CAPACITY);
            pos[u] = 0;
          }
          dv[u] = __ldg(A.list_doc + pos[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const int e = e0 + u * GP_THREADS + tid;
          if (e < E) {
            uint32_t x = (uint32_t)(dv[u] - (int32_t)r0);
            if (x >= (uint32_t)(x1 - x0)) {  // a document outside the piece: not reachable
              atomicOr(A.flags, TACHIOM_FLAG_CAPACITY);
              x = 0;
            }
            const uint32_t t = kc == 1 ? sg[u] : __umulhi(sg[u], kc_magic), rk = sg[u] - t * (uint32_t)kc;
            S.kin[e] = (x << 12) | (t << 7) | rk;
            atomicAdd(&S.cnt[(x - (uint32_t)x0) >> bsh], 1u);
          }
        }
      }
      __syncthreads();
      gp_block_scan(S.cnt, nb, wsum);
      // scatter by bucket; afterwards cnt[b] is the end of bucket b
      for (int e = tid; e < E; e += GP_THREADS) {
        const uint32_t k = S.kin[e];
        const uint32_t b = ((k >> 12) - (uint32_t)x0) >> bsh;
        const uint32_t d = atomicAdd(&S.cnt[b], 1u);
        if (d < (uint32_t)E) S.kout[d] = k;
        else atomicOr(A.flags, TACHIOM_FLAG_CAPACITY);
      }
      __syncthreads();
      // every key to its place in its bucket: its rank among the bucket's (distinct) keys
      for (int f = tid; f < E; f += GP_THREADS) {
        const uint32_t k = S.kout[f];
        const uint32_t b = ((k >> 12) - (uint32_t)x0) >> bsh;
        const uint32_t end = S.cnt[b], st = b == 0 ? 0u : S.cnt[b - 1];
        uint32_t below = 0;
        for (uint32_t h = st; h < end; h++) below += S.kout[h] < k ? 1u : 0u;
        if (st + below < (uint32_t)E) S.kin[st + below] = k;
        else atomicOr(A.flags, TACHIOM_FLAG_CAPACITY);
      }
      __syncthreads();
      // S~ of every reached document (the thread holding the first key of its run), kept if it
      // beats the running cut
      for (int f0 = 0; f0 < E; f0 += GP_THREADS) {
        const int f = f0 + tid;
        bool keep = false;
        uint64_t ck = 0ull;
        if (f < E) {
          const uint32_t k = S.kin[f], x = k >> 12;
          if (f == 0 || (S.kin[f - 1] >> 12) != x) {
            float sum = 0.f;
            uint32_t prev = 0xffffffffu;
            for (int h = f; h < E; h++) {
              const uint32_t kh = S.kin[h];
              if ((kh >> 12) != x) break;
              const uint32_t t = (kh >> 7) & 31u;
              if (t != prev) {
                const float v = S.sc[t * kc + (kh & 127u)];
                sum = (prev == 0xffffffffu) ? v : sum + v;
                prev = t;
              }
            }
            ck = comp_key(sum, (int32_t)(r0 + x));
            keep = ck > thr;
          }
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        int wb = 0;
        if (lane == 0 && m) wb = atomicAdd(&s_lcount, __popc(m));
        wb = __shfl_sync(0xffffffffu, wb, 0);
        const int li = wb + __popc(m & ((1u << lane) - 1u));
        if (keep) {
          if (li < A.lbcap) S.lbuf[li] = ck;
          else atomicOr(A.flags, TACHIOM_FLAG_CAPACITY);
        }
      }
      __syncthreads();
    }
    // every thread has read the empty stack before thread 0 sets up the next chunk's (without
    // this barrier a late thread could read the next chunk's s_sp = 1 and enter the loop alone)
    __syncthreads();
  }
  // the group's exact top-kappa_d
  int n = s_lcount;
  if (n > kdq) {
    gp_compact(S.lbuf, n, kdq, S.kin, S.cnt, small, wsum, sh, A.flags);
    n = kdq;
  }
  uint64_t *out = A.pool + ((int64_t)q * A.ng + g) * A.kd;
  for (int i = tid; i < n; i += GP_THREADS) out[i] = S.lbuf[i];
  if (tid == 0) A.pool_n[q * A.ng + g] = n;
}

// ---------------------------------------------------------------------------------
// Per query: the union of its groups' parts (n <= SEL_CAP keys) in shared memory; the first
// min(n, kappa_d) by (S~ desc, doc asc) are written. A buffer larger than kappa_d is cut to
// its kappa_d largest keys by the radix select first; the kept keys are sorted.
constexpr int PS_THREADS = 1024;
__global__ void __launch_bounds__(PS_THREADS)
k_pool_select(const uint64_t *__restrict__ pool, const int32_t *__restrict__ pool_n, int ng, const int32_t *meta,
              int nq, int kd, int32_t *__restrict__ cand, float *__restrict__ cand_s, int32_t *__restrict__ ncand) {
  extern __shared__ __align__(16) uint64_t ssm[];  // [SEL_CAP] keys, then [next_pow2(kappa_d)] kept keys
  __shared__ uint32_t hist[1 << KSEL_BITS];
  __shared__ uint64_t small[64];
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t sh[8];
  __shared__ int s_off[65];
  __shared__ int s_cnt;
  const int q = blockIdx.x, tid = threadIdx.x;
  const int kdq = min(kd, meta[4 * nq + 2 + q]);
  if (tid == 0) {
    int o = 0;
    for (int g = 0; g < ng; g++) {
      s_off[g] = o;
      o += pool_n[q * ng + g];
    }
    s_off[ng] = o;
    s_cnt = 0;
  }
  __syncthreads();
  const int n = min(s_off[ng], SEL_CAP);
  for (int g = 0; g < ng; g++) {
    const uint64_t *src = pool + ((int64_t)q * ng + g) * kd;
    const int o = s_off[g], c = s_off[g + 1] - o;
    for (int i = tid; i < c; i += PS_THREADS)
      if (o + i < SEL_CAP) ssm[o + i] = src[i];
  }
  __syncthreads();
  const int m = min(n, kdq);
  uint64_t *keys = ssm;
  if (n <= kdq) {
    const int np = next_pow2(max(n, 2));
    for (int i = n + tid; i < np; i += PS_THREADS) keys[i] = 0ull;
    __syncthreads();
    block_sort_desc(keys, np);
  } else {
    const uint64_t T = block_kth_largest(keys, n, kdq, hist, small, wsum, sh);
    uint64_t *kept = ssm + SEL_CAP;
    const int np = next_pow2(max(kdq, 2));
    for (int i = kdq + tid; i < np; i += PS_THREADS) kept[i] = 0ull;
    for (int i = tid; i < n; i += PS_THREADS) {
      const uint64_t k = keys[i];
      if (k >= T) {
        const int d = atomicAdd(&s_cnt, 1);
        if (d < kdq) kept[d] = k;
      }
    }
    __syncthreads();
    block_sort_desc(kept, np);
    keys = kept;
  }
  for (int i = tid; i < kd; i += PS_THREADS) {
    const uint64_t v = i < m ? keys[i] : 0ull;
    cand[(int64_t)q * kd + i] = v ? comp_id(v) : -1;
    cand_s[(int64_t)q * kd + i] = v ? comp_score(v) : -INFINITY;
  }
  if (tid == 0) ncand[q] = m;
}

// ---------------------------------------------------------------------------------
// launch geometry
static int gp_sms(int dev) {
  static int cached[64] = {0};
  if (dev >= 0 && dev < 64 && cached[dev]) return cached[dev];
  int n = 148;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  if (dev >= 0 && dev < 64) cached[dev] = n;
  return n;
}

// key buffer capacity for (kappa_c, kappa_d): the largest that keeps two CTAs per SM, else
// the largest that fits one
static int gp_ecap(int kc, int kd) {
  const int nseg = MAX_NTOK * kc;
  for (size_t budget : {(size_t)GP_SMEM_TWO_PER_SM, (size_t)GP_SMEM_MAX - 4096}) {
    const size_t fixed = gp_smem_bytes(nseg, 0, kd);
    if (fixed >= budget) continue;
    int ecap = (int)std::min<size_t>(GP_ECAP_MAX, (budget - fixed) / 16) & ~255;
    if (ecap >= std::max(GP_ECAP_MIN, nseg)) return ecap;
  }
  return 0;
}

// range groups per query: at most SEL_CAP / kappa_d (the selection holds every group's part), the
// range count and 64; by default about 8 CTAs per SM over the batch, and at least enough that a
// group spans one chunk of at most 2^20 documents (measured on 8.8M documents: 10 single-chunk
// groups per query 0.52 ms, 5 two-chunk groups 0.59 ms); a plan's value g > 0 asks for 2 g groups
// (within the same caps)
static int gather_groups_cap(const Index &ix, int kd) {
  return std::min(64, std::min(std::max(1, SEL_CAP / std::max(1, kd)), std::max(1, ix.n_ranges)));
}
int gather_groups(const Index &ix, int nq, int kd, int forced) {
  const int cap = gather_groups_cap(ix, kd);
  if (forced > 0) return std::min(cap, 2 * forced);
  const int sms = gp_sms(ix.device);
  const int per_chunk = std::max(1, GP_XMAX / std::max(1, ix.range_docs));  // ranges of one chunk
  const int chunks = (ix.n_ranges + per_chunk - 1) / per_chunk;
  return std::min(cap, std::max(chunks, std::max(1, (8 * sms + nq - 1) / std::max(1, nq))));
}

size_t gather_pool_elems(const Index &ix, int nq, int kd) {
  return (size_t)nq * gather_groups_cap(ix, kd) * kd;  // room for any plan's count
}

tachiom_status launch_gather(const Index &ix, const int32_t *meta, int nq, const int32_t *top_ids, const float *top_s,
                             int kc, int kd, uint64_t *pool, int32_t *pool_n, bool force_split, int groups,
                             uint32_t *flags, cudaStream_t s) {
  if (nq <= 0) return TACHIOM_OK;
  if (nq > 65535) return fail(TACHIOM_ERR_CAPACITY, "gather: more than 65535 queries in one batch");
  TPROF("gather", s);
  const int ecap = gp_ecap(kc, kd);
  if (ecap == 0) return fail(TACHIOM_ERR_CAPACITY, "gather: kappa_c %d with kappa_d %d does not fit", kc, kd);
  GpArgs A;
  A.meta = meta;
  A.nq = nq;
  A.top_ids = top_ids;
  A.top_s = top_s;
  A.kc = kc;
  A.list_off = ix.list_off;
  A.list_doc = ix.list_doc;
  A.list_roff = ix.list_roff;
  A.nr = ix.n_ranges;
  A.D = ix.D;
  A.RD = ix.range_docs;
  A.C = ix.C;
  A.ng = gather_groups(ix, nq, kd, groups);
  A.kd = kd;
  A.ecap = ecap;
  A.lbcap = kd + ecap;
  A.split_cap = force_split ? GP_SPLIT_FORCED : ecap;
  A.pool = pool;
  A.pool_n = pool_n;
  A.nlist = ix.n_list;
  A.flags = flags;
  const size_t smem = gp_smem_bytes(MAX_NTOK * kc, ecap, A.lbcap);
  TCUDA(cudaFuncSetAttribute(k_gather_pool, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_gather_pool<<<dim3(A.ng, nq), GP_THREADS, smem, s>>>(A);
  TLAUNCH();
  return TACHIOM_OK;
}

tachiom_status launch_select_kd(const Index &ix, const int32_t *meta, int nq, int kd, const uint64_t *pool,
                                const int32_t *pool_n, int groups, int32_t *cand, float *cand_s, int32_t *ncand,
                                cudaStream_t s) {
  if (nq <= 0) return TACHIOM_OK;
  TPROF("select_kd", s);
  const int ng = gather_groups(ix, nq, kd, groups);
  const size_t smem = (size_t)SEL_CAP * 8 + (size_t)next_pow2(std::max(kd, 2)) * 8;
  TCUDA(cudaFuncSetAttribute(k_pool_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_pool_select<<<nq, PS_THREADS, smem, s>>>(pool, pool_n, ng, meta, nq, kd, cand, cand_s, ncand);
  TLAUNCH();
  return TACHIOM_OK;
}

}  // namespace tachiom
