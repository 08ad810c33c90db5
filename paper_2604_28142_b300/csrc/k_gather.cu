// Step (b): inverted-list gather and centroid-only late interaction
// (Sec. 2.2, Gather steps 2-4), then the kappa_d truncation.
//
// k_gather: one CTA per (query, range of R documents). Each Top_i arrives
// sorted by (score desc, id asc), so the best retrieved centroid of token i
// for document d is the one of smallest rank u in Top_i. For each query token
// i in ascending order the CTA walks, for every j in Top_i, the slice of L_j
// that falls in its range (lists are doc-sorted and a per-(list, range) offset
// table locates the slice) and raises a shared-memory word per document to
//     code = (i + 1) << 8 | (255 - u)          (atomicMax)
// so the word holds the latest token that reached d and, within it, the best
// rank. The thread whose atomicMax replaces an earlier token's code is the
// only one that sees it, and it folds that token's maximum
//     s~_i'(d) = <q_i', c_{Top_i'[u']}>
// into S~(q, d); a barrier separates the tokens, and the codes left after the
// last token are folded at the end. Every document's S~ is therefore summed
// in ascending i, and the candidate scores are bit-identical run to run. The
// range's S~ values go to a dense per-query array (-inf = not reached), and a
// 4096-bin histogram of their keys goes to the query's histogram for the
// selection.
//
// Selection of the kappa_d best (S~ desc, doc asc): the histogram locates the
// bin that holds the kappa_d-th key; up to two more histogram levels narrow
// it when that bin is wide; every key at or above the cut is collected and
// sorted exactly. A cut inside a run of equal keys wider than the buffer
// takes the ordered tie pass (lowest doc ids first).
#include <algorithm>

#include "tachiom_internal.cuh"

namespace tachiom {

constexpr int G_THREADS = 1024;
constexpr int G_SEGCAP = 1536;  // (query token, retrieved centroid) segments described at once
constexpr int G_REG = 4;        // list entries per thread and token kept in registers

// Per (token, centroid) segment of a list inside the CTA's document range:
// start (absolute position in list_doc), exclusive prefix of the lengths within
// its token, and the code (i + 1) << 8 | (255 - rank).
struct GSeg {
  int32_t start;
  int32_t pref;
  uint32_t key;
};

// S~(d) += the score a code stands for (the first token sets it)
__device__ __forceinline__ void gather_fold(float *S, int x, uint32_t code, const float *__restrict__ tsq, int kc) {
  const int tok = (int)(code >> 8) - 1, u = 255 - (int)(code & 255u);
  const float sv = __ldg(tsq + (int64_t)tok * kc + u);
  const float cur = S[x];
  S[x] = (cur == -INFINITY) ? sv : cur + sv;
}

// The (range, query) pairs k_gather_sort could not hold, one after another per CTA.
__global__ void __launch_bounds__(G_THREADS, 1)
k_gather_tok(const int32_t *__restrict__ qoff, const int32_t *__restrict__ top_ids,
             const float *__restrict__ top_s, int kc, const int64_t *__restrict__ list_off,
             const int32_t *__restrict__ list_doc, const int32_t *__restrict__ list_roff, int nr1,
             int64_t D, int RD, int64_t C, float *__restrict__ dense, uint32_t *__restrict__ hist,
             uint32_t *__restrict__ flags, const int2 *__restrict__ items, const int *__restrict__ nitems) {
  extern __shared__ __align__(16) uint32_t gsm[];
  uint32_t *best = gsm;                                   // [RD] code of the latest token (0: none)
  float *S = reinterpret_cast<float *>(gsm + RD);         // [RD] running S~
  uint32_t *h = gsm + 2 * RD;                             // [NBINS1]
  GSeg *seg = reinterpret_cast<GSeg *>(gsm + 2 * RD + NBINS1);  // [G_SEGCAP]
  __shared__ int tok_total[MAX_NTOK];
  const int n_items = *nitems;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
  __syncthreads();  // the previous item's shared state is no longer read
  const int r = items[item].x, q = items[item].y, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int64_t r0 = (int64_t)r * RD;
  const int nd = (int)min((int64_t)RD, D - r0);
  for (int x = tid; x < RD; x += G_THREADS) {
    best[x] = 0u;
    S[x] = -INFINITY;
  }
  for (int b = tid; b < NBINS1; b += G_THREADS) h[b] = 0u;
  const int row_b = qoff[q], row_e = qoff[q + 1];
  const float *tsq = top_s + (int64_t)row_b * kc;  // Top_i scores of this query's tokens
  const int per_group = max(1, G_SEGCAP / kc);  // tokens whose segments fit at once

  for (int i0 = row_b; i0 < row_e; i0 += per_group) {
    const int ng = min(per_group, row_e - i0);
    __syncthreads();  // previous group's segments are no longer read
    // describe every segment of the group in parallel (independent loads)
    for (int e = tid; e < ng * kc; e += G_THREADS) {
      const int ti = e / kc;
      int32_t jj = top_ids[(int64_t)(i0 + ti) * kc + (e % kc)];
      if (jj >= C) {
        atomicOr(flags, TACHIOM_FLAG_BAD_INPUT);
        jj = -1;
      }
      GSeg g;
      g.start = 0;
      g.pref = 0;  // length until the scan below
      g.key = 0u;
      if (jj >= 0) {
        const int lo = list_roff[(int64_t)jj * nr1 + r], hi = list_roff[(int64_t)jj * nr1 + r + 1];
        g.start = (int32_t)(list_off[jj] + lo);
        g.pref = hi - lo;
        g.key = ((uint32_t)(i0 + ti - row_b + 1) << 8) | (uint32_t)(255 - e % kc);
      }
      seg[e] = g;
    }
    __syncthreads();
    // exclusive prefix of the lengths within each token: one warp per token
    for (int ti = warp; ti < ng; ti += G_THREADS / 32) {
      GSeg *sg = seg + ti * kc;
      int carry = 0;
      for (int u0 = 0; u0 < kc; u0 += 32) {
        const int u = u0 + lane;
        const int len = u < kc ? sg[u].pref : 0;
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        if (u < kc) sg[u].pref = carry + incl - len;
        carry += __shfl_sync(0xffffffffu, incl, 31);
      }
      if (lane == 0) tok_total[ti] = carry;
    }
    __syncthreads();
    // Tokens in order, one barrier each; each thread keeps the list entries it
    // handles for a token in registers, loaded two tokens ahead so that their
    // latency overlaps the current token's work. The three register sets keep
    // fixed roles in a 3-way unrolled loop: a register copy would wait for the
    // load still in flight.
    int32_t d0[G_REG], d1[G_REG], d2[G_REG];
    uint32_t k0[G_REG], k1[G_REG], k2[G_REG];
    auto fetch = [&](int ti, int32_t (&d)[G_REG], uint32_t (&k)[G_REG]) {
      const GSeg *sg = seg + ti * kc;
      const int total = ti < ng ? tok_total[ti] : 0;
#pragma unroll
      for (int u = 0; u < G_REG; u++) {
        // the load is issued unconditionally (position 0 for a missing entry, whose code
        // is 0): a select on its result would wait for it here instead of two tokens later
        const int e = tid + u * G_THREADS;
        int64_t pos = 0;
        k[u] = 0u;
        if (e < total) {
          int lo = 0, hi = kc;
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (sg[mid].pref <= e) lo = mid; else hi = mid;
          }
          pos = sg[lo].start + (e - sg[lo].pref);
          k[u] = sg[lo].key;
        }
        d[u] = __ldg(list_doc + pos);
      }
    };
    auto visit = [&](int x, uint32_t code) {
      const uint32_t old = atomicMax(&best[x], code);
      if (old != 0u && (old >> 8) != (code >> 8)) gather_fold(S, x, old, tsq, kc);
    };
    // token ti: fetch ti + 2 into (dn, kn), then fold the entries in (dc, kcur); dc holds
    // absolute doc ids, kcur = 0 marks no entry
    auto step = [&](int ti, const int32_t (&dc)[G_REG], const uint32_t (&kcur)[G_REG], int32_t (&dn)[G_REG],
                    uint32_t (&kn)[G_REG]) {
      fetch(ti + 2, dn, kn);
#pragma unroll
      for (int u = 0; u < G_REG; u++)
        if (kcur[u]) visit(dc[u] - (int32_t)r0, kcur[u]);
      const GSeg *sg = seg + ti * kc;
      const int total = tok_total[ti];
      for (int e = tid + G_REG * G_THREADS; e < total; e += G_THREADS) {
        int lo = 0, hi = kc;
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (sg[mid].pref <= e) lo = mid; else hi = mid;
        }
        visit(list_doc[sg[lo].start + (e - sg[lo].pref)] - (int32_t)r0, sg[lo].key);
      }
      __syncthreads();
    };
    fetch(0, d0, k0);
    fetch(1, d1, k1);
    for (int ti = 0; ti < ng; ti += 3) {
      step(ti, d0, k0, d2, k2);
      if (ti + 1 < ng) step(ti + 1, d1, k1, d0, k0);
      if (ti + 2 < ng) step(ti + 2, d2, k2, d1, k1);
    }
  }
  // the codes of the last token that reached each document
  __syncthreads();
  for (int x = tid; x < nd; x += G_THREADS) {
    const uint32_t c = best[x];
    if (c) gather_fold(S, x, c, tsq, kc);
  }
  float *out = dense + (int64_t)q * D + r0;
  for (int x = tid; x < nd; x += G_THREADS) {
    const float v = S[x];
    out[x] = v;
    if (v != -INFINITY) atomicAdd(&h[fkey(v) >> 20], 1u);
  }
  __syncthreads();
  uint32_t *hq = hist + (int64_t)q * NBINS1;
  for (int b = tid; b < NBINS1; b += G_THREADS)
    if (h[b]) atomicAdd(&hq[b], h[b]);
  }
}

// ---------------------------------------------------------------------------------
// k_gather_sort: one CTA per (range of R documents, query). Every (token i,
// rank u) slice of L_{Top_i[u]} inside the range is described at once, and
// each of its entries becomes a 32-bit key
//     (d - r0) << 12 | i << 7 | u
// loaded with all loads in flight. A counting sort by document (16-bit counts
// in shared memory, a block-wide scan, a scatter) puts each document's keys
// into one run, and each key then finds its place in its (short) run by
// counting the run's smaller keys, so a run is ordered by token, then rank.
// One pass over the range's documents writes S~: for a reached document, the
// first key of each token holds the token's best (lowest) rank - Top_i is
// sorted by score desc, so that is the token's maximum - and the scores are
// added in ascending i, the order (and so the FP32 sums) of the token-serial
// form.
// A range with more entries than the key buffers hold is left to k_gather_tok.
constexpr int GS_THREADS = 1024;
constexpr int GS_ECAP_MAX = 16384;

__host__ __device__ inline size_t gs_fixed(int kc, int RD) {
  return (size_t)MAX_NTOK * kc * sizeof(GSeg)   // slice descriptors
         + (size_t)MAX_NTOK * kc * 4             // Top_i scores
         + (size_t)NBINS1 * 4                    // histogram
         + (size_t)((RD + 1) / 2) * 4;           // packed 16-bit per-document counts / cursors
}
inline int gs_ecap(int kc, int RD) {
  const size_t avail = 227 * 1024 - 1024 - gs_fixed(kc, RD);
  return (int)std::min<size_t>(GS_ECAP_MAX, avail / 8) & ~1023;
}

__device__ __forceinline__ uint32_t gs_get16(const uint32_t *w, int x) { return (w[x >> 1] >> ((x & 1) << 4)) & 0xffffu; }

__global__ void __launch_bounds__(GS_THREADS, 1)
k_gather_sort(const int32_t *__restrict__ qoff, const int32_t *__restrict__ top_ids,
              const float *__restrict__ top_s, int kc, const int64_t *__restrict__ list_off,
              const int32_t *__restrict__ list_doc, const int32_t *__restrict__ list_roff, int nr1,
              int64_t D, int RD, int64_t C, int ecap, float *__restrict__ dense, uint32_t *__restrict__ hist,
              uint32_t *__restrict__ flags, int2 *__restrict__ ovf, int *__restrict__ novf) {
  extern __shared__ __align__(16) unsigned char gsr[];
  GSeg *seg = reinterpret_cast<GSeg *>(gsr);                                                 // [32 * kc]
  float *sc = reinterpret_cast<float *>(gsr + (size_t)MAX_NTOK * kc * sizeof(GSeg));        // [32 * kc]
  uint32_t *h = reinterpret_cast<uint32_t *>(sc + MAX_NTOK * kc);                           // [NBINS1]
  uint32_t *cnt = h + NBINS1;                                                                // [RD / 2]
  uint32_t *kin = cnt + (RD + 1) / 2;                                                        // [ecap]
  uint32_t *kout = kin + ecap;                                                               // [ecap]
  __shared__ uint32_t wsum[GS_THREADS / 32];
  __shared__ int s_nr;  // reached documents of the range
  const int r = blockIdx.x, q = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_nr = 0;
  const int64_t r0 = (int64_t)r * RD;
  const int nd = (int)min((int64_t)RD, D - r0);
  const int row_b = qoff[q], ntok = qoff[q + 1] - row_b;
  const int nseg = ntok * kc;
  // slice descriptors (length in .pref until the scan), the scores, empty counts and histogram;
  // two descriptors per thread, their loads issued together
  for (int e0 = tid; e0 < nseg; e0 += 2 * GS_THREADS) {
    int32_t jj[2];
    float sv[2];
#pragma unroll
    for (int u = 0; u < 2; u++) {
      const int e = e0 + u * GS_THREADS;
      jj[u] = e < nseg ? top_ids[(int64_t)row_b * kc + e] : -1;
      sv[u] = e < nseg ? top_s[(int64_t)row_b * kc + e] : 0.f;
    }
    int lo[2] = {0, 0}, hi[2] = {0, 0};
    int64_t lb[2] = {0, 0};
#pragma unroll
    for (int u = 0; u < 2; u++) {
      if (jj[u] >= C) {
        atomicOr(flags, TACHIOM_FLAG_BAD_INPUT);
        jj[u] = -1;
      }
      if (jj[u] >= 0) {
        lo[u] = list_roff[(int64_t)jj[u] * nr1 + r];
        hi[u] = list_roff[(int64_t)jj[u] * nr1 + r + 1];
        lb[u] = list_off[jj[u]];
      }
    }
#pragma unroll
    for (int u = 0; u < 2; u++) {
      const int e = e0 + u * GS_THREADS;
      if (e < nseg) {
        GSeg g;
        g.start = (int32_t)(lb[u] + lo[u]);
        g.pref = hi[u] - lo[u];
        g.key = (uint32_t)((e / kc) << 7 | (e % kc));
        seg[e] = g;
        sc[e] = sv[u];
      }
    }
  }
  for (int b = tid; b < NBINS1; b += GS_THREADS) h[b] = 0u;
  for (int x = tid; x < (RD + 1) / 2; x += GS_THREADS) cnt[x] = 0u;
  for (int x = tid; x < ecap; x += GS_THREADS) kout[x] = 0u;  // slice marks (below)
  __syncthreads();
  // exclusive prefix of the slice lengths: thread t owns descriptors [t * per, (t + 1) * per)
  uint32_t total;
  {
    const int per = (nseg + GS_THREADS - 1) / GS_THREADS;
    const int s0 = min(nseg, tid * per), s1 = min(nseg, s0 + per);
    uint32_t mine = 0;
    for (int e = s0; e < s1; e++) mine += (uint32_t)seg[e].pref;
    uint32_t inc = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    uint32_t base = 0;
    total = 0;
    for (int w = 0; w < GS_THREADS / 32; w++) {
      if (w < warp) base += wsum[w];
      total += wsum[w];
    }
    base += inc - mine;
    for (int e = s0; e < s1; e++) {
      const int len = seg[e].pref;
      seg[e].pref = (int32_t)base;
      if (len > 0 && base < (uint32_t)ecap) kout[base] = (uint32_t)e;  // a slice marks its first entry
      base += (uint32_t)len;
    }
  }
  if (total > (uint32_t)ecap) {
    // too many entries for the key buffers: the token-serial kernel takes this range
    if (tid == 0) {
      const int k = atomicAdd(novf, 1);
      ovf[k] = make_int2(r, q);
    }
    return;
  }
  // every document of the range starts unreached (-inf); the reached ones are written below
  float *out = dense + (int64_t)q * D + r0;
  for (int x = tid; x < nd; x += GS_THREADS) out[x] = -INFINITY;
  __syncthreads();
  const int n = (int)total;
  // every entry's slice: a running maximum over the marks (slices are in prefix order)
  {
    const int per = (n + GS_THREADS - 1) / GS_THREADS;
    const int e0 = min(n, tid * per), e1 = min(n, e0 + per);
    uint32_t run = 0;
    for (int e = e0; e < e1; e++) run = max(run, kout[e]);
    uint32_t inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc = max(inc, y);
    }
    __syncthreads();  // wsum of the length scan is no longer read
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    uint32_t before = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) before = 0;
    for (int w = 0; w < warp; w++) before = max(before, wsum[w]);
    for (int e = e0; e < e1; e++) {
      before = max(before, kout[e]);
      kout[e] = before;
    }
  }
  __syncthreads();
  // the keys (four entries per thread in flight) and the per-document counts
  for (int e0 = 0; e0 < n; e0 += 4 * GS_THREADS) {
    int64_t pos[4];
    uint32_t code[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const int e = e0 + u * GS_THREADS + tid;
      pos[u] = 0;
      code[u] = 0u;
      if (e < n) {
        const GSeg g = seg[kout[e]];
        pos[u] = g.start + (e - g.pref);
        code[u] = g.key;
      }
    }
    int32_t dv[4];
#pragma unroll
    for (int u = 0; u < 4; u++) dv[u] = __ldg(list_doc + pos[u]);
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const int e = e0 + u * GS_THREADS + tid;
      if (e < n) {
        const uint32_t x = (uint32_t)(dv[u] - (int32_t)r0);
        kin[e] = (x << 12) | code[u];
        atomicAdd(&cnt[x >> 1], 1u << ((x & 1u) << 4));
      }
    }
  }
  __syncthreads();
  // exclusive scan of the counts in place: warp w owns a contiguous block of words (two
  // documents each), read lane-consecutively (no bank conflicts): the block totals, then the
  // block's words in rounds of 32 with a running carry
  {
    const int nw = (RD + 1) / 2;
    const int wper = ((nw + GS_THREADS / 32 - 1) / (GS_THREADS / 32) + 31) & ~31;  // words per warp
    const int w0 = warp * wper, w1 = min(nw, w0 + wper);
    uint32_t tot = 0;
    for (int x = w0 + lane; x < w1; x += 32) {
      const uint32_t v = cnt[x];
      tot += (v & 0xffffu) + (v >> 16);
    }
    tot = __reduce_add_sync(0xffffffffu, tot);
    __syncthreads();  // wsum of the slice scans is no longer read
    if (lane == 0) wsum[warp] = tot;
    __syncthreads();
    uint32_t carry = 0;
    for (int w = 0; w < warp; w++) carry += wsum[w];
    for (int xb = w0; xb < w1; xb += 32) {
      const int x = xb + lane;
      const uint32_t v = x < w1 ? cnt[x] : 0u;
      const uint32_t c0 = v & 0xffffu, c1 = v >> 16, sw = c0 + c1;
      uint32_t inc = sw;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      const uint32_t start = carry + inc - sw;
      if (x < w1) cnt[x] = start | ((start + c0) << 16);
      carry += __shfl_sync(0xffffffffu, inc, 31);
    }
  }
  __syncthreads();
  // scatter: cursor(d) runs from start(d) to start(d) + count(d) = start(d + 1)
  for (int e = tid; e < n; e += GS_THREADS) {
    const uint32_t k = kin[e], x = k >> 12;
    const uint32_t old = atomicAdd(&cnt[x >> 1], 1u << ((x & 1u) << 4));
    kout[(old >> ((x & 1u) << 4)) & 0xffffu] = k;
  }
  __syncthreads();
  // each key to its place in its document's run, ordered by (token, rank): its rank
  // among the run's keys (all distinct)
  for (int f = tid; f < n; f += GS_THREADS) {
    const uint32_t k = kout[f], x = k >> 12;
    const uint32_t end = gs_get16(cnt, (int)x), start = x == 0 ? 0u : gs_get16(cnt, (int)x - 1);
    uint32_t below = 0;
    for (uint32_t g = start; g < end; g++) below += kout[g] < k ? 1u : 0u;
    kin[start + below] = k;
  }
  __syncthreads();
  // the reached documents, listed in kout (free now) with warp-aggregated appends
  for (int b0 = 0; b0 < nd; b0 += GS_THREADS) {
    const int x = b0 + tid;
    bool reached = false;
    if (x < nd) reached = gs_get16(cnt, x) > (x == 0 ? 0u : gs_get16(cnt, x - 1));
    const unsigned m = __ballot_sync(0xffffffffu, reached);
    int base = 0;
    if (lane == 0 && m) base = atomicAdd(&s_nr, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (reached) kout[base + __popc(m & ((1u << lane) - 1u))] = (uint32_t)x;
  }
  __syncthreads();
  // S~ per reached document: the first key of each token run is the token's best rank; the
  // tokens come in ascending i
  const int nr = s_nr;
  for (int i = tid; i < nr; i += GS_THREADS) {
    const int x = (int)kout[i];
    const uint32_t end = gs_get16(cnt, x), start = x == 0 ? 0u : gs_get16(cnt, x - 1);
    float S = 0.f;
    uint32_t prev = 0xffffffffu;
    for (uint32_t f = start; f < end; f++) {
      const uint32_t kf = kin[f], t = (kf >> 7) & 31u;
      if (t != prev) {
        const float v = sc[t * kc + (kf & 127u)];
        S = (prev == 0xffffffffu) ? v : S + v;
        prev = t;
      }
    }
    out[x] = S;
    atomicAdd(&h[fkey(S) >> 20], 1u);
  }
  __syncthreads();
  uint32_t *hq = hist + (int64_t)q * NBINS1;
  for (int b = tid; b < NBINS1; b += GS_THREADS)
    if (h[b]) atomicAdd(&hq[b], h[b]);
}

tachiom_status launch_gather(const Index &ix, const int32_t *meta_qoff, int nq, const int32_t *top_ids,
                             const float *top_s, int kc, float *dense, uint32_t *hist, int2 *ovf, int *novf,
                             bool tok_only, uint32_t *flags, cudaStream_t s) {
  if (nq <= 0) return TACHIOM_OK;
  TPROF("gather", s);
  TCUDA(cudaMemsetAsync(hist, 0, (size_t)nq * NBINS1 * 4, s));
  TCUDA(cudaMemsetAsync(novf, 0, sizeof(int), s));
  // tok_only: no key buffer, so every range with entries goes to the token-serial kernel
  const int ecap = tok_only ? 0 : gs_ecap(kc, ix.range_docs);
  const size_t sm1 = gs_fixed(kc, ix.range_docs) + (size_t)ecap * 8;
  TCUDA(cudaFuncSetAttribute(k_gather_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
  k_gather_sort<<<dim3(ix.n_ranges, nq), GS_THREADS, sm1, s>>>(meta_qoff, top_ids, top_s, kc, ix.list_off,
                                                              ix.list_doc, ix.list_roff, ix.n_ranges + 1, ix.D,
                                                              ix.range_docs, ix.C, ecap, dense, hist, flags, ovf,
                                                              novf);
  TLAUNCH();
  // the ranges that overflowed, token by token (a CTA per SM, each taking items in turn)
  const size_t sm2 = (size_t)ix.range_docs * 8 + NBINS1 * 4 + (size_t)G_SEGCAP * sizeof(GSeg);
  TCUDA(cudaFuncSetAttribute(k_gather_tok, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix.device);
  k_gather_tok<<<sms, G_THREADS, sm2, s>>>(meta_qoff, top_ids, top_s, kc, ix.list_off, ix.list_doc, ix.list_roff,
                                           ix.n_ranges + 1, ix.D, ix.range_docs, ix.C, dense, hist, flags, ovf,
                                           novf);
  TLAUNCH();
  return TACHIOM_OK;
}

// ---------------------------------------------------------------------------------
// kappa_d selection
// state[q][*]: 0 prefix (key bits fixed so far), 1 level reached (1..3), 2 above
// (count of keys strictly above the current bin range), 3 done, 4 kmin (collect
// keys >= kmin), 5 collected count, 6 tie mode, 7 spare.
constexpr int S_PREFIX = 0, S_LEVEL = 1, S_ABOVE = 2, S_DONE = 3, S_KMIN = 4, S_CNT = 5, S_TIES = 6;
constexpr int SEL_CHUNK = 8192;
constexpr int SEL_LOCAL = 1024;  // keys a collect block gathers before reserving them
constexpr int SEL_THREADS = 256;

// level L bins: L1 key>>20 (4096), L2 (key>>8)&0xfff (4096), L3 key&0xff (256)
__device__ __forceinline__ int level_shift(int L) { return L == 1 ? 20 : (L == 2 ? 8 : 0); }
__device__ __forceinline__ int level_bins(int L) { return L == 3 ? 256 : 4096; }

// One block per query: the bin holding the cut (the need-th key from the top
// among the keys that share the prefix found so far). Thread t sums bins
// [nb - (t+1) w, nb - t w) (w = nb / 256), a block scan from the top finds the
// thread whose chunk holds the cut, and that thread walks its chunk.
constexpr int FIND_THREADS = 256;
__global__ void __launch_bounds__(FIND_THREADS)
k_sel_find(const uint32_t *__restrict__ hist, uint32_t *__restrict__ state, const int32_t *__restrict__ meta, int nq,
           int kd_max, int L, uint32_t *__restrict__ flags) {
  __shared__ uint32_t wsum[FIND_THREADS / 32];
  const int q = blockIdx.x;
  const int kd = min(kd_max, meta[4 * nq + 2 + q]);
  uint32_t *st = state + (int64_t)q * 8;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (L == 1) {
    if (tid == 0) {
      st[S_PREFIX] = 0; st[S_LEVEL] = 1; st[S_ABOVE] = 0; st[S_DONE] = 0; st[S_KMIN] = 1;
      st[S_CNT] = 0; st[S_TIES] = 0;
    }
  } else if (st[S_DONE]) {
    return;
  }
  const uint32_t *hq = hist + (int64_t)q * NBINS1;
  const int nb = level_bins(L);
  const int w = nb / FIND_THREADS;
  const int top = nb - tid * w;  // this thread's chunk is [top - w, top)
  uint32_t mine = 0;
  for (int b = top - 1; b >= top - w; b--) mine += hq[b];
  // inclusive scan of the chunk sums, from the top bin down (thread order)
  uint32_t inc = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  uint32_t before = 0;
  for (int u = 0; u < warp; u++) before += wsum[u];
  const uint32_t excl = before + inc - mine;  // keys in bins above this chunk
  const uint32_t total = before + inc;        // ... and including it (for the last thread: all keys)
  const uint32_t above = st[S_ABOVE];
  const uint32_t need = (uint32_t)kd > above ? (uint32_t)kd - above : 0;
  const int sh = level_shift(L);
  const uint32_t prefix = st[S_PREFIX];
  __syncthreads();  // every thread has read the state before one rewrites it
  if (tid == FIND_THREADS - 1 && total < need) {
    // fewer keys than needed in the whole range: take everything in it
    const uint32_t lo_key = (L == 1) ? 1u : (prefix << (sh + (L == 2 ? 12 : 8)));
    st[S_KMIN] = lo_key == 0 ? 1u : lo_key;
    st[S_DONE] = 1;
    return;
  }
  if (!(excl < need && need <= total)) return;
  // the cut lies in this chunk: walk it from the top
  uint32_t cum = excl;
  int b = top - 1;
  for (; b > top - w; b--) {
    if (cum + hq[b] >= need) break;
    cum += hq[b];
  }
  const uint32_t newprefix = (L == 1) ? (uint32_t)b : ((prefix << (L == 2 ? 12 : 8)) | (uint32_t)b);
  uint32_t kmin = newprefix << sh;
  if (kmin == 0) kmin = 1;
  st[S_PREFIX] = newprefix;
  st[S_LEVEL] = L;
  st[S_ABOVE] = above + cum;
  st[S_KMIN] = kmin;
  if (above + cum + hq[b] <= (uint32_t)SEL_CAP) {
    st[S_DONE] = 1;
  } else if (L == 3) {
    // exact key reached and still too many equal keys: ordered tie pass
    st[S_DONE] = 1;
    st[S_TIES] = 1;
    atomicOr(flags, TACHIOM_FLAG_SELECT_TIES);
  }
}

// The dense row q, chunk [b0, e0): f(x, v) for every reached document, with
// 16-byte loads (4 in flight per thread) on the aligned middle of the chunk.
template <typename F>
__device__ __forceinline__ void sel_scan(const float *__restrict__ dq, int64_t row_base, int64_t b0, int64_t e0,
                                         F f) {
  const int64_t xa = min(e0, b0 + ((4 - ((row_base + b0) & 3)) & 3));
  const int64_t xe = xa + ((e0 - xa) & ~(int64_t)15);
  for (int64_t x = b0 + threadIdx.x; x < xa; x += blockDim.x) f(x, dq[x]);
  const float4 *v4 = reinterpret_cast<const float4 *>(dq + xa);
  const int64_t n4 = (xe - xa) >> 2;
  for (int64_t i = threadIdx.x; i < n4; i += 4 * (int64_t)blockDim.x) {
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; u++)
      v[u] = (i + u * blockDim.x < n4) ? v4[i + u * blockDim.x] : make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const int64_t x = xa + 4 * (i + u * blockDim.x);
      f(x, v[u].x);
      f(x + 1, v[u].y);
      f(x + 2, v[u].z);
      f(x + 3, v[u].w);
    }
  }
  for (int64_t x = xe + threadIdx.x; x < e0; x += blockDim.x) f(x, dq[x]);
}

__global__ void __launch_bounds__(SEL_THREADS)
k_sel_hist(const float *__restrict__ dense, int64_t D, const uint32_t *__restrict__ state,
           uint32_t *__restrict__ hist, int L) {
  const int q = blockIdx.y;
  const uint32_t *st = state + (int64_t)q * 8;
  if (st[S_DONE]) return;
  __shared__ uint32_t h[NBINS1];
  const int nb = level_bins(L);
  for (int b = threadIdx.x; b < nb; b += SEL_THREADS) h[b] = 0u;
  __syncthreads();
  const uint32_t prefix = st[S_PREFIX];
  const int psh = (L == 2) ? 20 : 8;  // bits above this level's bins
  const int sh = level_shift(L);
  const int64_t b0 = (int64_t)blockIdx.x * SEL_CHUNK;
  const int64_t e0 = min(D, b0 + SEL_CHUNK);
  const float *dq = dense + (int64_t)q * D;
  sel_scan(dq, (int64_t)q * D, b0, e0, [&](int64_t, float v) {
    if (v == -INFINITY) return;
    const uint32_t k = fkey(v);
    if ((k >> psh) == prefix) atomicAdd(&h[(k >> sh) & (nb - 1)], 1u);
  });
  __syncthreads();
  uint32_t *hq = hist + (int64_t)q * NBINS1;
  for (int b = threadIdx.x; b < nb; b += SEL_THREADS)
    if (h[b]) atomicAdd(&hq[b], h[b]);
}

__global__ void __launch_bounds__(SEL_THREADS)
k_sel_collect(const float *__restrict__ dense, int64_t D, uint32_t *__restrict__ state,
              uint64_t *__restrict__ selbuf, uint32_t *__restrict__ flags) {
  const int q = blockIdx.y;
  uint32_t *st = state + (int64_t)q * 8;
  const uint32_t kmin = st[S_KMIN];
  const bool ties = st[S_TIES] != 0;
  const int64_t b0 = (int64_t)blockIdx.x * SEL_CHUNK;
  const int64_t e0 = min(D, b0 + SEL_CHUNK);
  const float *dq = dense + (int64_t)q * D;
  uint64_t *buf = selbuf + (int64_t)q * SEL_CAP;
  // the block's keys are gathered in shared memory and reserved in the query's buffer with one
  // atomic (the per-query counter is shared by every block of the query)
  __shared__ uint64_t sk[SEL_LOCAL];
  __shared__ uint32_t scnt, sbase;
  if (threadIdx.x == 0) scnt = 0u;
  __syncthreads();
  sel_scan(dq, (int64_t)q * D, b0, e0, [&](int64_t x, float v) {
    if (v == -INFINITY) return;
    const uint32_t k = fkey(v);
    if (ties ? (k > kmin) : (k >= kmin)) {
      const uint32_t p = atomicAdd(&scnt, 1u);
      if (p < (uint32_t)SEL_LOCAL) {
        sk[p] = comp_key(v, (int32_t)x);
      } else {
        const uint32_t pos = atomicAdd(&st[S_CNT], 1u);
        if (pos < (uint32_t)SEL_CAP) buf[pos] = comp_key(v, (int32_t)x);
        else atomicOr(flags, TACHIOM_FLAG_CAPACITY);
      }
    }
  });
  __syncthreads();
  const uint32_t n = min(scnt, (uint32_t)SEL_LOCAL);
  if (threadIdx.x == 0) sbase = n ? atomicAdd(&st[S_CNT], n) : 0u;
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const uint32_t pos = sbase + i;
    if (pos < (uint32_t)SEL_CAP) buf[pos] = sk[i];
    else atomicOr(flags, TACHIOM_FLAG_CAPACITY);
  }
}

// ordered pass for a cut inside a long run of equal keys: the lowest doc ids win
__global__ void __launch_bounds__(1024)
k_sel_ties(const float *__restrict__ dense, int64_t D, uint32_t *__restrict__ state,
           uint64_t *__restrict__ selbuf, const int32_t *__restrict__ meta, int nq, int kd_max) {
  const int q = blockIdx.x;
  const int kd = min(kd_max, meta[4 * nq + 2 + q]);
  uint32_t *st = state + (int64_t)q * 8;
  if (!st[S_TIES]) return;
  __shared__ int s_taken;
  __shared__ int warp_cnt[32];
  const uint32_t kmin = st[S_KMIN];
  const float *dq = dense + (int64_t)q * D;
  uint64_t *buf = selbuf + (int64_t)q * SEL_CAP;
  const int base = (int)umin(st[S_CNT], (uint32_t)SEL_CAP);
  const int need = kd - base;
  if (threadIdx.x == 0) s_taken = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t c0 = 0; c0 < D; c0 += 1024) {
    if (s_taken >= need) break;
    int64_t x = c0 + threadIdx.x;
    bool hit = x < D && dq[x] != -INFINITY && fkey(dq[x]) == kmin;
    unsigned m = __ballot_sync(0xffffffffu, hit);
    if (lane == 0) warp_cnt[warp] = __popc(m);
    __syncthreads();
    int before = s_taken;
    for (int w = 0; w < warp; w++) before += warp_cnt[w];
    before += __popc(m & ((1u << lane) - 1));
    if (hit && before < need && base + before < SEL_CAP) buf[base + before] = comp_key(dq[x], (int32_t)x);
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int w = 0; w < 32; w++) t += warp_cnt[w];
      s_taken += t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) st[S_CNT] = (uint32_t)(base + min(s_taken, need));
}

// Per query: the collected keys (n <= SEL_CAP, all at or above the cut) in
// shared memory; the first min(n, kappa_d) by (S~ desc, doc asc) are written.
// Small buffers are sorted whole. A large one first finds the kappa_d-th
// largest key T by a radix select over the 64-bit keys (8 passes of 8 bits; the
// keys are unique, the doc id being part of the key), keeps the kappa_d keys
// >= T and sorts only those.
constexpr int SORT_THREADS = 1024;
constexpr int SORT_SMALL = 2048;
__global__ void __launch_bounds__(SORT_THREADS)
k_sel_sort(uint32_t *__restrict__ state, uint64_t *__restrict__ selbuf, const int32_t *__restrict__ meta, int nq,
           int kd, int32_t *__restrict__ cand, float *__restrict__ cand_s, int32_t *__restrict__ ncand) {
  extern __shared__ __align__(16) uint64_t ssm[];  // [SEL_CAP] keys, then [next_pow2(kappa_d)] kept keys
  __shared__ uint32_t hist[256];
  __shared__ uint64_t s_prefix;
  __shared__ uint32_t s_need;
  __shared__ int s_cnt;
  const int q = blockIdx.x;
  const int kdq = min(kd, meta[4 * nq + 2 + q]);  // this query's cut; the row stride stays kd
  const uint32_t *st = state + (int64_t)q * 8;
  const int n = (int)umin(st[S_CNT], (uint32_t)SEL_CAP);
  const uint64_t *buf = selbuf + (int64_t)q * SEL_CAP;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = min(n, kdq);
  uint64_t *keys = ssm;
  if (n <= SORT_SMALL || n <= kdq) {
    const int np = next_pow2(max(n, 2));
    for (int i = tid; i < np; i += SORT_THREADS) keys[i] = i < n ? buf[i] : 0ull;
    __syncthreads();
    block_sort_desc(keys, np);
  } else {
    for (int i = tid; i < n; i += SORT_THREADS) keys[i] = buf[i];
    uint64_t prefix = 0ull;
    uint32_t need = (uint32_t)kdq;
    for (int pass = 0; pass < 8; pass++) {
      const int shift = 56 - 8 * pass;
      const uint64_t hi = pass == 0 ? 0ull : (~0ull << (shift + 8));
      if (tid < 256) hist[tid] = 0u;
      __syncthreads();
      for (int b0 = 0; b0 < n; b0 += SORT_THREADS) {
        const int i = b0 + tid;
        int dg = -1;
        if (i < n) {
          const uint64_t k = keys[i];
          if ((k & hi) == prefix) dg = (int)((k >> shift) & 255u);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        if (dg >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[dg], (uint32_t)__popc(peers));
      }
      __syncthreads();
      if (warp == 0) {
        // lane l: digits [248 - 8l, 256 - 8l), from the top
        uint32_t c = 0;
        for (int d = 255 - 8 * lane; d > 247 - 8 * lane; d--) c += hist[d];
        uint32_t inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
          if (lane >= o) inc += y;
        }
        const uint32_t excl = inc - c;
        if (excl < need && need <= inc) {
          uint32_t cum = excl;
          int d = 255 - 8 * lane;
          for (; d > 248 - 8 * lane; d--) {
            if (cum + hist[d] >= need) break;
            cum += hist[d];
          }
          s_prefix = prefix | ((uint64_t)d << shift);
          s_need = need - cum;
        }
      }
      __syncthreads();
      prefix = s_prefix;
      need = s_need;
    }
    // prefix is now the kappa_d-th largest key: keep the kappa_d keys >= it, sort them
    uint64_t *kept = ssm + SEL_CAP;
    const int np = next_pow2(max(kdq, 2));
    if (tid == 0) s_cnt = 0;
    for (int i = kdq + tid; i < np; i += SORT_THREADS) kept[i] = 0ull;
    __syncthreads();
    for (int i = tid; i < n; i += SORT_THREADS) {
      const uint64_t k = keys[i];
      if (k >= prefix) {
        const int pos = atomicAdd(&s_cnt, 1);
        if (pos < kdq) kept[pos] = k;
      }
    }
    __syncthreads();
    block_sort_desc(kept, np);
    keys = kept;
  }
  for (int i = tid; i < kd; i += SORT_THREADS) {
    const uint64_t v = i < m ? keys[i] : 0ull;
    cand[(int64_t)q * kd + i] = v ? comp_id(v) : -1;
    cand_s[(int64_t)q * kd + i] = v ? comp_score(v) : -INFINITY;
  }
  if (tid == 0) ncand[q] = m;
}

tachiom_status launch_select_kd(const Index &ix, const int32_t *meta, int nq, int kd, const float *dense,
                                const uint32_t *hist,
                                uint32_t *hist2, uint32_t *state, uint64_t *selbuf, int32_t *cand,
                                float *cand_s, int32_t *ncand, uint32_t *flags, cudaStream_t s) {
  if (nq <= 0) return TACHIOM_OK;
  TPROF("select_kd", s);
  const int64_t D = ix.D;
  dim3 grid((unsigned)((D + SEL_CHUNK - 1) / SEL_CHUNK), nq);
  k_sel_find<<<nq, FIND_THREADS, 0, s>>>(hist, state, meta, nq, kd, 1, flags);
  TLAUNCH();
  for (int L = 2; L <= 3; L++) {
    TCUDA(cudaMemsetAsync(hist2, 0, (size_t)nq * NBINS1 * 4, s));
    k_sel_hist<<<grid, SEL_THREADS, 0, s>>>(dense, D, state, hist2, L);
    TLAUNCH();
    k_sel_find<<<nq, FIND_THREADS, 0, s>>>(hist2, state, meta, nq, kd, L, flags);
    TLAUNCH();
  }
  k_sel_collect<<<grid, SEL_THREADS, 0, s>>>(dense, D, state, selbuf, flags);
  TLAUNCH();
  k_sel_ties<<<nq, 1024, 0, s>>>(dense, D, state, selbuf, meta, nq, kd);
  TLAUNCH();
  const size_t smem = (size_t)SEL_CAP * 8 + (size_t)next_pow2(std::max(kd, 2)) * 8;
  TCUDA(cudaFuncSetAttribute(k_sel_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_sel_sort<<<nq, SORT_THREADS, smem, s>>>(state, selbuf, meta, nq, kd, cand, cand_s, ncand);
  TLAUNCH();
  return TACHIOM_OK;
}

}  // namespace tachiom
