// Step (c) with the centroid term on the tensor cores (BF16 path), then the
// FP32 repair of the top-k boundary.
//
// S(q,d) = sum_i max_{t in d} ( <q_i, c_a(t)> + rho_t * sum_m T[m][code_{t,m}][i] )
//
// k_refine_tc computes the same sum as k_refine, with the centroid term from
// mma.sync m16n8k16 (rows: 16 document tokens, columns: 8 query tokens,
// K = 128): the centroid rows are gathered (bf16, exact for a bf16-stored
// table) into a padded per-warp staging tile and read with ldmatrix; the query
// side is split into q = q_hi + q_lo (both bf16), so two MMAs give the product
// to about 2^-17 relative. The residual term is the same ADC lookup as
// k_refine: FP32 tables in shared memory in the query-token-major micro-block
// layout, 16-byte code loads, the same summation order over m, so it is
// bit-identical to the FP32 path; only the centroid term differs, by at most
// delta_c per (i, t).
//
// k_refine_window turns the approximate scores into a short list per query:
// with Delta = n_q * delta_c (+ rounding of the sums) bounding |S_approx -
// S_fp32|, every document of the exact top-k has S_approx >= (approximate
// k-th score) - 2 Delta, so rescoring that window with the FP32 kernels and
// keeping its top-k gives the FP32 path's answer.
#include <cuda_fp16.h>

#include "tachiom_internal.cuh"

namespace tachiom {

constexpr int RT_THREADS = 256;
constexpr int RT_WARPS = RT_THREADS / 32;
constexpr int RT_DOCS_PER_CTA = 128;
constexpr int RT_ROW_BYTES = 272;  // 256-byte bf16 row + 16 bytes of padding (conflict-free ldmatrix)
constexpr int RT_STAGE = 16 * RT_ROW_BYTES;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void mma16816(float *d, const uint32_t *a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// position of a warp in its stream of 16-token chunks over its candidate documents
struct ChunkPos {
  int slot;       // candidate slot of the current document
  int64_t tb, te; // its tokens
  int64_t c0;     // first token of the chunk
};

// Advance to the next chunk: the next 16 tokens of the same document, else the
// first chunk of the warp's next candidate that has tokens. Candidates that are
// empty documents get S = 0 here; out-of-range ids raise the bad-input flag.
__device__ __forceinline__ bool next_chunk(ChunkPos &p, int s_end, int step, const int32_t *cand_q,
                                           const int64_t *doc_off, int64_t D, float *part_row,
                                           uint32_t *flags, int lane) {
  if (p.c0 + 16 < p.te) {
    p.c0 += 16;
    return true;
  }
  for (p.slot += step; p.slot < s_end; p.slot += step) {
    const int32_t d = cand_q[p.slot];
    if (d < 0) continue;
    if (d >= D) {
      if (lane == 0) {
        atomicOr(flags, TACHIOM_FLAG_BAD_INPUT);
        part_row[p.slot] = 0.f;
      }
      continue;
    }
    p.tb = doc_off[d];
    p.te = doc_off[d + 1];
    if (p.te == p.tb) {
      if (lane == 0) part_row[p.slot] = 0.f;
      continue;
    }
    p.c0 = p.tb;
    return true;
  }
  return false;
}

template <int M>
__global__ void __launch_bounds__(RT_THREADS, 1)
k_refine_tc(const float *__restrict__ queries, const int32_t *__restrict__ meta, int nq,
            const int32_t *__restrict__ cand, int kd, const int64_t *__restrict__ doc_off,
            const int32_t *__restrict__ tok_cid, const uint8_t *__restrict__ codes,
            const uint16_t *__restrict__ rnorm, const float *__restrict__ codebooks,
            const __nv_bfloat16 *__restrict__ cent_bf16, float *__restrict__ part, int ngroups, int64_t D,
            uint32_t *__restrict__ flags) {
  constexpr int G = 128 / M;                 // query tokens per CTA (table = 128 KB)
  constexpr int DS = 128 / M;
  constexpr int NT = (G + 7) / 8;            // n-tiles of 8 query tokens
  constexpr int CW = (M >= 16 ? M / 16 : 1); // 16-byte code words per token (8-byte for M = 8)
  extern __shared__ __align__(16) unsigned char rts[];
  float *tab = reinterpret_cast<float *>(rts);                    // [M][256][G]
  float *qs = tab + M * 256 * G;                                   // [G][128]
  unsigned char *stage_all = reinterpret_cast<unsigned char *>(qs + G * DIM);  // [warps][2][16 rows][272 B]

  const int q = blockIdx.z, grp = blockIdx.y;
  const int ntok = meta[3 * nq + 2 + q];
  const int i0g = grp * G;
  if (i0g >= ntok) return;
  const int s_begin = blockIdx.x * RT_DOCS_PER_CTA;
  const int s_end = min(kd, s_begin + RT_DOCS_PER_CTA);
  const int32_t *cand_q = cand + (int64_t)q * kd;
  {
    // nothing to do in this slice (a short FP32 window): skip the tables
    int any = 0;
    for (int i = s_begin + (int)threadIdx.x; i < s_end && !any; i += RT_THREADS) any = cand_q[i] >= 0;
    if (!__syncthreads_or(any)) return;
  }
  const int ng = min(G, ntok - i0g);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gq = lane >> 2, tig = lane & 3;

  const float *qrow = queries + (int64_t)(meta[q] + i0g) * DIM;
  for (int x = tid; x < G * DIM; x += RT_THREADS) qs[x] = (x / DIM < ng) ? qrow[x] : 0.f;
  __syncthreads();
  // ADC tables T[m][j][g] = <q_g^(m), w_{m,j}> (same arithmetic as k_refine)
  for (int mj = tid; mj < M * 256; mj += RT_THREADS) {
    const int m = mj / 256;
    const float *w = codebooks + (int64_t)mj * DS;
    float wv[DS];
#pragma unroll
    for (int u = 0; u < DS; u++) wv[u] = w[u];
#pragma unroll
    for (int g = 0; g < G; g++) {
      float a = 0.f;
#pragma unroll
      for (int u = 0; u < DS; u++) a = fmaf(qs[g * DIM + m * DS + u], wv[u], a);
      tab[mj * G + g] = a;
    }
  }
  __syncthreads();
  // B fragments of the query tokens, split hi + lo
  uint32_t bh[NT][8][2], bl[NT][8][2];
#pragma unroll
  for (int nt = 0; nt < NT; nt++) {
    const int n = nt * 8 + gq;
#pragma unroll
    for (int s = 0; s < 8; s++) {
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int k = s * 16 + h * 8 + tig * 2;
        const float x0 = n < G ? qs[n * DIM + k] : 0.f, x1 = n < G ? qs[n * DIM + k + 1] : 0.f;
        const float h0 = __bfloat162float(__float2bfloat16_rn(x0));
        const float h1 = __bfloat162float(__float2bfloat16_rn(x1));
        bh[nt][s][h] = pack_bf16(h0, h1);
        bl[nt][s][h] = pack_bf16(x0 - h0, x1 - h1);
      }
    }
  }
  unsigned char *stage = stage_all + warp * 2 * RT_STAGE;
  const uint32_t stage_s = (uint32_t)__cvta_generic_to_shared(stage);
  // ldmatrix row address of this lane: matrix j = lane / 8 -> rows (j & 1) * 8 + lane % 8, cols (j >> 1) * 8
  const uint32_t lm_off = (uint32_t)((((lane >> 3) & 1) * 8 + (lane & 7)) * RT_ROW_BYTES + ((lane >> 4) * 8) * 2);
  float *part_row = part + ((int64_t)q * ngroups + grp) * kd;

  // issue the gathers of one chunk: centroid rows (cp.async into stage b) and, into
  // registers, the codes and norms of this thread's two tokens (rows gq, gq + 8)
  auto issue = [&](const ChunkPos &p, int b, uint4 (&cw)[2][CW], float (&rh)[2]) {
    const int64_t tl = p.c0 + (lane & 15);
    const int32_t cid_l = (tl < p.te) ? tok_cid[tl] : 0;
    const uint32_t dst0 = stage_s + (uint32_t)(b * RT_STAGE);
#pragma unroll
    for (int it = 0; it < 8; it++) {
      const int qq = it * 32 + lane;
      const int row = qq >> 4, pc = qq & 15;
      const int32_t cr = __shfl_sync(0xffffffffu, cid_l, row);
      const __nv_bfloat16 *src = cent_bf16 + (int64_t)cr * DIM + pc * 8;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst0 + (uint32_t)(row * RT_ROW_BYTES + pc * 16)),
                   "l"(src)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int64_t t = p.c0 + gq + h * 8;
      if (t < p.te) {
#pragma unroll
        for (int u = 0; u < CW; u++) {
          if constexpr (M >= 16) {
            cw[h][u] = *reinterpret_cast<const uint4 *>(codes + t * M + u * 16);
          } else {
            const uint2 v2 = *reinterpret_cast<const uint2 *>(codes + t * M);
            cw[h][u] = make_uint4(v2.x, v2.y, 0u, 0u);
          }
        }
        rh[h] = __half2float(__ushort_as_half(rnorm[t]));
      } else {
        rh[h] = 0.f;
      }
    }
  };

  ChunkPos cur;
  cur.slot = s_begin + warp - RT_WARPS;
  cur.tb = cur.te = cur.c0 = 0;
  bool has = next_chunk(cur, s_end, RT_WARPS, cand_q, doc_off, D, part_row, flags, lane);
  uint4 cw_cur[2][CW], cw_nxt[2][CW];
  float rh_cur[2], rh_nxt[2];
  int b = 0;
  if (has) issue(cur, b, cw_cur, rh_cur);
  float mx[NT][2];
#pragma unroll
  for (int nt = 0; nt < NT; nt++) mx[nt][0] = mx[nt][1] = -INFINITY;
  while (has) {
    ChunkPos nxt = cur;
    const bool hn = next_chunk(nxt, s_end, RT_WARPS, cand_q, doc_off, D, part_row, flags, lane);
    if (hn) {
      issue(nxt, b ^ 1, cw_nxt, rh_nxt);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncwarp();
    // centroid term: 16 tokens x 8 query tokens per n-tile, K = 128
    float acc[NT][4];
#pragma unroll
    for (int nt = 0; nt < NT; nt++) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
    const uint32_t lm = stage_s + (uint32_t)(b * RT_STAGE) + lm_off;
#pragma unroll
    for (int s = 0; s < 8; s++) {
      uint32_t a[4];
      asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                   : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                   : "r"(lm + s * 32)
                   : "memory");
#pragma unroll
      for (int nt = 0; nt < NT; nt++) {
        mma16816(acc[nt], a, bh[nt][s][0], bh[nt][s][1]);
        mma16816(acc[nt], a, bl[nt][s][0], bl[nt][s][1]);
      }
    }
    // residual term from the tables, same order over m as the FP32 kernel
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int64_t t = cur.c0 + gq + h * 8;
      if (t >= cur.te) continue;
      const uint8_t *cb = reinterpret_cast<const uint8_t *>(cw_cur[h]);
#pragma unroll
      for (int nt = 0; nt < NT; nt++) {
        const int i0 = nt * 8 + tig * 2;
        if (i0 >= G) continue;
        float r0 = 0.f, r1 = 0.f;
#pragma unroll
        for (int m = 0; m < M; m++) {
          const float2 tv = *reinterpret_cast<const float2 *>(tab + (m * 256 + cb[m]) * G + i0);
          r0 += tv.x;
          r1 += tv.y;
        }
        mx[nt][0] = fmaxf(mx[nt][0], fmaf(rh_cur[h], r0, acc[nt][h * 2 + 0]));
        mx[nt][1] = fmaxf(mx[nt][1], fmaf(rh_cur[h], r1, acc[nt][h * 2 + 1]));
      }
    }
    if (!hn || nxt.slot != cur.slot) {
      // the document is complete: max over the 8 lanes sharing tig, then the sum over query tokens
      float sum = 0.f;
#pragma unroll
      for (int nt = 0; nt < NT; nt++) {
#pragma unroll
        for (int e = 0; e < 2; e++) {
          float v = mx[nt][e];
          v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 4));
          v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 8));
          v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 16));
          const int i = nt * 8 + tig * 2 + e;
          if (i < ng) sum += v;
          mx[nt][e] = -INFINITY;
        }
      }
      sum += __shfl_xor_sync(0xffffffffu, sum, 1);
      sum += __shfl_xor_sync(0xffffffffu, sum, 2);
      if (lane == 0) part_row[cur.slot] = sum;
    }
    __syncwarp();  // stage b is free for the chunk after next
    cur = nxt;
    has = hn;
    b ^= 1;
#pragma unroll
    for (int h = 0; h < 2; h++) {
      rh_cur[h] = rh_nxt[h];
#pragma unroll
      for (int u = 0; u < CW; u++) cw_cur[h][u] = cw_nxt[h][u];
    }
  }
}

template <int M>
static tachiom_status launch_refine_tc_m(const Index &ix, const float *queries, const int32_t *meta, int nq,
                                         const int32_t *cand, int kd, float *part, uint32_t *flags, cudaStream_t s) {
  constexpr int G = 128 / M;
  const int ngroups = refine_groups(M);
  const size_t smem = ((size_t)M * 256 * G + (size_t)G * DIM) * 4 + (size_t)RT_WARPS * 2 * RT_STAGE;
  dim3 grid((kd + RT_DOCS_PER_CTA - 1) / RT_DOCS_PER_CTA, ngroups, nq);
  TCUDA(cudaFuncSetAttribute(k_refine_tc<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_refine_tc<M><<<grid, RT_THREADS, smem, s>>>(queries, meta, nq, cand, kd, ix.doc_off, ix.tok_cid, ix.codes,
                                                 ix.rnorm, ix.codebooks, ix.cent_bf16, part, ngroups, ix.D, flags);
  TLAUNCH();
  return TACHIOM_OK;
}

tachiom_status launch_refine_tc(const Index &ix, const float *queries, const int32_t *meta, int nq,
                                const int32_t *cand, int kd, float *part, uint32_t *flags, cudaStream_t s) {
  if (nq <= 0) return TACHIOM_OK;
  TPROF("refine_tc", s);
  switch (ix.M) {
    case 8: return launch_refine_tc_m<8>(ix, queries, meta, nq, cand, kd, part, flags, s);
    case 16: return launch_refine_tc_m<16>(ix, queries, meta, nq, cand, kd, part, flags, s);
    case 32: return launch_refine_tc_m<32>(ix, queries, meta, nq, cand, kd, part, flags, s);
  }
  return fail(TACHIOM_ERR_INVALID, "unsupported pq_m %d", ix.M);
}

// Per query: approximate S = sum of group partials; the documents whose S is
// within 2 * Delta of the approximate k-th score go to `win` (padded with -1),
// in (S desc, doc asc) order.
__global__ void __launch_bounds__(1024)
k_refine_window(const int32_t *__restrict__ meta, int nq, const int32_t *__restrict__ cand, int kd,
                const float *__restrict__ part, int ngroups, int G, float delta_per_token,
                int32_t *__restrict__ win) {
  extern __shared__ __align__(16) uint64_t wsm[];
  __shared__ float s_lim;
  const int q = blockIdx.x;
  const int ntok = meta[3 * nq + 2 + q];
  const int k = meta[2 * nq + 2 + q];
  const int gq = (ntok + G - 1) / G;
  const int np = next_pow2(max(kd, 2));
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    uint64_t v = 0ull;
    if (i < kd) {
      const int32_t d = cand[(int64_t)q * kd + i];
      if (d >= 0) {
        float s = 0.f;
        for (int g = 0; g < gq; g++) s += part[((int64_t)q * ngroups + g) * kd + i];
        v = comp_key(s, d);
      }
    }
    wsm[i] = v;
  }
  __syncthreads();
  block_sort_desc(wsm, np);
  if (threadIdx.x == 0) {
    const uint64_t kth = wsm[min(k, np) - 1];
    if (!kth) {
      s_lim = -INFINITY;  // fewer than k candidates: all of them
    } else {
      const float sk = comp_score(kth);
      // Delta: n_q centroid-term bounds plus the rounding of two differently ordered sums
      const float delta = ntok * delta_per_token + 4.f * ldexpf(fabsf(sk) + 1.f, -20);
      s_lim = sk - 2.f * delta;
    }
  }
  __syncthreads();
  const float lim = s_lim;
  for (int i = threadIdx.x; i < kd; i += blockDim.x) {
    const uint64_t v = i < np ? wsm[i] : 0ull;
    win[(int64_t)q * kd + i] = (v && comp_score(v) >= lim) ? comp_id(v) : -1;
  }
}

tachiom_status launch_refine_window(const Index &ix, const int32_t *meta, int nq, const int32_t *cand, int kd,
                                    const float *part, float delta_per_token, int32_t *win, cudaStream_t s) {
  if (nq <= 0) return TACHIOM_OK;
  TPROF("refine_window", s);
  const size_t smem = (size_t)next_pow2(std::max(kd, 2)) * 8;
  TCUDA(cudaFuncSetAttribute(k_refine_window, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_refine_window<<<nq, 1024, smem, s>>>(meta, nq, cand, kd, part, refine_groups(ix.M), 128 / ix.M,
                                         delta_per_token, win);
  TLAUNCH();
  return TACHIOM_OK;
}

// diagnostics: the approximate S of every candidate slot (sum of the group partials)
__global__ void k_refine_sum(const int32_t *__restrict__ meta, int nq, const int32_t *__restrict__ cand, int kd,
                             const float *__restrict__ part, int ngroups, int G, float *__restrict__ out) {
  const int q = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kd) return;
  const int gq = (meta[3 * nq + 2 + q] + G - 1) / G;
  float s = 0.f;
  for (int g = 0; g < gq; g++) s += part[((int64_t)q * ngroups + g) * kd + i];
  out[(int64_t)q * kd + i] = cand[(int64_t)q * kd + i] >= 0 ? s : -INFINITY;
}

tachiom_status launch_refine_sum(const Index &ix, const int32_t *meta, int nq, const int32_t *cand, int kd,
                                 const float *part, float *out, cudaStream_t s) {
  if (nq <= 0) return TACHIOM_OK;
  k_refine_sum<<<dim3((kd + 255) / 256, nq), 256, 0, s>>>(meta, nq, cand, kd, part, refine_groups(ix.M), 128 / ix.M,
                                                          out);
  TLAUNCH();
  return TACHIOM_OK;
}

// Per query: the documents that can still be in the exact top-k after the
// decode-and-MMA pass, each with its own bound da: sa - da <= S <= sa + da. The
// k-th largest lower bound L is at most the exact k-th score, so a document
// with sa + da < L is strictly below it and never reaches the top-k; the others
// (sorted by upper bound, first) go to the FP32 kernel. A document whose bound
// is not finite is always kept. The bounds are widened by 2^-22 (|sa| + da) to
// cover the rounding of the two sums.
__device__ __forceinline__ void window_bounds(float s, float e, float *lo, float *up) {
  if (isfinite(s) && e <= 3.0e38f) {
    const float w = ldexpf(fabsf(s) + e, -22);
    *lo = (s - e) - w;
    *up = (s + e) + w;
  } else {
    *lo = -INFINITY;
    *up = INFINITY;
  }
}

__global__ void __launch_bounds__(1024)
k_refine_window_b(const int32_t *__restrict__ meta, int nq, const int32_t *__restrict__ cand, int kd,
                  const float *__restrict__ sa, const float *__restrict__ da, int32_t *__restrict__ win,
                  int32_t *__restrict__ win_slot) {
  extern __shared__ __align__(16) uint64_t wsm2[];
  __shared__ float s_lim;
  const int q = blockIdx.x;
  const int k = meta[2 * nq + 2 + q];
  const int np = next_pow2(max(kd, 2));
  for (int pass = 0; pass < 2; pass++) {
    // pass 0: keys of the lower bounds (for L); pass 1: keys of the upper bounds
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
      uint64_t v = 0ull;
      if (i < kd) {
        const int32_t d = cand[(int64_t)q * kd + i];
        const float s = sa[(int64_t)q * kd + i];
        if (d >= 0 && s != -INFINITY) {
          float lo, up;
          window_bounds(s, da[(int64_t)q * kd + i], &lo, &up);
          v = comp_key(pass == 0 ? lo : up, i);  // the slot rides in the key: win_slot below
        }
      }
      wsm2[i] = v;
    }
    __syncthreads();
    block_sort_desc(wsm2, np);
    if (pass == 0) {
      if (threadIdx.x == 0) {
        const uint64_t kth = wsm2[min(k, np) - 1];
        s_lim = kth ? comp_score(kth) : -INFINITY;
      }
      __syncthreads();
    }
  }
  const float lim = s_lim;
  for (int i = threadIdx.x; i < kd; i += blockDim.x) {
    const uint64_t v = i < np ? wsm2[i] : 0ull;
    const bool in = v && comp_score(v) >= lim;
    const int32_t slot = in ? comp_id(v) : -1;
    win[(int64_t)q * kd + i] = in ? cand[(int64_t)q * kd + slot] : -1;
    win_slot[(int64_t)q * kd + i] = slot;
  }
}

tachiom_status launch_refine_window_b(const Index &ix, const int32_t *meta, int nq, const int32_t *cand, int kd,
                                      const float *sa, const float *da, int32_t *win, int32_t *win_slot,
                                      cudaStream_t s) {
  if (nq <= 0) return TACHIOM_OK;
  TPROF("refine_window", s);
  const size_t smem = (size_t)next_pow2(std::max(kd, 2)) * 8;
  TCUDA(cudaFuncSetAttribute(k_refine_window_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_refine_window_b<<<nq, 1024, smem, s>>>(meta, nq, cand, kd, sa, da, win, win_slot);
  TLAUNCH();
  return TACHIOM_OK;
}

}  // namespace tachiom
