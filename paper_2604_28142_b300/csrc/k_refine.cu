// Steps (c) and (d): PQ-ADC refinement with full MaxSim (Sec. 2.2, Refine) and
// the final top-k.
//
//   S(q,d) = sum_i max_{t in d} ( <q_i, c_a(t)> + rho_t * sum_m T[m][code_{t,m}][i] )
//   T[m][j][i] = <q_i^(m), w_{m,j}>                  (ADC lookup tables)
//
// The tables use the paper's query-token-major layout (Sec. 2.2, "Distance
// Table Layout"): subspace m, then codeword j, then a contiguous micro-block of
// query tokens, so one code of one document token fetches the distances of
// all the CTA's query tokens from consecutive words. A full table for 32
// query tokens (M x 256 x 32 fp32 = 512 KB at M = 16) does not fit in shared
// memory, so a CTA owns a group of G = 128 / M query tokens (a 128 KB table)
// and the per-group partial sums of the max are added in ascending group
// order by the final kernel.
//
// Work mapping: a CTA = (query, token group, slice of candidates); a warp
// takes one candidate document at a time with one lane per document token;
// each lane loads its token's codes with 16-byte vector loads, its residual
// norm and its centroid row, and keeps a running max per query token of the
// group; a butterfly max across the lanes finishes the document.
#include <cuda_fp16.h>

#include "tachiom_internal.cuh"

namespace tachiom {

constexpr int R_THREADS = 512;
constexpr int R_DOCS_PER_CTA = 128;

int refine_groups(int M) { return (MAX_NTOK + (128 / M) - 1) / (128 / M); }

__device__ __forceinline__ float half_bits_to_float(uint16_t h) {
  return __half2float(__ushort_as_half(h));
}

template <int M, bool BF16C>
__global__ void __launch_bounds__(R_THREADS, 1)
k_refine(const float *__restrict__ queries, const int32_t *__restrict__ meta, int nq,
         const int32_t *__restrict__ cand, int kd, const int64_t *__restrict__ doc_off,
         const int32_t *__restrict__ tok_cid, const uint8_t *__restrict__ codes,
         const uint16_t *__restrict__ rnorm, const float *__restrict__ codebooks,
         const float *__restrict__ cent_f32, const __nv_bfloat16 *__restrict__ cent_bf16,
         float *__restrict__ part, int ngroups, int64_t D, uint32_t *__restrict__ flags) {
  constexpr int G = 128 / M;   // query tokens per CTA
  constexpr int DS = 128 / M;  // dims per subspace
  extern __shared__ __align__(16) float rsm[];
  float *tab = rsm;                   // [M][256][G]
  float *qs = tab + M * 256 * G;      // [G][128]

  const int q = blockIdx.z, grp = blockIdx.y;
  const int *qoff = meta;
  const int ntok = meta[3 * nq + 2 + q];
  const int i0 = grp * G;
  if (i0 >= ntok) return;
  {
    // nothing to do in this slice (e.g. the tail of a short rescoring window): skip the tables
    const int sb = blockIdx.x * R_DOCS_PER_CTA, se = min(kd, sb + R_DOCS_PER_CTA);
    int any = 0;
    for (int i = sb + (int)threadIdx.x; i < se && !any; i += R_THREADS) any = cand[(int64_t)q * kd + i] >= 0;
    if (!__syncthreads_or(any)) return;
  }
  const int ng = min(G, ntok - i0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  const float *qrow = queries + (int64_t)(qoff[q] + i0) * DIM;
  for (int x = tid; x < G * DIM; x += R_THREADS) qs[x] = (x / DIM < ng) ? qrow[x] : 0.f;
  __syncthreads();
  // K0: the group's tables, T[m][j][g] = <q_g^(m), w_{m,j}>
  for (int mj = tid; mj < M * 256; mj += R_THREADS) {
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

  // K4: candidates of this CTA's slice, one warp per document
  const int s_begin = blockIdx.x * R_DOCS_PER_CTA;
  const int s_end = min(kd, s_begin + R_DOCS_PER_CTA);
  for (int slot = s_begin + warp; slot < s_end; slot += R_THREADS / 32) {
    const int32_t d = cand[(int64_t)q * kd + slot];
    if (d < 0) continue;
    if (d >= D) {
      if (lane == 0) {
        atomicOr(flags, TACHIOM_FLAG_BAD_INPUT);
        part[((int64_t)q * ngroups + grp) * kd + slot] = 0.f;
      }
      continue;
    }
    const int64_t tb = doc_off[d], te = doc_off[d + 1];
    float mx[G];
#pragma unroll
    for (int g = 0; g < G; g++) mx[g] = -INFINITY;
    for (int64_t t = tb + lane; t < te; t += 32) {
      // codes: M bytes per token, 16-byte vector loads
      uint8_t cb[M];
      if constexpr (M == 8) {
        uint2 v = *reinterpret_cast<const uint2 *>(codes + t * M);
        *reinterpret_cast<uint2 *>(cb) = v;
      } else {
#pragma unroll
        for (int u = 0; u < M / 16; u++) {
          uint4 v = *reinterpret_cast<const uint4 *>(codes + t * M + u * 16);
          *reinterpret_cast<uint4 *>(cb + u * 16) = v;
        }
      }
      const float rho = rnorm ? half_bits_to_float(rnorm[t]) : 0.f;  // no norms: the centroid term alone
      const int32_t j = tok_cid[t];
      // centroid contribution <q_g, c_j>
      float ct[G];
#pragma unroll
      for (int g = 0; g < G; g++) ct[g] = 0.f;
      if (BF16C) {
        // the row in two halves, each loaded whole (8 loads in flight), used in k order
        const uint4 *crow = reinterpret_cast<const uint4 *>(cent_bf16 + (int64_t)j * DIM);
#pragma unroll 1
        for (int hh = 0; hh < 2; hh++) {
        uint4 cr[DIM / 16];
#pragma unroll
        for (int k8 = 0; k8 < DIM / 16; k8++) cr[k8] = crow[hh * (DIM / 16) + k8];
#pragma unroll
        for (int kq = 0; kq < DIM / 16; kq++) {
          const uint4 u = cr[kq];
          const int k8 = hh * (DIM / 16) + kq;
          float c[8] = {__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                        __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u),
                        __uint_as_float(u.z << 16), __uint_as_float(u.z & 0xffff0000u),
                        __uint_as_float(u.w << 16), __uint_as_float(u.w & 0xffff0000u)};
#pragma unroll
          for (int g = 0; g < G; g++) {
            const float4 qa = *reinterpret_cast<const float4 *>(&qs[g * DIM + k8 * 8]);
            const float4 qb = *reinterpret_cast<const float4 *>(&qs[g * DIM + k8 * 8 + 4]);
            float a = ct[g];
            a = fmaf(qa.x, c[0], a); a = fmaf(qa.y, c[1], a); a = fmaf(qa.z, c[2], a); a = fmaf(qa.w, c[3], a);
            a = fmaf(qb.x, c[4], a); a = fmaf(qb.y, c[5], a); a = fmaf(qb.z, c[6], a); a = fmaf(qb.w, c[7], a);
            ct[g] = a;
          }
        }
        }
      } else {
        // the row in batches, each loaded whole (4 or 8 loads in flight), used in k order
        const float4 *crow = reinterpret_cast<const float4 *>(cent_f32 + (int64_t)j * DIM);
        constexpr int NB = G >= 16 ? DIM / 32 : DIM / 16;  // float4 per batch (register budget)
#pragma unroll 1
        for (int hh = 0; hh < DIM / 4 / NB; hh++) {
          float4 cr[NB];
#pragma unroll
          for (int k4 = 0; k4 < NB; k4++) cr[k4] = crow[hh * NB + k4];
#pragma unroll
          for (int k4 = 0; k4 < NB; k4++) {
            const float4 c = cr[k4];
            const int kk = hh * NB + k4;
#pragma unroll
            for (int g = 0; g < G; g++) {
              const float4 qa = *reinterpret_cast<const float4 *>(&qs[g * DIM + kk * 4]);
              float a = ct[g];
              a = fmaf(qa.x, c.x, a); a = fmaf(qa.y, c.y, a); a = fmaf(qa.z, c.z, a); a = fmaf(qa.w, c.w, a);
              ct[g] = a;
            }
          }
        }
      }
      // residual contribution from the tables (micro-block of G query tokens per code)
      float rs[G];
#pragma unroll
      for (int g = 0; g < G; g++) rs[g] = 0.f;
#pragma unroll
      for (int m = 0; m < M; m++) {
        const float *blk = tab + (m * 256 + cb[m]) * G;
        if constexpr (G % 4 == 0) {
#pragma unroll
          for (int g4 = 0; g4 < G / 4; g4++) {
            float4 v = *reinterpret_cast<const float4 *>(blk + g4 * 4);
            rs[g4 * 4 + 0] += v.x; rs[g4 * 4 + 1] += v.y; rs[g4 * 4 + 2] += v.z; rs[g4 * 4 + 3] += v.w;
          }
        } else {
#pragma unroll
          for (int g = 0; g < G; g++) rs[g] += blk[g];
        }
      }
#pragma unroll
      for (int g = 0; g < G; g++) mx[g] = fmaxf(mx[g], fmaf(rho, rs[g], ct[g]));
    }
#pragma unroll
    for (int g = 0; g < G; g++) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx[g] = fmaxf(mx[g], __shfl_xor_sync(0xffffffffu, mx[g], o));
    }
    if (lane == 0) {
      float sum = 0.f;
      if (te > tb) {
#pragma unroll
        for (int g = 0; g < G; g++)
          if (g < ng) sum += mx[g];
      }
      part[((int64_t)q * ngroups + grp) * kd + slot] = sum;
    }
  }
}

template <int M>
static tachiom_status launch_refine_m(const Index &ix, const float *queries, const int32_t *meta, int nq,
                                      const int32_t *cand, int kd, float *part, uint32_t *flags,
                                      cudaStream_t s, bool centroid_only) {
  const uint16_t *rn = centroid_only ? nullptr : ix.rnorm;
  constexpr int G = 128 / M;
  const int ngroups = refine_groups(M);
  size_t smem = ((size_t)M * 256 * G + (size_t)G * DIM) * 4;
  dim3 grid((kd + R_DOCS_PER_CTA - 1) / R_DOCS_PER_CTA, ngroups, nq);
  if (ix.cdtype == TACHIOM_DTYPE_BF16) {
    TCUDA(cudaFuncSetAttribute(k_refine<M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_refine<M, true><<<grid, R_THREADS, smem, s>>>(queries, meta, nq, cand, kd, ix.doc_off, ix.tok_cid,
                                                     ix.codes, rn, ix.codebooks, ix.cent_f32,
                                                     ix.cent_bf16, part, ngroups, ix.D, flags);
  } else {
    TCUDA(cudaFuncSetAttribute(k_refine<M, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_refine<M, false><<<grid, R_THREADS, smem, s>>>(queries, meta, nq, cand, kd, ix.doc_off, ix.tok_cid,
                                                      ix.codes, rn, ix.codebooks, ix.cent_f32,
                                                      ix.cent_bf16, part, ngroups, ix.D, flags);
  }
  TLAUNCH();
  return TACHIOM_OK;
}

tachiom_status launch_refine(const Index &ix, const float *queries, const int32_t *meta, int nq,
                             const int32_t *cand, int kd, float *part, uint32_t *flags, cudaStream_t s,
                             bool centroid_only) {
  if (nq <= 0) return TACHIOM_OK;
  TPROF(centroid_only ? "centroid_interaction" : "refine", s);
  switch (ix.M) {
    case 8: return launch_refine_m<8>(ix, queries, meta, nq, cand, kd, part, flags, s, centroid_only);
    case 16: return launch_refine_m<16>(ix, queries, meta, nq, cand, kd, part, flags, s, centroid_only);
    case 32: return launch_refine_m<32>(ix, queries, meta, nq, cand, kd, part, flags, s, centroid_only);
  }
  return fail(TACHIOM_ERR_INVALID, "unsupported pq_m %d", ix.M);
}

// ---------------------------------------------------------------------------------
// The FP32 refine for a short list of documents (the window the reduced-precision
// pass leaves), one CTA per (query, document). A document is taken in chunks of
// 64 tokens: the chunk's centroid ids, codes and norms are loaded at once, then
// its centroid rows and the codewords its codes select are copied to shared
// memory with cp.async (one wave of copies per chunk, the next chunk's issued
// before the current one is computed: two buffers). Lane i holds query token
// i in registers; a warp takes 4 document tokens at a time (4 independent FMA
// chains) and reads their rows and codewords from shared memory (broadcast).
// Every number is the one k_refine produces: the centroid term is the same fmaf
// chain over k = 0..127, each table entry T[m][code][i] is the same fmaf chain
// over the subspace's dims (computed here instead of looked up), rs adds them in
// ascending m from 0, fmaf(rho, rs, ct) is maxed over the tokens, and the group
// partial sums are formed in the same order. So the scores are bit-identical to
// k_refine's and k_final_topk ranks them as before. The list is compacted: the
// first id < 0 ends it.
constexpr int RW_WARPS = 8;
constexpr int RW_THREADS = RW_WARPS * 32;
constexpr int RW_CTAS = 16;      // CTAs per query, each taking documents blockIdx.x, +16, ...
constexpr int RW_CHUNK = 64;     // document tokens staged at once
constexpr int RW_TPW = 4;        // document tokens per warp step

template <bool BF16C>
constexpr size_t rw_buf_bytes() {
  return (size_t)RW_CHUNK * DIM * (BF16C ? 2 : 4)        // centroid rows
         + (size_t)RW_CHUNK * DIM * 4                      // the chunk's codewords (M x DS = 128 floats per token)
         + (size_t)RW_CHUNK * (4 + 4 + 32);                // centroid id, rho, codes (<= 32 bytes)
}
template <bool BF16C>
constexpr size_t rw_smem() {
  return 2 * rw_buf_bytes<BF16C>() + (size_t)RW_WARPS * MAX_NTOK * 4;  // two chunk buffers, per-warp maxima
}

__device__ __forceinline__ void rw_cp16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}

template <int M, bool BF16C>
__global__ void __launch_bounds__(RW_THREADS, 1)
k_refine_win(const float *__restrict__ queries, const int32_t *__restrict__ meta, int nq,
             const int32_t *__restrict__ cand, int kd, const int64_t *__restrict__ doc_off,
             const int32_t *__restrict__ tok_cid, const uint8_t *__restrict__ codes,
             const uint16_t *__restrict__ rnorm, const float *__restrict__ codebooks,
             const float *__restrict__ cent_f32, const __nv_bfloat16 *__restrict__ cent_bf16,
             const int32_t *__restrict__ only, float *__restrict__ part, int ngroups, int64_t D,
             uint32_t *__restrict__ flags) {
  constexpr int G = 128 / M;
  constexpr int DS = 128 / M;
  constexpr int RB = BF16C ? DIM * 2 : DIM * 4;  // bytes per centroid row
  constexpr size_t BUF = rw_buf_bytes<BF16C>();
  extern __shared__ __align__(16) unsigned char rwm[];
  // buffer b: rows [CHUNK][RB], codewords [CHUNK][128], centroid ids, rho, codes [CHUNK][32]
  auto rows_of = [&](int b) { return rwm + b * BUF; };
  auto cw_of = [&](int b) { return reinterpret_cast<float *>(rwm + b * BUF + RW_CHUNK * RB); };
  auto cid_of = [&](int b) { return reinterpret_cast<int32_t *>(cw_of(b) + RW_CHUNK * DIM); };
  auto rh_of = [&](int b) { return reinterpret_cast<float *>(cid_of(b) + RW_CHUNK); };
  auto cds_of = [&](int b) { return reinterpret_cast<uint8_t *>(rh_of(b) + RW_CHUNK); };
  float *mxs = reinterpret_cast<float *>(rwm + 2 * BUF);  // [WARPS][32]
  const int q = blockIdx.y;
  const int ntok = meta[3 * nq + 2 + q];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (only) {
    // nothing listed among this CTA's slots (the usual case): leave before any other load
    int any = 0;
    for (int slot = blockIdx.x + tid * gridDim.x; slot < kd && !any; slot += blockDim.x * gridDim.x) {
      if (cand[(int64_t)q * kd + slot] < 0) break;
      any = only[(int64_t)q * kd + slot];
    }
    if (!__syncthreads_or(any)) return;
  }
  // this lane's query token, in registers
  float qv[DIM];
  {
    const float4 *qr = reinterpret_cast<const float4 *>(queries + ((int64_t)meta[q] + min(lane, max(ntok - 1, 0))) * DIM);
#pragma unroll
    for (int k4 = 0; k4 < DIM / 4; k4++) {
      const float4 v = qr[k4];
      qv[4 * k4] = v.x; qv[4 * k4 + 1] = v.y; qv[4 * k4 + 2] = v.z; qv[4 * k4 + 3] = v.w;
    }
  }
  // chunk staging: the ids, norms and codes (plain loads), then, after a barrier, the copies
  // of the rows and of the selected codewords (cp.async, one commit group per chunk)
  auto stage_meta = [&](int b, int64_t c0, int nt) {
    int32_t *cid = cid_of(b);
    float *rh = rh_of(b);
    uint8_t *cds = cds_of(b);
    for (int x = tid; x < nt; x += RW_THREADS) {
      cid[x] = tok_cid[c0 + x];
      rh[x] = __half2float(__ushort_as_half(rnorm[c0 + x]));
    }
    for (int x = tid; x < nt * M; x += RW_THREADS) cds[(x / M) * 32 + x % M] = codes[c0 * M + x];
  };
  auto stage_copy = [&](int b, int nt) {
    constexpr int RC = RB / 16, WC = DS * 4 / 16;
    unsigned char *rows = rows_of(b);
    float *cw = cw_of(b);
    const int32_t *cid = cid_of(b);
    const uint8_t *cds = cds_of(b);
    for (int x = tid; x < nt * RC; x += RW_THREADS) {
      const int t = x / RC, c = x % RC;
      const unsigned char *src = BF16C ? reinterpret_cast<const unsigned char *>(cent_bf16 + (int64_t)cid[t] * DIM)
                                       : reinterpret_cast<const unsigned char *>(cent_f32 + (int64_t)cid[t] * DIM);
      rw_cp16(rows + t * RB + c * 16, src + c * 16);
    }
    for (int x = tid; x < nt * M * WC; x += RW_THREADS) {
      const int t = x / (M * WC), r = x % (M * WC), m = r / WC, c = r % WC;
      rw_cp16(cw + t * DIM + m * DS + c * 4, codebooks + ((int64_t)m * 256 + cds[t * 32 + m]) * DS + c * 4);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  const int gq = (ntok + G - 1) / G;
  for (int slot = blockIdx.x; slot < kd; slot += gridDim.x) {
    const int32_t d = cand[(int64_t)q * kd + slot];
    if (d < 0) break;
    if (only && !only[(int64_t)q * kd + slot]) continue;  // only the listed documents
    if (d >= D) {
      if (tid == 0) atomicOr(flags, TACHIOM_FLAG_BAD_INPUT);
      if (tid < gq) part[((int64_t)q * ngroups + tid) * kd + slot] = 0.f;
      continue;
    }
    __syncthreads();  // the previous document's maxima have been summed, its buffers are free
    const int64_t tb = doc_off[d], te = doc_off[d + 1];
    const int nch = (int)((te - tb + RW_CHUNK - 1) / RW_CHUNK);
    float mx = -INFINITY;
    if (nch > 0) {
      stage_meta(0, tb, (int)min((int64_t)RW_CHUNK, te - tb));
      __syncthreads();
      stage_copy(0, (int)min((int64_t)RW_CHUNK, te - tb));
    }
    for (int ch = 0; ch < nch; ch++) {
      const int b = ch & 1;
      const int64_t c0 = tb + (int64_t)ch * RW_CHUNK;
      const int nt = (int)min((int64_t)RW_CHUNK, te - c0);
      if (ch + 1 < nch) {
        // the next chunk goes to the other buffer while this one is computed
        const int64_t c1 = c0 + RW_CHUNK;
        const int nt1 = (int)min((int64_t)RW_CHUNK, te - c1);
        stage_meta(b ^ 1, c1, nt1);
        __syncthreads();
        stage_copy(b ^ 1, nt1);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
      } else {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
      }
      __syncthreads();  // this chunk's copies are visible to every thread
      const unsigned char *rows = rows_of(b);
      const float *cw = cw_of(b);
      const float *rh = rh_of(b);
      for (int t0 = warp * RW_TPW; t0 < nt; t0 += RW_WARPS * RW_TPW) {
        int tt[RW_TPW];
#pragma unroll
        for (int j = 0; j < RW_TPW; j++) tt[j] = min(t0 + j, nt - 1);  // a missing token repeats the last one
        float ct[RW_TPW], rs[RW_TPW];
#pragma unroll
        for (int j = 0; j < RW_TPW; j++) ct[j] = rs[j] = 0.f;
        if (BF16C) {
#pragma unroll
          for (int k8 = 0; k8 < DIM / 8; k8++) {
#pragma unroll
            for (int j = 0; j < RW_TPW; j++) {
              const uint4 u = reinterpret_cast<const uint4 *>(rows + tt[j] * RB)[k8];
              const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
              for (int h = 0; h < 4; h++) {
                ct[j] = fmaf(qv[k8 * 8 + 2 * h], __uint_as_float(w[h] << 16), ct[j]);
                ct[j] = fmaf(qv[k8 * 8 + 2 * h + 1], __uint_as_float(w[h] & 0xffff0000u), ct[j]);
              }
            }
          }
        } else {
#pragma unroll
          for (int k4 = 0; k4 < DIM / 4; k4++) {
#pragma unroll
            for (int j = 0; j < RW_TPW; j++) {
              const float4 c = reinterpret_cast<const float4 *>(rows + tt[j] * RB)[k4];
              ct[j] = fmaf(qv[k4 * 4 + 0], c.x, ct[j]);
              ct[j] = fmaf(qv[k4 * 4 + 1], c.y, ct[j]);
              ct[j] = fmaf(qv[k4 * 4 + 2], c.z, ct[j]);
              ct[j] = fmaf(qv[k4 * 4 + 3], c.w, ct[j]);
            }
          }
        }
#pragma unroll
        for (int m = 0; m < M; m++) {
#pragma unroll
          for (int j = 0; j < RW_TPW; j++) {
            const float *wt = cw + tt[j] * DIM + m * DS;
            float a = 0.f;
#pragma unroll
            for (int u = 0; u < DS; u++) a = fmaf(qv[m * DS + u], wt[u], a);
            rs[j] += a;
          }
        }
#pragma unroll
        for (int j = 0; j < RW_TPW; j++) mx = fmaxf(mx, fmaf(rh[tt[j]], rs[j], ct[j]));
      }
      __syncthreads();  // buffer b is free for chunk ch + 2
    }
    mxs[warp * MAX_NTOK + lane] = mx;
    __syncthreads();
    if (tid < gq) {
      const int grp = tid, i0 = grp * G, ng = min(G, ntok - i0);
      float sum = 0.f;
      if (te > tb) {
        for (int g = 0; g < ng; g++) {
          float v = mxs[i0 + g];
#pragma unroll
          for (int w = 1; w < RW_WARPS; w++) v = fmaxf(v, mxs[w * MAX_NTOK + i0 + g]);
          sum += v;
        }
      }
      part[((int64_t)q * ngroups + grp) * kd + slot] = sum;
    }
  }
}

template <int M>
static tachiom_status launch_refine_win_m(const Index &ix, const float *queries, const int32_t *meta, int nq,
                                          const int32_t *cand, int kd, const int32_t *only, float *part,
                                          uint32_t *flags, cudaStream_t s) {
  dim3 grid(std::min(RW_CTAS, kd), nq);
  if (ix.cdtype == TACHIOM_DTYPE_BF16) {
    TCUDA(cudaFuncSetAttribute(k_refine_win<M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)rw_smem<true>()));
    k_refine_win<M, true><<<grid, RW_THREADS, rw_smem<true>(), s>>>(
        queries, meta, nq, cand, kd, ix.doc_off, ix.tok_cid, ix.codes, ix.rnorm, ix.codebooks, ix.cent_f32,
        ix.cent_bf16, only, part, refine_groups(M), ix.D, flags);
  } else {
    TCUDA(cudaFuncSetAttribute(k_refine_win<M, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)rw_smem<false>()));
    k_refine_win<M, false><<<grid, RW_THREADS, rw_smem<false>(), s>>>(
        queries, meta, nq, cand, kd, ix.doc_off, ix.tok_cid, ix.codes, ix.rnorm, ix.codebooks, ix.cent_f32,
        ix.cent_bf16, only, part, refine_groups(M), ix.D, flags);
  }
  TLAUNCH();
  return TACHIOM_OK;
}

tachiom_status launch_refine_win(const Index &ix, const float *queries, const int32_t *meta, int nq,
                                 const int32_t *cand, int kd, float *part, uint32_t *flags, cudaStream_t s) {
  return launch_refine_win_only(ix, queries, meta, nq, cand, kd, nullptr, part, flags, s);
}

tachiom_status launch_refine_win_only(const Index &ix, const float *queries, const int32_t *meta, int nq,
                                      const int32_t *cand, int kd, const int32_t *only, float *part,
                                      uint32_t *flags, cudaStream_t s) {
  if (nq <= 0) return TACHIOM_OK;
  TPROF(only ? "refine_win_fp32" : "refine_win", s);
  switch (ix.M) {
    case 8: return launch_refine_win_m<8>(ix, queries, meta, nq, cand, kd, only, part, flags, s);
    case 16: return launch_refine_win_m<16>(ix, queries, meta, nq, cand, kd, only, part, flags, s);
    case 32: return launch_refine_win_m<32>(ix, queries, meta, nq, cand, kd, only, part, flags, s);
  }
  return fail(TACHIOM_ERR_INVALID, "unsupported pq_m %d", ix.M);
}

// ---------------------------------------------------------------------------------
// step (d): S = sum of the group partials (ascending group), then the first k by
// (S desc, doc asc); rows padded with (-1, -inf)
__global__ void __launch_bounds__(1024)
k_final_topk(const int32_t *__restrict__ meta, int nq, const int32_t *__restrict__ cand, int kd,
             const float *__restrict__ part, int ngroups, int G, int32_t *__restrict__ out_ids,
             float *__restrict__ out_s) {
  extern __shared__ __align__(16) uint64_t fsm[];
  const int q = blockIdx.x;
  const int ntok = meta[3 * nq + 2 + q];
  const int k = meta[2 * nq + 2 + q];
  const int koff = meta[nq + 1 + q];
  const int gq = (ntok + G - 1) / G;
  const int np = next_pow2(max(kd, 2));
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    uint64_t v = 0ull;
    if (i < kd) {
      int32_t d = cand[(int64_t)q * kd + i];
      if (d >= 0) {
        float s = 0.f;
        for (int g = 0; g < gq; g++) s += part[((int64_t)q * ngroups + g) * kd + i];
        v = comp_key(s, d);
      }
    }
    fsm[i] = v;
  }
  __syncthreads();
  block_sort_desc(fsm, np);
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    uint64_t v = i < np ? fsm[i] : 0ull;
    out_ids[koff + i] = v ? comp_id(v) : -1;
    out_s[koff + i] = v ? comp_score(v) : -INFINITY;
  }
}

tachiom_status launch_final_topk(const Index &ix, const int32_t *meta, int nq, const int32_t *cand, int kd,
                                 const float *part, int32_t *out_ids, float *out_s, cudaStream_t s) {
  if (nq <= 0) return TACHIOM_OK;
  TPROF("final_topk", s);
  size_t smem = (size_t)next_pow2(std::max(kd, 2)) * 8;
  TCUDA(cudaFuncSetAttribute(k_final_topk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_final_topk<<<nq, 1024, smem, s>>>(meta, nq, cand, kd, part, refine_groups(ix.M), 128 / ix.M, out_ids,
                                      out_s);
  TLAUNCH();
  return TACHIOM_OK;
}

}  // namespace tachiom
