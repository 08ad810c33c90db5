// Step (c), reduced-precision pass: decode, then tensor cores.
//
// S(q,d) = sum_i max_{t in d} <q_i, x_t>,  x_t = c_a(t) + rho_t r^_t
//
// is the same number as the ADC form of Sec. 2.2 (Refine): the lookup
// sum_m T[m][code_{t,m}][i] is <q_i, r^_t> split by subspace. On the B300 the
// dense form is cheaper: a warp rebuilds x_t for 16 document tokens (the bf16
// centroid row, gathered with cp.async one chunk ahead, plus rho_t times the
// token's codewords, read from an fp16 copy of the codebooks in shared memory
// with 16-byte code loads), rounds it to fp16, and one mma.sync chain
// (m16n8k16, 16 tokens x 8 query tokens per n-tile, all 32 query tokens of the
// query) scores the tile. The CTA keeps every query token, so codes and rows
// are read once per query. fp16 rather than bf16 operands: the same tensor
// rate, a unit roundoff of 2^-11 instead of 2^-8, so the bound below, and with
// it the window the FP32 kernel has to rescore, is about 8x narrower. The
// values here (unit-scale embeddings) are far inside the fp16 range; a value
// that overflows it gives an infinite bound, which sends the document to the
// FP32 kernel.
//
// The result is approximate; it only chooses the documents the FP32 kernel
// (k_refine, lookup tables) rescores. Rigorous bound, per document d:
//   |<h(q_i), h(x_t)> - <q_i, x_t>| <= ||e_qi|| ||x_t|| + ||h(q_i)|| ||e_xt||
//                                     + 2^-17 ||h(q_i)|| ||h(x_t)||
// with h() the rounding to fp16, e_q = h(q) - q, e_x = h(x~) - x (x~ built from the fp16 codewords;
// the codeword rounding enters e_x through a per-codeword error table). Taking
// the max over t and summing over i gives Delta_d >= |S_approx(d) - S(d)|.
// The documents are then compared with the FP32 kernel's scores, whose own
// rounding (a chain of at most 150 FP32 operations per query token, over the
// terms of <q, c> and rho <q, w>, with ||c|| <= cnorm and ||rho w|| <= ||x|| +
// cnorm) is below 2^-16 ||q_i|| (||x_t|| + 2 cnorm) per query token; Delta_d
// carries that term too.
#include <cuda_fp16.h>

#include "tachiom_internal.cuh"

namespace tachiom {

constexpr int RD_DOCS_PER_CTA = 64;
constexpr int RD_ROW = 272;              // query tile row: 128 2-byte values + 16 bytes padding (conflict-free ldmatrix)
constexpr int RD_SMEM_MAX = 227 * 1024;

// Document tiles (16 rows of 128 fp16 values). With codewords of 8 or more dims (M = 8, 16) the
// rows are unpadded and XOR-swizzled: 16-byte chunk c of row r sits at chunk c ^ (r & 7). The
// codebook is then code-major ([256][M][ds]), so the piece of a codeword that covers chunk c lies
// in 16-byte bank group c & 7 whatever the code; lane j of a decode phase takes its chunks in the
// order (alpha j) ^ v, v = 0..7 (alpha j: j times x in GF(8), x^3 = x + 1), so in every step the 8
// lanes of a phase read 8 different codeword bank groups and - as (alpha + 1) j ^ v is also a
// permutation of j - 8 different row bank groups. With 4-dim codewords (M = 32) the rows keep the
// query tile's padding and the codebook stays subspace-major ([M][256][ds]).
template <int M>
constexpr bool rd_swz() { return 128 / M >= 8; }
template <int M>
constexpr int rd_pitch() { return rd_swz<M>() ? 256 : RD_ROW; }
template <int M>
constexpr int rd_tile() { return 16 * rd_pitch<M>(); }
__host__ __device__ constexpr int rd_gf8_mulx(int j) { return ((j << 1) & 7) ^ ((j & 4) ? 3 : 0); }

// shared memory: fp16 codebooks, codeword error table, query norms, the fp16
// query tile [32][RD_ROW], then per warp two tiles (centroid rows land by
// cp.async and are decoded in place)
template <int M>
constexpr int rd_fixed_bytes() {
  return M * 256 * (128 / M) * 2 + M * 256 * 4 + 64 * 4 + 32 * RD_ROW;
}
// per warp: two tiles, and in the window variant the chunk's row norms and the exact maxima
template <int M, bool WIN>
constexpr int rd_warp_bytes() { return 2 * rd_tile<M>() + (WIN ? 256 : 0); }
template <int M, bool WIN>
constexpr int rd_warps() {
  return (RD_SMEM_MAX - rd_fixed_bytes<M>()) / rd_warp_bytes<M, WIN>() > 16
             ? 16
             : (RD_SMEM_MAX - rd_fixed_bytes<M>()) / rd_warp_bytes<M, WIN>();
}

__device__ __forceinline__ void rd_mma(float *d, const uint32_t *a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void rd_ldm4(uint32_t *r, uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr)
               : "memory");
}

struct DecPos {
  int slot;
  int64_t tb, te, c0;
  float2 xe;  // main pass: the document's norm maxima (k_doc_decode_norms), loaded with its bounds
};

// next 16-token chunk of the warp's document, or the next document of the CTA's
// slice (taken from a shared counter, so the warps stay balanced)
// bad(slot, empty): answer a slot whose document is out of range (empty = false) or has no
// tokens (empty = true); called by lane 0. doc_xe: null in the window variant.
template <typename BadFn>
__device__ __forceinline__ bool dec_next(DecPos &p, int s_end, int stride, int off, int *s_next,
                                         const int32_t *cand_q, const int64_t *doc_off, const float2 *doc_xe,
                                         int64_t D, BadFn bad, uint32_t *flags, int lane) {
  if (p.c0 + 16 < p.te) {
    p.c0 += 16;
    return true;
  }
  for (;;) {
    int slot = 0;
    if (lane == 0) slot = atomicAdd(s_next, 1);
    slot = __shfl_sync(0xffffffffu, slot, 0) * stride + off;  // the CTA's share of the slots
    if (slot >= s_end) return false;
    p.slot = slot;
    const int32_t d = cand_q[slot];
    if (d < 0) continue;
    if (d >= D) {
      if (lane == 0) {
        atomicOr(flags, TACHIOM_FLAG_BAD_INPUT);
        bad(slot, false);
      }
      continue;
    }
    p.tb = doc_off[d];
    p.te = doc_off[d + 1];
    if (doc_xe) p.xe = doc_xe[d];
    if (p.te == p.tb) {
      if (lane == 0) bad(slot, true);
      continue;
    }
    p.c0 = p.tb;
    return true;
  }
}

// The FP32 path's score of query token i against document token t: the fmaf chain over
// k = 0..127 of the centroid term, the table entries of the residual (each an fmaf chain over
// its subspace's dims) added in ascending m from 0, then fmaf(rho, rs, ct) - k_refine's numbers.
template <int M>
__device__ __forceinline__ float dec_exact(const float *__restrict__ qi, int64_t t,
                                           const int32_t *__restrict__ tok_cid, const uint8_t *__restrict__ codes,
                                           const uint16_t *__restrict__ rnorm, const float *__restrict__ codebooks,
                                           const float *__restrict__ cent_f32,
                                           const __nv_bfloat16 *__restrict__ cent_bf16, bool bf16c) {
  constexpr int DS = 128 / M;
  // first the token's centroid id, codes and norm, then every row and codeword load at once
  const int32_t j = tok_cid[t];
  uint8_t c8[M];
#pragma unroll
  for (int u = 0; u < M / 8; u++)
    *reinterpret_cast<uint2 *>(c8 + 8 * u) = *reinterpret_cast<const uint2 *>(codes + t * M + 8 * u);
  const float rho = __half2float(__ushort_as_half(rnorm[t]));
  const float4 *q4 = reinterpret_cast<const float4 *>(qi);
  float ct = 0.f;
  if (bf16c) {
    const uint4 *crow = reinterpret_cast<const uint4 *>(cent_bf16 + (int64_t)j * DIM);
    uint4 cr[DIM / 8];
#pragma unroll
    for (int k8 = 0; k8 < DIM / 8; k8++) cr[k8] = crow[k8];
#pragma unroll
    for (int k8 = 0; k8 < DIM / 8; k8++) {
      const uint4 u = cr[k8];
      const float4 qa = q4[2 * k8], qb = q4[2 * k8 + 1];
      ct = fmaf(qa.x, __uint_as_float(u.x << 16), ct);
      ct = fmaf(qa.y, __uint_as_float(u.x & 0xffff0000u), ct);
      ct = fmaf(qa.z, __uint_as_float(u.y << 16), ct);
      ct = fmaf(qa.w, __uint_as_float(u.y & 0xffff0000u), ct);
      ct = fmaf(qb.x, __uint_as_float(u.z << 16), ct);
      ct = fmaf(qb.y, __uint_as_float(u.z & 0xffff0000u), ct);
      ct = fmaf(qb.z, __uint_as_float(u.w << 16), ct);
      ct = fmaf(qb.w, __uint_as_float(u.w & 0xffff0000u), ct);
    }
  } else {
    const float4 *crow = reinterpret_cast<const float4 *>(cent_f32 + (int64_t)j * DIM);
#pragma unroll
    for (int hh = 0; hh < 2; hh++) {
      float4 cr[DIM / 8];
#pragma unroll
      for (int k4 = 0; k4 < DIM / 8; k4++) cr[k4] = crow[hh * (DIM / 8) + k4];
#pragma unroll
      for (int k4 = 0; k4 < DIM / 8; k4++) {
        const float4 c = cr[k4], qa = q4[hh * (DIM / 8) + k4];
        ct = fmaf(qa.x, c.x, ct);
        ct = fmaf(qa.y, c.y, ct);
        ct = fmaf(qa.z, c.z, ct);
        ct = fmaf(qa.w, c.w, ct);
      }
    }
  }
  // the residual: the subspaces' codewords in two batches of 64 floats
  float rs = 0.f;
#pragma unroll
  for (int hh = 0; hh < 2; hh++) {
    float w[DIM / 2];
#pragma unroll
    for (int mm = 0; mm < M / 2; mm++) {
      const int m = hh * (M / 2) + mm;
      const float4 *src = reinterpret_cast<const float4 *>(codebooks + ((int64_t)m * 256 + c8[m]) * DS);
#pragma unroll
      for (int u4 = 0; u4 < DS / 4; u4++) {
        const float4 v = src[u4];
        w[mm * DS + 4 * u4] = v.x; w[mm * DS + 4 * u4 + 1] = v.y;
        w[mm * DS + 4 * u4 + 2] = v.z; w[mm * DS + 4 * u4 + 3] = v.w;
      }
    }
#pragma unroll
    for (int mm = 0; mm < M / 2; mm++) {
      const int m = hh * (M / 2) + mm;
      float a = 0.f;
#pragma unroll
      for (int u = 0; u < DS; u++) a = fmaf(qi[m * DS + u], w[mm * DS + u], a);
      rs += a;
    }
  }
  return fmaf(rho, rs, ct);
}

// !WIN: sa[q][slot] = approximate S, da[q][slot] = its bound Delta_d, and per query token i
//       thr[q][slot][i] = (approximate max_t v_it) - (the bound of its error); a token t whose
//       approximate v_it plus its own bound is below thr cannot hold the exact maximum.
// WIN:  the same pass over the compacted window list cand (first id < 0 ends it): the pairs
//       (i, t) that pass the test against thr are appended to the list wl ({q * kd + slot,
//       (t - first token) << 5 | i}) for k_dec_exact_pairs; emx[q][slot][i] (the exact maxima
//       that kernel forms) starts at -inf; a document whose pairs do not fit the list is
//       marked in wovf[q][slot] for the all-pairs FP32 kernel.
template <int M, int WARPS, bool WIN>
__global__ void __launch_bounds__(WARPS * 32, 1)
k_refine_dec(const float *__restrict__ queries, const int32_t *__restrict__ meta, int nq,
             const int32_t *__restrict__ cand, int kd, const int64_t *__restrict__ doc_off,
             const int32_t *__restrict__ tok_cid, const uint8_t *__restrict__ codes,
             const uint16_t *__restrict__ rnorm, const __half *__restrict__ cbk_h16,
             const float *__restrict__ cbk_err2, const __nv_bfloat16 *__restrict__ cent_bf16,
             const float *__restrict__ cent_f32, int bf16c, const float2 *__restrict__ doc_xe, float cerr, float cnorm, float *__restrict__ sa, float *__restrict__ da, float *__restrict__ thr,
             const int32_t *__restrict__ win_slot, float *__restrict__ part, int ngroups, int2 *__restrict__ wl,
             unsigned long long *__restrict__ wl_n, int wl_cap, uint32_t *__restrict__ emx, int32_t *__restrict__ wovf, int64_t D,
             uint32_t *__restrict__ flags) {
  constexpr int DS = 128 / M;
  constexpr int NT = WARPS * 32;
  constexpr bool SWZ = rd_swz<M>();
  constexpr int PITCH = rd_pitch<M>(), TILE = rd_tile<M>();
  extern __shared__ __align__(16) unsigned char dsm[];
  __half *cbk = reinterpret_cast<__half *>(dsm);                           // fp16 codewords (layout above)
  float *cerr2 = reinterpret_cast<float *>(dsm + M * 256 * DS * 2);        // [M][256] ||h(w) - w||^2
  float *qn = cerr2 + M * 256;                                             // [32] ||e_q||, [32] ||h(q)||
  unsigned char *qsm = reinterpret_cast<unsigned char *>(qn + 64);         // [32][RD_ROW] fp16 query tokens
  unsigned char *tiles = qsm + 32 * RD_ROW;                                // [WARPS][2 tiles]
  __shared__ int s_next;

  const int q = blockIdx.y;
  const int ntok = meta[3 * nq + 2 + q];
  const int32_t *cand_q = cand + (int64_t)q * kd;
  int s_begin, s_end;
  if (WIN) {
    // the window list is compacted: its length is the number of ids >= 0
    __shared__ int s_nv;
    if (threadIdx.x == 0) s_nv = 0;
    __syncthreads();
    int nv = 0;
    for (int i = threadIdx.x; i < kd; i += NT) nv += cand_q[i] >= 0 ? 1 : 0;
    nv = __reduce_add_sync(0xffffffffu, nv);
    if ((threadIdx.x & 31) == 0 && nv) atomicAdd(&s_nv, nv);
    __syncthreads();
    s_begin = 0;
    s_end = s_nv;
  } else {
    s_begin = blockIdx.x * RD_DOCS_PER_CTA;
    s_end = min(kd, s_begin + RD_DOCS_PER_CTA);
  }
  {
    int any = 0;
    for (int i = s_begin + (int)threadIdx.x; i < s_end && !any; i += NT) any = cand_q[i] >= 0;
    if (!__syncthreads_or(any)) return;
  }
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gq = lane >> 2;
  // the fp16 codebooks (formed at index load in this kernel's layout) and, for the window
  // variant, the squared rounding error of each codeword
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(cbk_h16);
    uint4 *dst = reinterpret_cast<uint4 *>(cbk);
#pragma unroll 8
    for (int x = tid; x < 128 * 256 * 2 / 16; x += NT) dst[x] = src[x];
    if constexpr (WIN) {
      for (int x = tid; x < M * 256; x += NT) cerr2[x] = cbk_err2[x];
    }
  }
  // query tokens: the fp16 tile (B operand, zero rows past ntok) and the norms of the rounding error
  const float *qrow = queries + (int64_t)meta[q] * DIM;
  for (int x = tid; x < 32 * DIM / 2; x += NT) {
    const int i = x / (DIM / 2), k = (x % (DIM / 2)) * 2;
    const float x0 = i < ntok ? qrow[(int64_t)i * DIM + k] : 0.f;
    const float x1 = i < ntok ? qrow[(int64_t)i * DIM + k + 1] : 0.f;
    *reinterpret_cast<__half2 *>(qsm + i * RD_ROW + k * 2) = __floats2half2_rn(x0, x1);
  }
  for (int i = warp; i < 32; i += WARPS) {
    float e2 = 0.f, h2 = 0.f;
    if (i < ntok) {
      for (int k = lane; k < DIM; k += 32) {
        const float x = qrow[(int64_t)i * DIM + k];
        const float h = __half2float(__float2half_rn(x));
        e2 = fmaf(h - x, h - x, e2);
        h2 = fmaf(h, h, h2);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e2 += __shfl_xor_sync(0xffffffffu, e2, o);
      h2 += __shfl_xor_sync(0xffffffffu, h2, o);
    }
    if (lane == 0) {
      qn[i] = sqrtf(e2) * (1.f + ldexpf(1.f, -10));
      qn[32 + i] = sqrtf(h2) * (1.f + ldexpf(1.f, -10));
    }
  }
  // the window variant's CTAs of a query take every gridDim.x-th slot
  const int stride = WIN ? (int)gridDim.x : 1, off = WIN ? (int)blockIdx.x : 0;
  if (tid == 0) s_next = WIN ? 0 : s_begin;
  __syncthreads();

  unsigned char *wt = tiles + warp * 2 * TILE;
  // window variant: this warp's chunk row norms (xn, en per row)
  float *rnx = reinterpret_cast<float *>(tiles + WARPS * 2 * TILE + warp * 256);  // [16][2]
  const int G = 128 / M;                   // query tokens per group of the FP32 path's partial sums
  const int gq_n = (ntok + G - 1) / G;     // groups of this query
  const uint32_t wt_s = (uint32_t)__cvta_generic_to_shared(wt);
  const uint32_t qs_s = (uint32_t)__cvta_generic_to_shared(qsm);
  // ldmatrix row addresses: A (document tokens x dims) and B (query tokens x dims, two n-tiles per x4)
  // (swizzled tiles: row ((lane >> 3) & 1) * 8 + (lane & 7), logical chunk 2 s + (lane >> 4) of k-step s)
  const uint32_t la_off = SWZ ? (uint32_t)((((lane >> 3) & 1) * 8 + (lane & 7)) * PITCH)
                              : (uint32_t)((((lane >> 3) & 1) * 8 + (lane & 7)) * PITCH + ((lane >> 4) * 8) * 2);
  const uint32_t lb_off = (uint32_t)((((lane >> 4) * 8) + (lane & 7)) * RD_ROW + ((lane >> 3) & 1) * 16);
  float *sa_row = WIN ? nullptr : sa + (int64_t)q * kd;
  float *da_row = WIN ? nullptr : da + (int64_t)q * kd;
  // a slot whose document is out of range or empty: S = -inf (flagged) or 0, bound 0
  auto bad = [&](int slot, bool empty) {
    if (WIN) {
      for (int g = 0; g < gq_n; g++) part[((int64_t)q * ngroups + g) * kd + slot] = 0.f;
    } else {
      sa_row[slot] = empty ? 0.f : -INFINITY;
      da_row[slot] = 0.f;
    }
  };
  // decode layout: lane -> row lane & 15, dims (lane >> 4) * 64 .. +64 (the 8 lanes of a
  // 16-byte shared-memory phase then read 8 different rows: no bank conflicts)
  const int drow = lane & 15, dhalf = lane >> 4;
  const int j7 = drow & 7, ja = rd_gf8_mulx(j7);  // swizzled tiles: the lane's chunk order is ja ^ v

  // a chunk's centroid ids: lane l holds row l & 15 (a row past the document repeats its last
  // token, masked later); loaded a chunk ahead of the copies that use it
  auto load_cid = [&](const DecPos &p) -> int32_t { return tok_cid[min(p.c0 + (lane & 15), p.te - 1)]; };
  // copies of the chunk's 16 centroid rows into stage b, and this lane's codes and norm
  auto issue_rows = [&](const DecPos &p, int32_t cid_l, int b, uint4 &cw, float &rh) {
    const uint32_t dst0 = wt_s + (uint32_t)(b * TILE);
#pragma unroll
    for (int it = 0; it < 8; it++) {
      const int qq = it * 32 + lane;
      const int row = qq >> 4, pc = qq & 15;
      const int32_t cr = __shfl_sync(0xffffffffu, cid_l, row);
      const int pcs = SWZ ? (pc ^ (row & 7)) : pc;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst0 + (uint32_t)(row * PITCH + pcs * 16)),
                   "l"(cent_bf16 + (int64_t)cr * DIM + pc * 8)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    // this lane decodes row drow, half dhalf: codes of its subspaces, and the norm
    const int64_t t = min(p.c0 + drow, p.te - 1);
    if constexpr (M == 32) {
      cw = *reinterpret_cast<const uint4 *>(codes + t * M + dhalf * 16);
    } else if constexpr (M == 16) {
      const uint2 v = *reinterpret_cast<const uint2 *>(codes + t * M + dhalf * 8);
      cw = make_uint4(v.x, v.y, 0u, 0u);
    } else {
      const uint32_t v = *reinterpret_cast<const uint32_t *>(codes + t * M + dhalf * 4);
      cw = make_uint4(v, 0u, 0u, 0u);
    }
    rh = __half2float(__ushort_as_half(rnorm[t]));
  };

  // chunk pipeline: chunk n is decoded and multiplied (rows in stage n & 1, codes and norm
  // in the set X) while the rows of chunk n + 1 are copied to the other stage (its ids were
  // loaded a step earlier into the set Y) and the ids of chunk n + 2 load into X. The two
  // register sets swap roles in a loop unrolled twice, so no register holding a load in
  // flight is copied; only chunk positions (already resolved) move between p0, p1, p2.
  DecPos p0, p1, p2;
  p0.slot = p1.slot = p2.slot = 0;
  p0.tb = p0.te = p0.c0 = 0;
  p0.xe = make_float2(0.f, 0.f);
  p1 = p2 = p0;
  uint4 cwa = make_uint4(0u, 0u, 0u, 0u), cwb = make_uint4(0u, 0u, 0u, 0u);
  float rha = 0.f, rhb = 0.f;
  int32_t cida = 0, cidb = 0;
  float mx[4][2];
#pragma unroll
  for (int nt = 0; nt < 4; nt++) mx[nt][0] = mx[nt][1] = -INFINITY;
  float th[4][2];                  // window variant: thr of this lane's query tokens for the current document
#pragma unroll
  for (int nt = 0; nt < 4; nt++) th[nt][0] = th[nt][1] = INFINITY;

  // process the chunk P in stage B with codes CW and norm RH; HN: a next chunk exists, NSLOT its slot
  auto process = [&](const DecPos &P, const int B, const uint4 &CW, const float RH, const bool HN,
                     const int NSLOT) {
    __syncwarp();
    // decode in place: x~ = c + rho * w (fp16 codewords), rounded to fp16.
    // This lane: row drow, dims [dhalf * 64, +64) = subspaces [dhalf * M / 2, +M / 2).
    {
      unsigned char *xrow = wt + B * TILE + drow * PITCH;             // this lane's row
      const uint8_t *cb8 = reinterpret_cast<const uint8_t *>(&CW);  // codes of this lane's subspaces
      // the window variant measures each row's norms (its per-pair test needs them); the main
      // pass takes the document's maxima from doc_xe, formed at index load by the same arithmetic
      float x2 = 0.f, ex2 = 0.f, cwe2 = 0.f;
      if constexpr (WIN) {
#pragma unroll
        for (int mm = 0; mm < M / 2; mm++) cwe2 += cerr2[(dhalf * (M / 2) + mm) * 256 + cb8[mm]];
      }
#pragma unroll
      for (int v = 0; v < 8; v++) {  // 8 dims per step
        // the step's 16-byte chunk of the lane's half: in the lane's own order on swizzled tiles
        const int ch = SWZ ? (ja ^ v) : v;
        const int coff = SWZ ? ((dhalf * 8 + ch) ^ j7) << 4 : dhalf * 128 + v * 16;
        const uint4 cu = *reinterpret_cast<const uint4 *>(xrow + coff);
        const uint32_t cwd[4] = {cu.x, cu.y, cu.z, cu.w};
        uint32_t wv[4];
        if constexpr (SWZ) {
          // code-major codebook: the piece of codeword (code, m) for dims (ch * 8) % DS .. +8
          const int mloc = (ch * 8) / DS;
          const int m = dhalf * (M / 2) + mloc;
          const int code = (int)(__byte_perm(CW.x, CW.y, (uint32_t)mloc) & 0xffu);
          const uint4 t = *reinterpret_cast<const uint4 *>(cbk + (code * M + m) * DS + (ch * 8) % DS);
          wv[0] = t.x; wv[1] = t.y; wv[2] = t.z; wv[3] = t.w;
        } else {
          const int mm = 2 * v;
          const int m = dhalf * (M / 2) + mm;
          const uint2 t0 = *reinterpret_cast<const uint2 *>(cbk + (m * 256 + cb8[mm]) * DS);
          const uint2 t1 = *reinterpret_cast<const uint2 *>(cbk + ((m + 1) * 256 + cb8[mm + 1]) * DS);
          wv[0] = t0.x; wv[1] = t0.y; wv[2] = t1.x; wv[3] = t1.y;
        }
        uint32_t ob[4];
#pragma unroll
        for (int h = 0; h < 4; h++) {
          const float2 w = __half22float2(*reinterpret_cast<const __half2 *>(&wv[h]));
          const float c0 = __uint_as_float(cwd[h] << 16), c1 = __uint_as_float(cwd[h] & 0xffff0000u);
          const float xs0 = fmaf(RH, w.x, c0), xs1 = fmaf(RH, w.y, c1);
          const __half2 xb = __floats2half2_rn(xs0, xs1);
          if constexpr (WIN) {
            const float2 xf = __half22float2(xb);
            x2 = fmaf(xf.x, xf.x, fmaf(xf.y, xf.y, x2));
            ex2 = fmaf(xf.x - xs0, xf.x - xs0, fmaf(xf.y - xs1, xf.y - xs1, ex2));
          }
          ob[h] = *reinterpret_cast<const uint32_t *>(&xb);
        }
        *reinterpret_cast<uint4 *>(xrow + coff) = make_uint4(ob[0], ob[1], ob[2], ob[3]);
      }
      if constexpr (WIN) {
        // the two halves of the row: ||x^||, ||e_x|| (fp16 rounding of x~, plus rho times the
        // codeword rounding, plus the FP32 rounding of x~ itself)
        x2 += __shfl_xor_sync(0xffffffffu, x2, 16);
        ex2 += __shfl_xor_sync(0xffffffffu, ex2, 16);
        cwe2 += __shfl_xor_sync(0xffffffffu, cwe2, 16);
        if (P.c0 + drow < P.te && dhalf == 0) {
          const float slack = 1.f + ldexpf(1.f, -10);
          const float xn = sqrtf(x2) * slack;
          rnx[2 * drow] = xn;
          rnx[2 * drow + 1] = (sqrtf(ex2) + RH * sqrtf(cwe2)) * slack + ldexpf(xn, -22);
        }
      }
    }
    __syncwarp();
    float acc[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; nt++) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
    const uint32_t la = wt_s + (uint32_t)(B * TILE) + la_off;
#pragma unroll
    for (int s = 0; s < 8; s++) {
      uint32_t a[4];
      rd_ldm4(a, SWZ ? la + (uint32_t)((((2 * s) + (lane >> 4)) ^ (lane & 7)) << 4) : la + s * 32);
#pragma unroll
      for (int np = 0; np < 2; np++) {
        uint32_t bb[4];
        rd_ldm4(bb, qs_s + lb_off + (uint32_t)(np * 16 * RD_ROW + s * 32));
        rd_mma(acc[2 * np], a, bb[0], bb[1]);
        rd_mma(acc[2 * np + 1], a, bb[2], bb[3]);
      }
    }
    const int tig = lane & 3;
    if (WIN) {
      // thresholds of this lane's query tokens, at the document's first chunk
      if (P.c0 == P.tb) {
        const float *tq = thr + ((int64_t)q * kd + win_slot[(int64_t)q * kd + P.slot]) * 32;
#pragma unroll
        for (int nt = 0; nt < 4; nt++) {
          th[nt][0] = tq[nt * 8 + tig * 2];
          th[nt][1] = tq[nt * 8 + tig * 2 + 1];
        }
        emx[((int64_t)q * kd + P.slot) * 32 + lane] = fkey(-INFINITY);
      }
      // pairs whose approximate value plus its own bound reaches thr: scored exactly
      uint32_t fl = 0u;
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int row = gq + h * 8;
        if (P.c0 + row >= P.te) continue;
        const float xn = rnx[2 * row], en = rnx[2 * row + 1];
#pragma unroll
        for (int nt = 0; nt < 4; nt++) {
#pragma unroll
          for (int e = 0; e < 2; e++) {
            const int i = nt * 8 + tig * 2 + e;
            const float eps = (qn[i] * (xn + en + cerr) + qn[32 + i] * (en + cerr) + ldexpf(qn[32 + i] * xn, -17) +
                               ldexpf((qn[i] + qn[32 + i]) * (xn + en + 2.f * cnorm), -16)) *
                              (1.f + ldexpf(1.f, -9));
            if (i < ntok && !(acc[nt][h * 2 + e] + eps < th[nt][e])) fl |= 1u << (h * 8 + nt * 2 + e);
          }
        }
      }
      // append them to the list: a warp-wide scan of the counts, one atomic per warp
      const int nf = __popc(fl);
      int pre = nf;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, pre, o);
        if (lane >= o) pre += y;
      }
      const int tot = __shfl_sync(0xffffffffu, pre, 31);
      if (tot > 0) {
        // the counter keeps counting once the list is full (every pair of a tied window can pass
        // the test: billions of offers), so it is 64-bit and never wraps
        unsigned long long wb = 0ull;
        if (lane == 31) wb = atomicAdd(wl_n, (unsigned long long)tot);
        wb = __shfl_sync(0xffffffffu, wb, 31) + (unsigned long long)(pre - nf);
        if (wb + (unsigned long long)nf > (unsigned long long)wl_cap) {
          if (nf) wovf[(int64_t)q * kd + P.slot] = 1;  // the list is full: this document goes to the FP32 kernel
          // a reservation that straddles the cap leaves its positions below the cap unwritten: they
          // get the sentinel (-1), so the reader never takes a pair from an earlier batch
          for (unsigned long long p = wb; p < (unsigned long long)wl_cap && p < wb + (unsigned long long)nf; p++)
            wl[p] = make_int2(-1, 0);
        } else {
          int base = (int)wb;
          const int sid = q * kd + P.slot;
          while (fl) {
            const int b = __ffs(fl) - 1;
            fl &= fl - 1u;
            const int h = b >> 3, nt = (b >> 1) & 3, e = b & 1;
            const int i = nt * 8 + tig * 2 + e;
            wl[base++] = make_int2(sid, (int)((P.c0 + gq + h * 8 - P.tb) << 5) | i);
          }
        }
      }
    } else {
      // running max per query token over this thread's tokens (rows gq, gq + 8)
#pragma unroll
      for (int h = 0; h < 2; h++) {
        if (P.c0 + gq + h * 8 >= P.te) continue;
#pragma unroll
        for (int nt = 0; nt < 4; nt++) {
          mx[nt][0] = fmaxf(mx[nt][0], acc[nt][h * 2 + 0]);
          mx[nt][1] = fmaxf(mx[nt][1], acc[nt][h * 2 + 1]);
        }
      }
    }
    if (!WIN && (!HN || NSLOT != P.slot)) {
      // document complete: max over the lanes sharing tig, sum over query tokens, the bound
      // (xm, em: max over the document's tokens of ||x^_t|| and ||e_x,t||)
      const float xm = P.xe.x, em = P.xe.y;
      float sum = 0.f, dl = 0.f;
#pragma unroll
      for (int nt = 0; nt < 4; nt++) {
#pragma unroll
        for (int e = 0; e < 2; e++) {
          float v = mx[nt][e];
          v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 4));
          v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 8));
          v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 16));
          const int i = nt * 8 + tig * 2 + e;
          float ti = -INFINITY;
          if (i < ntok) {
            sum += v;
            // |<q^, x^> - <q, x>| <= ||e_q|| ||x|| + ||q^|| ||x^ - x||, ||x|| <= ||x^|| + ||x^ - x||
            const float ei = qn[i] * (xm + em + cerr) + qn[32 + i] * (em + cerr) + ldexpf(qn[32 + i] * xm, -17) +
                             ldexpf((qn[i] + qn[32 + i]) * (xm + em + 2.f * cnorm), -16);
            dl += ei;
            // the token of the approximate maximum is within ei of it: no exact maximum lies below
            ti = v - ei * (1.f + ldexpf(1.f, -9)) - ldexpf(fabsf(v) + 1.f, -20);
          }
          if (gq == 0) thr[((int64_t)q * kd + P.slot) * 32 + i] = ti;
          mx[nt][e] = -INFINITY;
        }
      }
      sum += __shfl_xor_sync(0xffffffffu, sum, 1);
      sum += __shfl_xor_sync(0xffffffffu, sum, 2);
      dl += __shfl_xor_sync(0xffffffffu, dl, 1);
      dl += __shfl_xor_sync(0xffffffffu, dl, 2);
      if (lane == 0) {
        sa_row[P.slot] = sum;
        da_row[P.slot] = dl * (1.f + ldexpf(1.f, -10)) + ldexpf(fabsf(sum) + 1.f, -20) * 8.f;
      }
    }
  };

  bool v0 = dec_next(p0, s_end, stride, off, &s_next, cand_q, doc_off, WIN ? nullptr : doc_xe, D, bad, flags, lane), v1 = false, v2 = false;
  if (v0) {
    cida = load_cid(p0);
    issue_rows(p0, cida, 0, cwa, rha);
    p1 = p0;
    v1 = dec_next(p1, s_end, stride, off, &s_next, cand_q, doc_off, WIN ? nullptr : doc_xe, D, bad, flags, lane);
    if (v1) cidb = load_cid(p1);
  }
  int n = 0;
  auto step = [&](int32_t &xcid, const uint4 &xcw, const float &xrh, const int32_t &ycid, uint4 &ycw, float &yrh) {
    v2 = false;
    if (v1) {
      p2 = p1;
      v2 = dec_next(p2, s_end, stride, off, &s_next, cand_q, doc_off, WIN ? nullptr : doc_xe, D, bad, flags, lane);
      if (v2) xcid = load_cid(p2);
      issue_rows(p1, ycid, (n + 1) & 1, ycw, yrh);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    process(p0, n & 1, xcw, xrh, v1, p1.slot);
    __syncwarp();
    p0 = p1;
    v0 = v1;
    p1 = p2;
    v1 = v2;
    n++;
  };
  while (v0) {
    step(cida, cwa, rha, cidb, cwb, rhb);
    if (!v0) break;
    step(cidb, cwb, rhb, cida, cwa, rha);
  }
}

template <int M>
__global__ void __launch_bounds__(256)
k_dec_exact_pairs(const float *__restrict__ queries, const int32_t *__restrict__ meta, int nq, int kd,
                  const int32_t *__restrict__ win, const int64_t *__restrict__ doc_off,
                  const int32_t *__restrict__ tok_cid, const uint8_t *__restrict__ codes,
                  const uint16_t *__restrict__ rnorm, const float *__restrict__ codebooks,
                  const float *__restrict__ cent_f32, const __nv_bfloat16 *__restrict__ cent_bf16, int bf16c,
                  const int2 *__restrict__ wl, const unsigned long long *__restrict__ wl_n, int wl_cap,
                  uint32_t *__restrict__ emx, uint32_t *__restrict__ flags) {
  const int n = (int)min(*wl_n, (unsigned long long)wl_cap);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int2 e = wl[k];
    if (e.x < 0) continue;  // a sentinel below the cap
    if (e.x >= nq * kd) {   // not reachable: every entry below the cap is written by this batch
      atomicOr(flags, TACHIOM_FLAG_CAPACITY);
      continue;
    }
    const int sid = e.x, q = sid / kd, i = e.y & 31;
    const int64_t t = doc_off[win[sid]] + (e.y >> 5);
    const float v = dec_exact<M>(queries + ((int64_t)meta[q] + i) * DIM, t, tok_cid, codes, rnorm, codebooks,
                                 cent_f32, cent_bf16, bf16c != 0);
    atomicMax(&emx[(int64_t)sid * 32 + i], fkey(v));
  }
}

// Per window document: the exact maxima summed per group of query tokens, as k_refine forms
// part[q][group][slot]. Empty and out-of-range documents were answered by the window pass;
// a document marked in wovf is left to the all-pairs FP32 kernel.
__global__ void __launch_bounds__(256)
k_win_sums(const int32_t *__restrict__ meta, int nq, const int32_t *__restrict__ win, int kd,
           const int64_t *__restrict__ doc_off, int64_t D, const uint32_t *__restrict__ emx,
           const int32_t *__restrict__ wovf, int G, int ngroups, float *__restrict__ part) {
  const int q = blockIdx.y;
  const int ntok = meta[3 * nq + 2 + q];
  const int gq_n = (ntok + G - 1) / G;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < kd * gq_n; x += gridDim.x * blockDim.x) {
    const int slot = x / gq_n, grp = x % gq_n;
    const int64_t sid = (int64_t)q * kd + slot;
    const int32_t d = win[sid];
    if (d < 0) continue;
    if (d >= D || doc_off[d + 1] == doc_off[d] || wovf[sid]) continue;
    const int i0 = grp * G, ng = min(G, ntok - i0);
    float sum = 0.f;
    for (int g = 0; g < ng; g++) sum += funkey(emx[sid * 32 + i0 + g]);
    part[((int64_t)q * ngroups + grp) * kd + slot] = sum;
  }
}

// Per document d, the two norms the main pass's bound Delta_d takes: the max over d's tokens of
// ||h(x~_t)|| and of ||e_x,t||, where x~_t = fmaf(rho_t, h(w), c_t) element by element (c_t the BF16
// centroid row, h(w) the fp16 codeword), h() the rounding to fp16, and e_x,t the fp16 rounding of
// x~_t plus rho_t times the codeword rounding plus the FP32 rounding of x~_t. The per-element values
// are the decode pass's own; the sums run in another order, which the slack of 2^-10 covers (the
// FP32 rounding of a 128-term sum of squares is below 2^-16 of it). Depends on the index only, so it
// is formed once at load. One warp per document, lane l on dims 4l .. 4l + 3 of each token; an empty
// document gets (0, 0).
template <int M>
__global__ void __launch_bounds__(256)
k_doc_decode_norms(const int64_t *__restrict__ doc_off, int64_t D, const int32_t *__restrict__ tok_cid,
                   const uint8_t *__restrict__ codes, const uint16_t *__restrict__ rnorm,
                   const float *__restrict__ codebooks, const __nv_bfloat16 *__restrict__ cent_bf16,
                   float2 *__restrict__ doc_xe) {
  constexpr int DS = 128 / M;
  static_assert(DS % 4 == 0, "a lane's 4 dims lie in one subspace");
  const int lane = threadIdx.x & 31;
  const int m = (4 * lane) / DS, u0 = (4 * lane) % DS;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t d = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x >> 5); d < D; d += nw) {
    float xmax = 0.f, emax = 0.f;
    const int64_t te = doc_off[d + 1];
    for (int64_t t = doc_off[d]; t < te; t++) {
      const uint2 cr = *reinterpret_cast<const uint2 *>(cent_bf16 + (int64_t)tok_cid[t] * DIM + 4 * lane);
      const int code = codes[t * M + m];
      const float4 w4 = *reinterpret_cast<const float4 *>(codebooks + ((int64_t)m * 256 + code) * DS + u0);
      const float rh = __half2float(__ushort_as_half(rnorm[t]));
      const float c[4] = {__uint_as_float(cr.x << 16), __uint_as_float(cr.x & 0xffff0000u),
                          __uint_as_float(cr.y << 16), __uint_as_float(cr.y & 0xffff0000u)};
      const float w[4] = {w4.x, w4.y, w4.z, w4.w};
      float x2 = 0.f, ex2 = 0.f, cwe2 = 0.f;
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const float wr = __half2float(__float2half_rn(w[k]));
        cwe2 = fmaf(wr - w[k], wr - w[k], cwe2);
        const float xs = fmaf(rh, wr, c[k]);
        const float xf = __half2float(__float2half_rn(xs));
        x2 = fmaf(xf, xf, x2);
        ex2 = fmaf(xf - xs, xf - xs, ex2);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        x2 += __shfl_xor_sync(0xffffffffu, x2, o);
        ex2 += __shfl_xor_sync(0xffffffffu, ex2, o);
        cwe2 += __shfl_xor_sync(0xffffffffu, cwe2, o);
      }
      const float slack = 1.f + ldexpf(1.f, -10);
      const float xn = sqrtf(x2) * slack;
      xmax = fmaxf(xmax, xn);
      emax = fmaxf(emax, (sqrtf(ex2) + rh * sqrtf(cwe2)) * slack + ldexpf(xn, -22));
    }
    if (lane == 0) doc_xe[d] = make_float2(xmax, emax);
  }
}

// The decode pass's fp16 codebook, in the layout it keeps in shared memory (code-major
// [256][M][ds] for M = 8, 16; subspace-major [M][256][ds] for M = 32), each value rounded to
// nearest; and per codeword (m, j) the squared norm of its rounding error, [M][256].
template <int M>
__global__ void __launch_bounds__(256)
k_codebook_h16(const float *__restrict__ codebooks, __half *__restrict__ out, float *__restrict__ err2) {
  constexpr int DS = 128 / M;
  for (int mj = blockIdx.x * blockDim.x + threadIdx.x; mj < M * 256; mj += gridDim.x * blockDim.x) {
    const int m = mj / 256, j = mj % 256;
    __half *o = out + (rd_swz<M>() ? (j * M + m) * DS : mj * DS);
    float e2 = 0.f;
    for (int u = 0; u < DS; u++) {
      const float w = codebooks[(int64_t)mj * DS + u];
      const __half wb = __float2half_rn(w);
      o[u] = wb;
      const float d = __half2float(wb) - w;
      e2 = fmaf(d, d, e2);
    }
    err2[mj] = e2;
  }
}

template <int M>
static tachiom_status launch_decode_tables_m(const Index &ix, cudaStream_t s) {
  k_codebook_h16<M><<<M, 256, 0, s>>>(ix.codebooks, reinterpret_cast<__half *>(ix.cbk_h16), ix.cbk_err2);
  TLAUNCH();
  if (ix.D > 0) {
    const int64_t blocks = (ix.D + 7) / 8;
    const unsigned grid = (unsigned)(blocks < 8192 ? blocks : 8192);
    k_doc_decode_norms<M><<<grid, 256, 0, s>>>(ix.doc_off, ix.D, ix.tok_cid, ix.codes, ix.rnorm, ix.codebooks,
                                               ix.cent_bf16, ix.doc_xe);
    TLAUNCH();
  }
  return TACHIOM_OK;
}

tachiom_status launch_decode_tables(const Index &ix, cudaStream_t s) {
  switch (ix.M) {
    case 8: return launch_decode_tables_m<8>(ix, s);
    case 16: return launch_decode_tables_m<16>(ix, s);
    case 32: return launch_decode_tables_m<32>(ix, s);
  }
  return fail(TACHIOM_ERR_INVALID, "unsupported pq_m %d", ix.M);
}

template <int M, bool WIN>
static tachiom_status launch_refine_dec_m(const Index &ix, const float *queries, const int32_t *meta, int nq,
                                          const int32_t *cand, int kd, float *sa, float *da, float *thr,
                                          const int32_t *win_slot, float *part, const WinScratch *ws,
                                          uint32_t *flags, cudaStream_t s) {
  constexpr int W = rd_warps<M, WIN>();
  static_assert(W >= 4, "decode refine: shared memory for fewer than 4 warps");
  const size_t smem = (size_t)rd_fixed_bytes<M>() + (size_t)W * rd_warp_bytes<M, WIN>();
  // the window variant takes a query's whole (short) list in one CTA
  dim3 grid(WIN ? 2 : (kd + RD_DOCS_PER_CTA - 1) / RD_DOCS_PER_CTA, nq);
  TCUDA(cudaFuncSetAttribute(k_refine_dec<M, W, WIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_refine_dec<M, W, WIN><<<grid, W * 32, smem, s>>>(
      queries, meta, nq, cand, kd, ix.doc_off, ix.tok_cid, ix.codes, ix.rnorm,
      reinterpret_cast<const __half *>(ix.cbk_h16), ix.cbk_err2, ix.cent_bf16, ix.cent_f32,
      ix.cdtype == TACHIOM_DTYPE_BF16 ? 1 : 0, ix.doc_xe, ix.cerr_max, ix.cnorm_max + ix.cerr_max, sa, da, thr,
      win_slot, part, refine_groups(M), ws ? ws->wl : nullptr, ws ? ws->wl_n : nullptr, ws ? ws->wl_cap : 0,
      ws ? ws->emx : nullptr, ws ? ws->wovf : nullptr, ix.D, flags);
  TLAUNCH();
  if (WIN) {
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix.device);
    k_dec_exact_pairs<M><<<sms * 4, 256, 0, s>>>(queries, meta, nq, kd, cand, ix.doc_off, ix.tok_cid, ix.codes,
                                                 ix.rnorm, ix.codebooks, ix.cent_f32, ix.cent_bf16,
                                                 ix.cdtype == TACHIOM_DTYPE_BF16 ? 1 : 0, ws->wl, ws->wl_n,
                                                 ws->wl_cap, ws->emx, flags);
    TLAUNCH();
    k_win_sums<<<dim3((kd * 4 + 255) / 256, nq), 256, 0, s>>>(meta, nq, cand, kd, ix.doc_off, ix.D, ws->emx, ws->wovf,
                                                              128 / M, refine_groups(M), part);
    TLAUNCH();
  }
  return TACHIOM_OK;
}

tachiom_status launch_refine_dec(const Index &ix, const float *queries, const int32_t *meta, int nq,
                                 const int32_t *cand, int kd, float *sa, float *da, float *thr, uint32_t *flags,
                                 cudaStream_t s) {
  if (nq <= 0) return TACHIOM_OK;
  TPROF("refine_dec", s);
  switch (ix.M) {
    case 8: return launch_refine_dec_m<8, false>(ix, queries, meta, nq, cand, kd, sa, da, thr, nullptr, nullptr, nullptr, flags, s);
    case 16: return launch_refine_dec_m<16, false>(ix, queries, meta, nq, cand, kd, sa, da, thr, nullptr, nullptr, nullptr, flags, s);
    case 32: return launch_refine_dec_m<32, false>(ix, queries, meta, nq, cand, kd, sa, da, thr, nullptr, nullptr, nullptr, flags, s);
  }
  return fail(TACHIOM_ERR_INVALID, "unsupported pq_m %d", ix.M);
}

tachiom_status launch_refine_dec_win(const Index &ix, const float *queries, const int32_t *meta, int nq,
                                     const int32_t *win, const int32_t *win_slot, int kd, float *thr, float *part,
                                     const WinScratch &ws, uint32_t *flags, cudaStream_t s) {
  if (nq <= 0) return TACHIOM_OK;
  TPROF("refine_win", s);
  TCUDA(cudaMemsetAsync(ws.wl_n, 0, sizeof(unsigned long long), s));
  TCUDA(cudaMemsetAsync(ws.wovf, 0, (size_t)nq * kd * sizeof(int32_t), s));
  switch (ix.M) {
    case 8: return launch_refine_dec_m<8, true>(ix, queries, meta, nq, win, kd, nullptr, nullptr, thr, win_slot, part, &ws, flags, s);
    case 16: return launch_refine_dec_m<16, true>(ix, queries, meta, nq, win, kd, nullptr, nullptr, thr, win_slot, part, &ws, flags, s);
    case 32: return launch_refine_dec_m<32, true>(ix, queries, meta, nq, win, kd, nullptr, nullptr, thr, win_slot, part, &ws, flags, s);
  }
  return fail(TACHIOM_ERR_INVALID, "unsupported pq_m %d", ix.M);
}

}  // namespace tachiom
