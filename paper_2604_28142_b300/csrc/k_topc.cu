// Step (a): every query token against every centroid, keeping the kappa_c best
// (Sec. 2.2, Gather step 1, in the exhaustive form the graph search
// approximates).
//
// This file holds the FP32 CUDA-core path (the plain comparator) and the
// merge that both precisions share:
//   k_topc_f32_scan  a CTA owns 32 query rows and one slice ("split") of the
//                    centroids; it forms 32 x 128 score tiles with FFMA and
//                    keeps, per row, every score that can still be among the
//                    row's kappa_c best seen so far (a threshold raised by
//                    periodic compaction of a shared-memory buffer);
//   k_topc_merge     one CTA per row merges the splits' survivors, optionally
//                    rescoring the ones near the boundary in FP32 (BF16 path),
//                    and writes the exact top-kappa_c by (score desc, id asc).
// The FP32 score of (row, centroid) is always the same sequence of fmaf over
// k = 0..127, in the scan, in the rescoring and in k_score_pairs, so every
// path produces bit-identical FP32 scores.
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <cstring>

#include "tachiom_internal.cuh"

namespace tachiom {

// Rows to BF16 (round to nearest) and, per row, the half-width of the window the
// BF16 scores must be repaired in. With e = bf16(q) - q and c_hat the BF16 copy of
// c (exact for a BF16-stored table):
//   |<bf16(q), c_hat> - <q, c>| <= |<e, c>| + |<bf16(q), c_hat - c>| + accumulation
//                                <= ||e|| cmax + ||bf16(q)|| (cerr + 2^-15 cmax)
// (Cauchy-Schwarz; cmax = max ||c_j||, cerr = max ||c_hat_j - c_j||; the last term
// bounds the FP32 accumulation of 128 products). margin = 2 * that bound.
__global__ void k_quantize_rows(const float *__restrict__ in, __nv_bfloat16 *__restrict__ out, int nrows,
                                float cmax, float cerr, float *__restrict__ margins) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nrows) return;
  const float4 x = reinterpret_cast<const float4 *>(in + (int64_t)warp * DIM)[lane];
  const float xs[4] = {x.x, x.y, x.z, x.w};
  float e2 = 0.f, h2 = 0.f;
  __nv_bfloat16 hb[4];
#pragma unroll
  for (int u = 0; u < 4; u++) {
    hb[u] = __float2bfloat16_rn(xs[u]);
    const float h = __bfloat162float(hb[u]);
    e2 = fmaf(h - xs[u], h - xs[u], e2);
    h2 = fmaf(h, h, h2);
  }
  reinterpret_cast<uint2 *>(out + (int64_t)warp * DIM)[lane] =
      make_uint2(*reinterpret_cast<uint16_t *>(&hb[0]) | ((uint32_t)*reinterpret_cast<uint16_t *>(&hb[1]) << 16),
                 *reinterpret_cast<uint16_t *>(&hb[2]) | ((uint32_t)*reinterpret_cast<uint16_t *>(&hb[3]) << 16));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    h2 += __shfl_xor_sync(0xffffffffu, h2, o);
  }
  if (lane == 0 && margins) {
    // the factor 1 + 2^-10 covers the FP32 rounding of these norms
    const float d = (sqrtf(e2) * cmax + sqrtf(h2) * (cerr + ldexpf(cmax, -15))) * (1.f + ldexpf(1.f, -10)) + 1e-7f;
    margins[warp] = 2.f * d;
  }
}

tachiom_status launch_quantize_bf16(const float *rows, __nv_bfloat16 *out, int64_t n, cudaStream_t s) {
  // n = rows x 128; no margins
  if (n <= 0) return TACHIOM_OK;
  TPROF("quantize_bf16", s);
  const int nrows = (int)(n / DIM);
  k_quantize_rows<<<(nrows + 7) / 8, 256, 0, s>>>(rows, out, nrows, 0.f, 0.f, nullptr);
  TLAUNCH();
  return TACHIOM_OK;
}

tachiom_status launch_quantize_rows(const Index &ix, const float *rows, __nv_bfloat16 *out, int nrows,
                                    float *margins, cudaStream_t s) {
  if (nrows <= 0) return TACHIOM_OK;
  TPROF("quantize_bf16", s);
  k_quantize_rows<<<(nrows + 7) / 8, 256, 0, s>>>(rows, out, nrows, ix.cnorm_max, ix.cerr_max, margins);
  TLAUNCH();
  return TACHIOM_OK;
}

// Rows to E4M3 (round to nearest, saturating) with a power-of-two scale per row: y = x * 2^s,
// 2^s the largest power of two with max_k |x_k| * 2^s <= 448, so max |y| is in (224, 448] and the
// scaling is exact; inv[r] = 2^-s and the decoded row is x~ = e4m3(y) * 2^-s. Per row, the rigorous
// bound of the E4M3 score error against a centroid c with e4m3 copy c~ (Cauchy-Schwarz; products of
// two E4M3 values are exact in FP32 and the accumulation of 128 of them adds at most 2^-15 ||x~|| cmax):
//   |<x~, c~> - <x, c>| <= ||x~ - x|| cmax + ||x~|| (cerr8 + 2^-15 cmax) = delta
// and margins[r] = 2 lambda delta (lambda = 1: the rigorous window). With err_max, the largest
// ||x~ - x|| over the rows is folded in by atomicMax (index load). One warp per row.
__global__ void k_quant_e4m3(const float *__restrict__ in, int64_t nrows, uint8_t *__restrict__ out,
                             float *__restrict__ inv, float cmax, float cerr8, float lambda,
                             float *__restrict__ margins, unsigned *__restrict__ err_max) {
  const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= nrows) return;
  const float4 x = reinterpret_cast<const float4 *>(in + r * DIM)[lane];
  const float xs[4] = {x.x, x.y, x.z, x.w};
  float amax = fmaxf(fmaxf(fabsf(x.x), fabsf(x.y)), fmaxf(fabsf(x.z), fabsf(x.w)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  int s = 0;
  if (amax > 0.f) {
    int e;
    frexpf(448.f / amax, &e);  // 448 / amax = f 2^e, f in [0.5, 1): 2^(e-1) <= 448 / amax
    s = min(e - 1, 126);
  }
  const float scale = ldexpf(1.f, s), iscale = ldexpf(1.f, -s);
  uint32_t packed = 0;
  float e2 = 0.f, h2 = 0.f;
#pragma unroll
  for (int u = 0; u < 4; u++) {
    const __nv_fp8_storage_t b = __nv_cvt_float_to_fp8(xs[u] * scale, __NV_SATFINITE, __NV_E4M3);
    packed |= (uint32_t)b << (8 * u);
    const __half_raw hr = __nv_cvt_fp8_to_halfraw(b, __NV_E4M3);
    const float d = __half2float(__half(hr)) * iscale;
    e2 = fmaf(d - xs[u], d - xs[u], e2);
    h2 = fmaf(d, d, h2);
  }
  reinterpret_cast<uint32_t *>(out + r * DIM)[lane] = packed;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    h2 += __shfl_xor_sync(0xffffffffu, h2, o);
  }
  if (lane == 0) {
    inv[r] = iscale;
    if (margins) {
      // the factor 1 + 2^-10 covers the FP32 rounding of these norms
      const float d = (sqrtf(e2) * cmax + sqrtf(h2) * (cerr8 + ldexpf(cmax, -15))) * (1.f + ldexpf(1.f, -10)) + 1e-7f;
      margins[r] = 2.f * lambda * d;
    }
    if (err_max) atomicMax(err_max, __float_as_uint(sqrtf(e2) * (1.f + ldexpf(1.f, -12))));
  }
}

tachiom_status launch_quantize_e4m3(const Index &ix, const float *rows, int nrows, uint8_t *out, float *inv,
                                    float lambda, float *margins, cudaStream_t s) {
  if (nrows <= 0) return TACHIOM_OK;
  TPROF("quantize_e4m3", s);
  k_quant_e4m3<<<(nrows + 7) / 8, 256, 0, s>>>(rows, nrows, out, inv, ix.cnorm_max, ix.cerr8_max, lambda, margins,
                                              nullptr);
  TLAUNCH();
  return TACHIOM_OK;
}

tachiom_status launch_cent_e4m3(Index &ix, cudaStream_t s) {
  unsigned *d = nullptr;
  if (cudaMalloc(&d, 4) != cudaSuccess) {
    cudaGetLastError();
    return fail(TACHIOM_ERR_OOM, "cudaMalloc of 4 bytes failed");
  }
  cudaMemsetAsync(d, 0, 4, s);
  const int64_t blocks = (ix.C + 7) / 8;
  k_quant_e4m3<<<(unsigned)blocks, 256, 0, s>>>(ix.cent_f32, ix.C, ix.cent_e4m3, ix.cent_inv_sc, 0.f, 0.f, 0.f,
                                                nullptr, d);
  unsigned h = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  if (e != cudaSuccess) return fail(TACHIOM_ERR_CUDA, "E4M3 centroid copy failed: %s", cudaGetErrorString(e));
  float f;
  memcpy(&f, &h, 4);
  ix.cerr8_max = f;
  return TACHIOM_OK;
}

// exact FP32 score: fmaf chain over k = 0..127
__device__ __forceinline__ float dot_f32(const float *__restrict__ q, const float *__restrict__ c) {
  float acc = 0.f;
#pragma unroll 8
  for (int k = 0; k < DIM; k++) acc = fmaf(q[k], c[k], acc);
  return acc;
}

// ---------------------------------------------------------------------------------
// FP32 scan
constexpr int F_ROWS = 32;    // query rows per CTA
constexpr int F_COLS = 128;   // centroids per tile
constexpr int F_CAP = 256;    // per-row candidate buffer (>= kappa_c + F_COLS)
constexpr int F_THREADS = 256;

struct RowBuf {
  float thr;  // entries below thr - margin can no longer reach the row's top kappa_c
  int cnt;
};

// Sort one row's buffer and keep what can still reach the top kappa_c.
// Called by one warp. Returns the new count; sets *lossy when the kept set
// does not fit the room the next tile needs.
__device__ __forceinline__ void compact_row(uint64_t *buf, RowBuf &rb, int kc, float margin, int room,
                                            int *lossy) {
  const int lane = threadIdx.x & 31;
  int n = rb.cnt;
  if (n > F_CAP) n = F_CAP;
  for (int i = n + lane; i < F_CAP; i += 32) buf[i] = 0ull;
  __syncwarp();
  warp_sort_desc(buf, F_CAP);
  if (n >= kc) {
    float t = comp_score(buf[kc - 1]);
    // keep every entry >= t - margin (ties and the rescoring window)
    int keep = kc;
    float lim = t - margin;
    // entries are sorted: count the kept prefix (n <= 256, sequential is cheap)
    if (lane == 0) {
      while (keep < n && comp_score(buf[keep]) >= lim) keep++;
      if (keep > F_CAP - room) {
        keep = F_CAP - room;
        *lossy = 1;
      }
      rb.cnt = keep;
      rb.thr = t;
    }
  } else if (lane == 0) {
    rb.cnt = n;
  }
  __syncwarp();
}

template <bool BF16SRC>
__global__ void __launch_bounds__(F_THREADS, 1)
k_topc_f32_scan(const float *__restrict__ rows, int nrows, const float *__restrict__ cent,
                const __nv_bfloat16 *__restrict__ cent_bf16, int64_t C, int64_t cols_per_split,
                int kc, int capout, uint64_t *__restrict__ split_out, int32_t *__restrict__ split_cnt,
                uint32_t *__restrict__ flags) {
  extern __shared__ __align__(16) unsigned char smem[];
  float *Qt = reinterpret_cast<float *>(smem);                 // [128][32]
  float *Bt = Qt + DIM * F_ROWS;                               // [128][128]
  uint64_t *buf = reinterpret_cast<uint64_t *>(Bt + DIM * F_COLS);  // [32][F_CAP]
  __shared__ RowBuf rb[F_ROWS];
  __shared__ int lossy[F_ROWS];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int row0 = blockIdx.x * F_ROWS;
  const int split = blockIdx.y, nsplit = gridDim.y;
  const int64_t c_begin = (int64_t)split * cols_per_split;
  const int64_t c_end = min(C, c_begin + cols_per_split);

  for (int i = tid; i < DIM * F_ROWS; i += F_THREADS) {
    int r = i / DIM, k = i % DIM;
    Qt[k * F_ROWS + r] = (row0 + r < nrows) ? rows[(int64_t)(row0 + r) * DIM + k] : 0.f;
  }
  if (tid < F_ROWS) {
    rb[tid].thr = -INFINITY;
    rb[tid].cnt = 0;
    lossy[tid] = 0;
  }
  __syncthreads();

  const int rg = warp;   // rows 4*rg .. 4*rg+3
  const int cg = lane;   // cols 4*cg .. 4*cg+3
  for (int64_t c0 = c_begin; c0 < c_end; c0 += F_COLS) {
    // load the tile transposed: lane l takes centroid c0 + (i % 32)*4 + ..., keep it simple:
    // thread loads 4 consecutive dims of one centroid and scatters them to Bt[k][col]
    for (int i = tid; i < F_COLS * (DIM / 4); i += F_THREADS) {
      int col = i % F_COLS, k4 = i / F_COLS;
      int64_t c = c0 + col;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (c < c_end) {
        if (BF16SRC) {
          uint2 u = *reinterpret_cast<const uint2 *>(cent_bf16 + c * DIM + k4 * 4);
          v.x = __uint_as_float(u.x << 16);
          v.y = __uint_as_float(u.x & 0xffff0000u);
          v.z = __uint_as_float(u.y << 16);
          v.w = __uint_as_float(u.y & 0xffff0000u);
        } else {
          v = *reinterpret_cast<const float4 *>(cent + c * DIM + k4 * 4);
        }
      }
      Bt[(k4 * 4 + 0) * F_COLS + col] = v.x;
      Bt[(k4 * 4 + 1) * F_COLS + col] = v.y;
      Bt[(k4 * 4 + 2) * F_COLS + col] = v.z;
      Bt[(k4 * 4 + 3) * F_COLS + col] = v.w;
    }
    __syncthreads();
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int b = 0; b < 4; b++) acc[a][b] = 0.f;
#pragma unroll 4
    for (int k = 0; k < DIM; k++) {
      float4 qa = *reinterpret_cast<const float4 *>(&Qt[k * F_ROWS + rg * 4]);
      float4 cb = *reinterpret_cast<const float4 *>(&Bt[k * F_COLS + cg * 4]);
      float qv[4] = {qa.x, qa.y, qa.z, qa.w};
      float cv[4] = {cb.x, cb.y, cb.z, cb.w};
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) acc[a][b] = fmaf(qv[a], cv[b], acc[a][b]);
    }
    // filter into the row buffers
#pragma unroll
    for (int a = 0; a < 4; a++) {
      int r = rg * 4 + a;
      float lim = rb[r].thr;  // margin 0 on the FP32 path
#pragma unroll
      for (int b = 0; b < 4; b++) {
        int64_t c = c0 + cg * 4 + b;
        if (c < c_end && row0 + r < nrows && acc[a][b] >= lim) {
          int pos = atomicAdd(&rb[r].cnt, 1);
          if (pos < F_CAP) buf[r * F_CAP + pos] = comp_key(acc[a][b], (int32_t)c);
          else lossy[r] = 1;
        }
      }
    }
    __syncthreads();
    // compaction of rows that could not take another full tile
    for (int r = warp; r < F_ROWS; r += F_THREADS / 32) {
      if (rb[r].cnt > F_CAP - F_COLS) compact_row(buf + r * F_CAP, rb[r], kc, 0.f, F_COLS, &lossy[r]);
    }
    __syncthreads();
  }
  // final compaction and output
  for (int r = warp; r < F_ROWS; r += F_THREADS / 32) {
    if (row0 + r >= nrows) continue;
    compact_row(buf + r * F_CAP, rb[r], kc, 0.f, 0, &lossy[r]);
    int n = rb[r].cnt;
    int nout = min(n, capout);
    uint64_t *dst = split_out + ((int64_t)(row0 + r) * nsplit + split) * capout;
    for (int i = lane; i < nout; i += 32) dst[i] = buf[r * F_CAP + i];
    if (lane == 0) {
      split_cnt[(int64_t)(row0 + r) * nsplit + split] = nout | ((lossy[r] || n > capout) ? (1 << 30) : 0);
    }
  }
}

tachiom_status launch_topc_f32(const Index &ix, const float *rows, int nrows, int kc, int splits,
                               int capout, uint64_t *split, int32_t *split_cnt, uint32_t *flags,
                               cudaStream_t s) {
  if (nrows <= 0) return TACHIOM_OK;
  TPROF("topc_f32_scan", s);
  int64_t per = (ix.C + splits - 1) / splits;
  per = (per + F_COLS - 1) / F_COLS * F_COLS;
  dim3 grid((nrows + F_ROWS - 1) / F_ROWS, splits);
  size_t smem = (size_t)DIM * F_ROWS * 4 + (size_t)DIM * F_COLS * 4 + (size_t)F_ROWS * F_CAP * 8;
  if (ix.cdtype == TACHIOM_DTYPE_BF16) {
    TCUDA(cudaFuncSetAttribute(k_topc_f32_scan<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_topc_f32_scan<true><<<grid, F_THREADS, smem, s>>>(rows, nrows, ix.cent_f32, ix.cent_bf16, ix.C, per,
                                                        kc, capout, split, split_cnt, flags);
  } else {
    TCUDA(cudaFuncSetAttribute(k_topc_f32_scan<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_topc_f32_scan<false><<<grid, F_THREADS, smem, s>>>(rows, nrows, ix.cent_f32, ix.cent_bf16, ix.C, per,
                                                         kc, capout, split, split_cnt, flags);
  }
  TLAUNCH();
  return TACHIOM_OK;
}

// ---------------------------------------------------------------------------------
// merge (and, for the BF16 path, FP32 rescoring of the boundary window)
constexpr int M_THREADS = 512;
constexpr int M_MAX = 16384;  // entries one row's merge sorts

__global__ void __launch_bounds__(M_THREADS)
k_topc_merge(const float *__restrict__ rows, int nrows, const float *__restrict__ cent, int64_t C,
             int kc, int splits, int capout, const uint64_t *__restrict__ split_in,
             const int32_t *__restrict__ split_cnt, const float *__restrict__ margins, int rescore,
             int32_t *__restrict__ top_ids, float *__restrict__ top_s, uint32_t *__restrict__ flags,
             int32_t *__restrict__ lossy_rows) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t *a = reinterpret_cast<uint64_t *>(smem);  // [M_MAX]
  __shared__ int offs[1025];
  __shared__ int s_lossy, s_n;
  __shared__ float s_q[DIM];
  const int r = blockIdx.x;
  if (r >= nrows) return;
  const int tid = threadIdx.x;
  if (tid == 0) {
    int o = 0, lo = 0;
    for (int sp = 0; sp < splits; sp++) {
      int v = split_cnt[(int64_t)r * splits + sp];
      if (v & (1 << 30)) lo = 1;
      v &= (1 << 30) - 1;
      if (v > capout) {  // a slice's list overflowed: the row takes the exact fallback
        lo = 1;
        v = capout;
      }
      offs[sp] = o;
      o += v;
    }
    offs[splits] = o;
    s_lossy = lo || (o > M_MAX);
    s_n = min(o, M_MAX);
  }
  for (int k = tid; k < DIM; k += M_THREADS) s_q[k] = rows[(int64_t)r * DIM + k];
  __syncthreads();
  const int n = s_n;
  const int np = next_pow2(max(n, 2));
  for (int sp = 0; sp < splits; sp++) {
    int o = offs[sp], c = offs[sp + 1] - o;
    const uint64_t *src = split_in + ((int64_t)r * splits + sp) * capout;
    for (int i = tid; i < c; i += M_THREADS)
      if (o + i < M_MAX) a[o + i] = src[i];
  }
  for (int i = n + tid; i < np; i += M_THREADS) a[i] = 0ull;
  __syncthreads();
  block_sort_desc(a, np);
  if (rescore) {
    // window: every entry whose approximate score is >= (approx kappa_c-th) - margin
    __shared__ int s_w;
    if (tid == 0) {
      const float margin = margins ? margins[r] : 0.f;
      float t = (n >= kc) ? comp_score(a[kc - 1]) : -INFINITY;
      int w = 0;
      while (w < n && comp_score(a[w]) >= t - margin) w++;
      s_w = w;
    }
    __syncthreads();
    const int w = s_w;
    for (int i = tid; i < w; i += M_THREADS) {
      int32_t id = comp_id(a[i]);
      float sc = dot_f32(s_q, cent + (int64_t)id * DIM);
      a[i] = comp_key(sc, id);
    }
    const int wp = next_pow2(max(w, 2));
    for (int i = w + tid; i < wp; i += M_THREADS) a[i] = 0ull;
    __syncthreads();
    block_sort_desc(a, wp);
  }
  for (int i = tid; i < kc; i += M_THREADS) {
    uint64_t v = (i < n) ? a[i] : 0ull;
    top_ids[(int64_t)r * kc + i] = v ? comp_id(v) : -1;
    top_s[(int64_t)r * kc + i] = v ? comp_score(v) : -INFINITY;
  }
  if (tid == 0 && s_lossy) {
    lossy_rows[r] = 1;
    atomicOr(flags, TACHIOM_FLAG_TOPC_RESCUED);
  }
}

// Exact fallback for a row whose candidate buffer overflowed: one CTA scans all
// C centroids in FP32 and keeps a sorted top-kappa_c in shared memory.
__global__ void __launch_bounds__(M_THREADS)
k_topc_rescue(const float *__restrict__ rows, int nrows, const float *__restrict__ cent, int64_t C, int kc,
              const int32_t *__restrict__ lossy_rows, int32_t *__restrict__ top_ids,
              float *__restrict__ top_s) {
  const int r = blockIdx.x;
  if (r >= nrows || !lossy_rows[r]) return;
  __shared__ float s_q[DIM];
  __shared__ uint64_t best[1024];  // [0, 128): current top; [128, 128 + M_THREADS): new tile
  const int tid = threadIdx.x;
  for (int k = tid; k < DIM; k += M_THREADS) s_q[k] = rows[(int64_t)r * DIM + k];
  for (int i = tid; i < 1024; i += M_THREADS) best[i] = 0ull;
  __syncthreads();
  for (int64_t c0 = 0; c0 < C; c0 += M_THREADS) {
    int64_t c = c0 + tid;
    best[128 + tid] = (c < C) ? comp_key(dot_f32(s_q, cent + c * DIM), (int32_t)c) : 0ull;
    for (int i = 128 + M_THREADS + tid; i < 1024; i += M_THREADS) best[i] = 0ull;
    __syncthreads();
    block_sort_desc(best, 1024);
  }
  for (int i = tid; i < kc; i += M_THREADS) {
    uint64_t v = best[i];
    top_ids[(int64_t)r * kc + i] = v ? comp_id(v) : -1;
    top_s[(int64_t)r * kc + i] = v ? comp_score(v) : -INFINITY;
  }
}

tachiom_status launch_topc_merge(const Index &ix, const float *rows, int nrows, int kc, int splits,
                                 int capout, const uint64_t *split, const int32_t *split_cnt,
                                 const float *margins, int rescore, int32_t *top_ids, float *top_s,
                                 uint32_t *flags, cudaStream_t s) {
  if (nrows <= 0) return TACHIOM_OK;
  if (splits > 1024) return fail(TACHIOM_ERR_INVALID, "too many splits");
  TPROF("topc_merge", s);
  // per-row overflow marks live after the nrows x splits counters (the workspace
  // sizes split_cnt with nrows extra entries)
  int32_t *lossy = const_cast<int32_t *>(split_cnt) + (int64_t)nrows * splits;
  TCUDA(cudaMemsetAsync(lossy, 0, (size_t)nrows * 4, s));
  size_t smem = (size_t)M_MAX * 8;
  TCUDA(cudaFuncSetAttribute(k_topc_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_topc_merge<<<nrows, M_THREADS, smem, s>>>(rows, nrows, ix.cent_f32, ix.C, kc, splits, capout, split,
                                              split_cnt, margins, rescore, top_ids, top_s, flags, lossy);
  TLAUNCH();
  k_topc_rescue<<<nrows, M_THREADS, 0, s>>>(rows, nrows, ix.cent_f32, ix.C, kc, lossy, top_ids, top_s);
  TLAUNCH();
  return TACHIOM_OK;
}

tachiom_status launch_topc_rescue(const Index &ix, const float *rows, int nrows, int kc, const int32_t *lossy_rows,
                                  int32_t *top_ids, float *top_s, cudaStream_t s) {
  if (nrows <= 0) return TACHIOM_OK;
  TPROF("topc_rescue", s);
  k_topc_rescue<<<nrows, M_THREADS, 0, s>>>(rows, nrows, ix.cent_f32, ix.C, kc, lossy_rows, top_ids, top_s);
  TLAUNCH();
  return TACHIOM_OK;
}

// FP32 scores of given (row, centroid id) pairs (ids < 0 or >= C give -inf; ids >= C
// raise TACHIOM_FLAG_BAD_INPUT),
// each row's pairs then sorted by (score desc, id asc) as step (a) delivers them.
// One warp per row, kappa_c <= 128.
__global__ void __launch_bounds__(128)
k_score_pairs(const float *__restrict__ rows, int nrows, const float *__restrict__ cent, int64_t C,
              const int32_t *__restrict__ ids, int kc, int32_t *__restrict__ out_ids, float *__restrict__ out,
              uint32_t *__restrict__ flags) {
  __shared__ uint64_t keys[4][MAX_KC];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * 4 + warp;
  if (r >= nrows) return;
  const int np = next_pow2(max(kc, 2));
  for (int u = lane; u < np; u += 32) {
    uint64_t key = 0ull;
    if (u < kc) {
      const int32_t j = ids[(int64_t)r * kc + u];
      const bool ok = j >= 0 && j < C;
      if (j >= C) atomicOr(flags, TACHIOM_FLAG_BAD_INPUT);
      key = comp_key(ok ? dot_f32(rows + (int64_t)r * DIM, cent + (int64_t)j * DIM) : -INFINITY, ok ? j : -1);
    }
    keys[warp][u] = key;
  }
  __syncwarp();
  warp_sort_desc(keys[warp], np);
  for (int u = lane; u < kc; u += 32) {
    const uint64_t v = keys[warp][u];
    out_ids[(int64_t)r * kc + u] = comp_id(v);
    out[(int64_t)r * kc + u] = comp_score(v);
  }
}

tachiom_status launch_score_pairs(const Index &ix, const float *rows, int nrows, const int32_t *ids,
                                  int kc, int32_t *out_ids, float *scores, uint32_t *flags, cudaStream_t s) {
  if ((int64_t)nrows * kc <= 0) return TACHIOM_OK;
  TPROF("score_pairs", s);
  k_score_pairs<<<(unsigned)((nrows + 3) / 4), 128, 0, s>>>(rows, nrows, ix.cent_f32, ix.C, ids, kc, out_ids,
                                                            scores, flags);
  TLAUNCH();
  return TACHIOM_OK;
}

}  // namespace tachiom
