// Token-Aware Clustering on the GPU (Sec. 2.1, "Token-Aware Clustering"): the collection's
// vectors are grouped by token type, each type's spread s_j is measured, the centroid budget is
// shared out (tachiom_tac_allot, host), and every type is clustered on its own by Lloyd's
// kappa_j-means. Every type's subproblem only sees its own points and centroids, which is what
// makes the decomposition cheap (Sec. 2.1's speed-up bound).
//
// Layout and order (all deterministic, so a run repeats bit for bit):
//   - points are grouped by a stable radix sort on the type (within a type: collection order);
//   - sums run in compensated FP32 in a fixed order: warp w of a CTA takes the segment's elements
//     w, w + W, ..., lane l dims 4l .. 4l + 3, and the W warp partials are added in warp order;
//   - initial centroids of type j: its points at positions floor((r + 1/2) n_j / kappa_j),
//     r < kappa_j (evenly spaced, distinct since kappa_j <= n_j);
//   - a round: every point to the nearest centroid of its type (squared L2 in FP32, ties to the
//     lower centroid), then every centroid to the compensated FP32 mean of its members (a
//     centroid left without members keeps its place); after the last round, one more assignment
//     gives the labels;
//   - centroids are numbered type by type (type order), kappa_j each.
// The assignment of a type with many centroids (kappa_j >= 64 by default) is a dense product: its
// points (BF16, grouped order) times its centroids (BF16) on the tensor cores through a cuBLAS GEMM
// with FP32 accumulation, in row chunks; then per point the approximate best centroid, and every
// centroid whose approximate distance lies within a rigorous margin of it rescored with the FP32
// arithmetic of the small types' kernel. The margin covers the BF16 rounding of both operands and
// the FP32 rounding of both distance forms, so the rescored set holds every centroid whose FP32
// distance can be the minimum and the label is the one the FP32 kernel gives.
#include <cublas_v2.h>
#include <cub/cub.cuh>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <vector>

#include "tachiom_internal.cuh"

namespace tachiom {

namespace {

// device buffers of one call, freed on every return path
struct TacBufs {
  std::vector<void *> p;
  ~TacBufs() {
    for (void *x : p) cudaFree(x);
  }
  template <typename T>
  tachiom_status alloc(T **out, size_t n) {
    void *x = nullptr;
    const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
    const cudaError_t e = cudaMalloc(&x, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(TACHIOM_ERR_OOM, "tac_cluster: cudaMalloc of %zu bytes failed", bytes);
    }
    p.push_back(x);
    *out = static_cast<T *>(x);
    return TACHIOM_OK;
  }
};

// a cuBLAS handle bound to one stream, destroyed on every return path
struct Blas {
  cublasHandle_t h = nullptr;
  ~Blas() {
    if (h) cublasDestroy(h);
  }
};

constexpr int GEMM_MIN_KAPPA = 64;        // default: types with this many centroids take the GEMM path
constexpr int64_t GEMM_SCORES = 1 << 25;  // FP32 products one GEMM chunk may hold (128 MiB)

constexpr int TC_WARPS = 8;  // warps of the per-segment reduction CTAs

__global__ void k_tac_iota_check(const int32_t *__restrict__ types, int64_t n, int32_t n_types,
                                 int32_t *__restrict__ idx, uint32_t *__restrict__ bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    idx[i] = (int32_t)i;
    const int32_t t = types[i];
    if (t < 0 || t >= n_types) atomicOr(bad, 1u);
  }
}

__global__ void k_tac_iota(int32_t *__restrict__ idx, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    idx[i] = (int32_t)i;
}

// off[k] = first position of sorted keys[0, n) holding a key >= k, for k = 0 .. nk
__global__ void k_tac_bounds(const int32_t *__restrict__ keys, int64_t n, int64_t nk, int64_t *__restrict__ off) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= nk; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if ((int64_t)keys[mid] < k) lo = mid + 1;
      else hi = mid;
    }
    off[k] = lo;
  }
}

// Compensated FP32 addition (Neumaier): s + c carries the sum of the added values with an error of a
// few units in the last place of the sum, independent of how many values were added.
__device__ __forceinline__ void kadd(float &s, float &c, float x) {
  const float t = s + x;
  c += (fabsf(s) >= fabsf(x)) ? (s - t) + x : (x - t) + s;
  s = t;
}

// Mean of the vectors X[order[mem[e]]] for e in [b, e1) (mem may be null: identity) in compensated
// FP32, in a fixed order (warp w adds the members w, w + TC_WARPS, ...; the warps' sums are added in
// warp order), so a run repeats bit for bit; the CTA's TC_WARPS warps end with the mean in m[128]
__device__ void tac_segment_mean(const float *__restrict__ X, const int32_t *__restrict__ order,
                                 const int32_t *__restrict__ mem, int64_t b, int64_t e1, float2 (*red)[128],
                                 float *m) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
  for (int64_t q = b + warp; q < e1; q += TC_WARPS) {
    const int64_t p = mem ? (int64_t)mem[q] : q;
    const float4 v = *reinterpret_cast<const float4 *>(X + (int64_t)order[p] * DIM + 4 * lane);
    kadd(s0, c0, v.x);
    kadd(s1, c1, v.y);
    kadd(s2, c2, v.z);
    kadd(s3, c3, v.w);
  }
  red[warp][4 * lane] = make_float2(s0, c0);
  red[warp][4 * lane + 1] = make_float2(s1, c1);
  red[warp][4 * lane + 2] = make_float2(s2, c2);
  red[warp][4 * lane + 3] = make_float2(s3, c3);
  __syncthreads();
  if (threadIdx.x < DIM) {
    float t = 0.f, tc = 0.f;
    for (int w = 0; w < TC_WARPS; w++) {
      kadd(t, tc, red[w][threadIdx.x].x);
      kadd(t, tc, red[w][threadIdx.x].y);
    }
    m[threadIdx.x] = (t + tc) / (float)(e1 - b);
  }
  __syncthreads();
}

// s_j = (1 / n_j) sum ||x - mean_j||^2 over the type's points (0 for an absent type), compensated FP32
// in a fixed order
__global__ void __launch_bounds__(TC_WARPS * 32)
k_tac_type_spread(const float *__restrict__ X, const int32_t *__restrict__ order, const int64_t *__restrict__ off,
                  float *__restrict__ s) {
  __shared__ float2 red[TC_WARPS][128];
  __shared__ float mean[128];
  __shared__ float2 wacc[TC_WARPS];
  const int j = blockIdx.x;
  const int64_t b = off[j], e1 = off[j + 1];
  if (e1 == b) {
    if (threadIdx.x == 0) s[j] = 0.f;
    return;
  }
  tac_segment_mean(X, order, nullptr, b, e1, red, mean);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float m0 = mean[4 * lane], m1 = mean[4 * lane + 1], m2 = mean[4 * lane + 2], m3 = mean[4 * lane + 3];
  float q = 0.f, qc = 0.f;
  for (int64_t p = b + warp; p < e1; p += TC_WARPS) {
    const float4 v = *reinterpret_cast<const float4 *>(X + (int64_t)order[p] * DIM + 4 * lane);
    const float d0 = v.x - m0, d1 = v.y - m1, d2 = v.z - m2, d3 = v.w - m3;
    kadd(q, qc, fmaf(d3, d3, fmaf(d2, d2, fmaf(d1, d1, d0 * d0))));
  }
  // the lanes' compensated sums, added by a fixed butterfly
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oq = __shfl_xor_sync(0xffffffffu, q, o), oc = __shfl_xor_sync(0xffffffffu, qc, o);
    kadd(q, qc, oq);
    qc += oc;
  }
  if (lane == 0) wacc[warp] = make_float2(q, qc);
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f, tc = 0.f;
    for (int w = 0; w < TC_WARPS; w++) {
      kadd(t, tc, wacc[w].x);
      kadd(t, tc, wacc[w].y);
    }
    s[j] = (t + tc) / (float)(e1 - b);
  }
}

// initial centroid g (one warp each): point floor((r + 1/2) n_j / kappa_j) of its type j
__global__ void k_tac_init(const float *__restrict__ X, const int32_t *__restrict__ order,
                           const int64_t *__restrict__ off, const int32_t *__restrict__ ctype,
                           const int64_t *__restrict__ cbase, const int32_t *__restrict__ kappa, int64_t budget,
                           float *__restrict__ C) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t g = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); g < budget; g += nw) {
    const int32_t j = ctype[g];
    const int64_t r = g - cbase[j], nj = off[j + 1] - off[j];
    const int64_t pos = ((2 * r + 1) * nj) / (2 * (int64_t)kappa[j]);  // floor((r + 1/2) n_j / kappa_j), exact
    const float4 v = *reinterpret_cast<const float4 *>(X + (int64_t)order[off[j] + pos] * DIM + 4 * lane);
    *reinterpret_cast<float4 *>(C + g * DIM + 4 * lane) = v;
  }
}

// point p (grouped order, one warp each) to the nearest centroid of its type; -1 when the type
// has no centroid
__global__ void k_tac_assign(const float *__restrict__ X, const int32_t *__restrict__ order,
                             const int32_t *__restrict__ stype, int64_t n, const float *__restrict__ C,
                             const int64_t *__restrict__ cbase, const int32_t *__restrict__ kappa,
                             const uint8_t *__restrict__ gemm_type, int32_t *__restrict__ lab) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t p = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); p < n; p += nw) {
    const int32_t j = stype[p];
    if (gemm_type && gemm_type[j]) continue;  // assigned by the GEMM path
    const int64_t g0 = cbase[j], kj = kappa[j];
    const float4 x = *reinterpret_cast<const float4 *>(X + (int64_t)order[p] * DIM + 4 * lane);
    float best = INFINITY;
    int64_t bg = -1;
    for (int64_t g = g0; g < g0 + kj; g++) {
      const float4 c = *reinterpret_cast<const float4 *>(C + g * DIM + 4 * lane);
      const float e0 = x.x - c.x, e1 = x.y - c.y, e2 = x.z - c.z, e3 = x.w - c.w;
      float d = fmaf(e3, e3, fmaf(e2, e2, fmaf(e1, e1, e0 * e0)));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      if (d < best || bg < 0) {
        best = d;
        bg = g;
      }
    }
    if (lane == 0) lab[p] = (int32_t)bg;
  }
}

// grouped-order BF16 copy of the points and their norms (one warp per point, lane l dims 4l .. 4l + 3)
__global__ void k_tac_points_bf16(const float *__restrict__ X, const int32_t *__restrict__ order, int64_t n,
                                  __nv_bfloat16 *__restrict__ Xb, float *__restrict__ xn) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t p = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); p < n; p += nw) {
    const float4 x = *reinterpret_cast<const float4 *>(X + (int64_t)order[p] * DIM + 4 * lane);
    __nv_bfloat162 *d = reinterpret_cast<__nv_bfloat162 *>(Xb + p * DIM + 4 * lane);
    d[0] = __floats2bfloat162_rn(x.x, x.y);
    d[1] = __floats2bfloat162_rn(x.z, x.w);
    float q = fmaf(x.w, x.w, fmaf(x.z, x.z, fmaf(x.y, x.y, x.x * x.x)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if (lane == 0) xn[p] = sqrtf(q);
  }
}

// per centroid: its BF16 copy, its squared norm (FP32), and the largest norm of every type
__global__ void k_tac_cent_prep(const float *__restrict__ C, int64_t budget, const int32_t *__restrict__ ctype,
                                __nv_bfloat16 *__restrict__ Cb, float *__restrict__ cn2,
                                unsigned *__restrict__ cmax_type) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t g = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); g < budget; g += nw) {
    const float4 c = *reinterpret_cast<const float4 *>(C + g * DIM + 4 * lane);
    __nv_bfloat162 *d = reinterpret_cast<__nv_bfloat162 *>(Cb + g * DIM + 4 * lane);
    d[0] = __floats2bfloat162_rn(c.x, c.y);
    d[1] = __floats2bfloat162_rn(c.z, c.w);
    float q = fmaf(c.w, c.w, fmaf(c.z, c.z, fmaf(c.y, c.y, c.x * c.x)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if (lane == 0) {
      cn2[g] = q;
      atomicMax(cmax_type + ctype[g], __float_as_uint(sqrtf(q)));  // non-negative floats order as uints
    }
  }
}

// Points [p0, p0 + R) of type j (grouped order) against its k centroids g0 ..: S [R][k] holds the
// BF16 products <x^, c^>. One warp per point: the approximate best d~ = ||c||^2 - 2 <x^, c^>, then
// every centroid with d~ <= best + margin rescored with k_tac_assign's FP32 arithmetic, in ascending
// order with ties to the lower centroid. Margin: |<x^, c^> - <x, c>| <= 2^-8 ||x|| ||c|| (the BF16
// rounding of both operands) plus the FP32 accumulation, taken as 2^-6 ||x|| cmax_j; the FP32 forms
// of ||c||^2 and of the distance add at most 2^-16 (||x||^2 + cmax_j^2), taken as 2^-14 (...). With
// delta and e these, every centroid whose FP32 distance can be the minimum has d~ <= best + 4 delta
// + 2 e.
__global__ void k_tac_assign_gemm(const float *__restrict__ X, const int32_t *__restrict__ order, int64_t p0,
                                  int R, const float *__restrict__ S, int k, int64_t g0,
                                  const float *__restrict__ C, const float *__restrict__ cn2,
                                  const float *__restrict__ xn, const unsigned *__restrict__ cmax_type, int32_t j,
                                  int32_t *__restrict__ lab) {
  const int lane = threadIdx.x & 31;
  const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (q >= R) return;
  const int64_t p = p0 + q;
  const float *sp = S + (int64_t)q * k;
  float best = INFINITY;
  for (int g = lane; g < k; g += 32) best = fminf(best, fmaf(-2.f, sp[g], cn2[g0 + g]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = fminf(best, __shfl_xor_sync(0xffffffffu, best, o));
  const float xnorm = xn[p], cm = __uint_as_float(cmax_type[j]);
  const float delta = ldexpf(xnorm * cm, -6);
  const float e = ldexpf(fmaf(xnorm, xnorm, cm * cm), -14);
  const float thr = best + 4.f * delta + 2.f * e;
  const float4 x = *reinterpret_cast<const float4 *>(X + (int64_t)order[p] * DIM + 4 * lane);
  float bd = INFINITY;
  int64_t bg = -1;
  for (int b0 = 0; b0 < k; b0 += 32) {
    const int g = b0 + lane;
    const bool cand = g < k && !(fmaf(-2.f, sp[g], cn2[g0 + g]) > thr);
    unsigned m = __ballot_sync(0xffffffffu, cand);
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1u;
      const int64_t gg = g0 + b0 + b;
      const float4 c = *reinterpret_cast<const float4 *>(C + gg * DIM + 4 * lane);
      const float e0 = x.x - c.x, e1 = x.y - c.y, e2 = x.z - c.z, e3 = x.w - c.w;
      float d = fmaf(e3, e3, fmaf(e2, e2, fmaf(e1, e1, e0 * e0)));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      if (d < bd || bg < 0) {
        bd = d;
        bg = gg;
      }
    }
  }
  if (lane == 0) lab[p] = (int32_t)bg;
}

// centroid g (one CTA each) to the compensated FP32 mean of its members; no member: unchanged
__global__ void __launch_bounds__(TC_WARPS * 32)
k_tac_means(const float *__restrict__ X, const int32_t *__restrict__ order, const int32_t *__restrict__ mem,
            const int64_t *__restrict__ moff, float *__restrict__ C) {
  __shared__ float2 red[TC_WARPS][128];
  __shared__ float mean[128];
  const int64_t g = blockIdx.x;
  const int64_t b = moff[g], e1 = moff[g + 1];
  if (e1 == b) return;
  tac_segment_mean(X, order, mem, b, e1, red, mean);
  if (threadIdx.x < DIM) C[g * DIM + threadIdx.x] = mean[threadIdx.x];
}

__global__ void k_tac_scatter(const int32_t *__restrict__ lab, const int32_t *__restrict__ order, int64_t n,
                              int32_t *__restrict__ out) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    out[order[p]] = lab[p];
}

unsigned grid_for(int64_t items, int per_block) {
  const int64_t b = (items + per_block - 1) / per_block;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 148 * 64));
}

}  // namespace

}  // namespace tachiom

using namespace tachiom;

extern "C" tachiom_status tachiom_tac_cluster(const float *d_vectors, const int32_t *d_types, int64_t n_vectors,
                                              int32_t n_types, int64_t budget, const tachiom_tac_params *p,
                                              int32_t iters, int32_t *h_kappa, double *h_spread,
                                              float *d_centroids, int32_t *d_centroid_type, int32_t *d_labels,
                                              void *stream) {
  if (!p || !h_kappa || n_types <= 0 || n_vectors < 0 || n_vectors >= INT32_MAX || iters < 0 || budget < 0)
    return fail(TACHIOM_ERR_INVALID, "tac_cluster: bad argument (null params or kappa, n_types <= 0, "
                                     "n_vectors outside [0, 2^31 - 1), iters or budget < 0)");
  if (n_vectors > 0 && (!d_vectors || !d_types || !d_labels))
    return fail(TACHIOM_ERR_INVALID, "tac_cluster: NULL vectors, types or labels");
  if (budget > 0 && (!d_centroids || !d_centroid_type))
    return fail(TACHIOM_ERR_INVALID, "tac_cluster: NULL centroid outputs");
  if (((uintptr_t)d_vectors & 15u) || ((uintptr_t)d_centroids & 15u))
    return fail(TACHIOM_ERR_INVALID, "tac_cluster: vectors and centroids must be 16-byte aligned");
  if (budget >= INT32_MAX) return fail(TACHIOM_ERR_INVALID, "tac_cluster: budget must be below 2^31 - 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t N = n_vectors;
  TacBufs B;
  tachiom_status st;
#define TTRY(x)           \
  do {                    \
    if ((st = (x))) return st; \
  } while (0)
  int32_t *idx, *stype, *order, *lab, *labs, *mem, *kap_d;
  int64_t *off, *cbase_d, *moff;
  float *spr;
  uint32_t *bad;
  TTRY(B.alloc(&idx, (size_t)N));
  TTRY(B.alloc(&stype, (size_t)N));
  TTRY(B.alloc(&order, (size_t)N));
  TTRY(B.alloc(&lab, (size_t)N));
  TTRY(B.alloc(&labs, (size_t)N));
  TTRY(B.alloc(&mem, (size_t)N));
  TTRY(B.alloc(&off, (size_t)n_types + 1));
  TTRY(B.alloc(&spr, (size_t)n_types));
  TTRY(B.alloc(&kap_d, (size_t)n_types));
  TTRY(B.alloc(&cbase_d, (size_t)n_types));
  TTRY(B.alloc(&moff, (size_t)budget + 1));
  TTRY(B.alloc(&bad, 1));
  // the radix sorts' scratch: the larger of the two sorts (both N int32 pairs)
  size_t tmp_bytes = 0;
  TCUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, idx, stype, idx, order, (int)N, 0, 32, s));
  void *tmp = nullptr;
  TTRY(B.alloc(reinterpret_cast<unsigned char **>(&tmp), tmp_bytes));

  // 1. group by type (stable), type bounds, spreads
  TCUDA(cudaMemsetAsync(bad, 0, sizeof(uint32_t), s));
  if (N > 0) {
    k_tac_iota_check<<<grid_for(N, 256), 256, 0, s>>>(d_types, N, n_types, idx, bad);
    TLAUNCH();
    TCUDA(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, d_types, stype, idx, order, (int)N, 0, 32, s));
  }
  k_tac_bounds<<<grid_for((int64_t)n_types + 1, 256), 256, 0, s>>>(stype, N, n_types, off);
  TLAUNCH();
  k_tac_type_spread<<<n_types, TC_WARPS * 32, 0, s>>>(d_vectors, order, off, spr);
  TLAUNCH();
  std::vector<int64_t> hoff((size_t)n_types + 1);
  std::vector<float> hsf((size_t)n_types);
  std::vector<double> hs((size_t)n_types);
  uint32_t hbad = 0;
  TCUDA(cudaMemcpyAsync(hoff.data(), off, hoff.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TCUDA(cudaMemcpyAsync(hsf.data(), spr, hsf.size() * sizeof(float), cudaMemcpyDeviceToHost, s));
  TCUDA(cudaMemcpyAsync(&hbad, bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  TCUDA(cudaStreamSynchronize(s));
  if (hbad) return fail(TACHIOM_ERR_INVALID, "tac_cluster: a token type is outside [0, n_types)");
  for (int32_t j = 0; j < n_types; j++) hs[j] = (double)hsf[j];
  if (h_spread) std::copy(hs.begin(), hs.end(), h_spread);

  // 2. the allotment (host), the centroid numbering
  std::vector<int64_t> hn((size_t)n_types);
  for (int32_t j = 0; j < n_types; j++) hn[j] = hoff[j + 1] - hoff[j];
  TTRY(tachiom_tac_allot(hn.data(), hs.data(), n_types, budget, p, h_kappa));
  std::vector<int64_t> hcb((size_t)n_types);
  std::vector<int32_t> hct((size_t)budget);
  int64_t acc = 0;
  for (int32_t j = 0; j < n_types; j++) {
    hcb[j] = acc;
    for (int32_t r = 0; r < h_kappa[j]; r++) hct[(size_t)(acc + r)] = j;
    acc += h_kappa[j];
  }
  if (budget > 0)
    TCUDA(cudaMemcpyAsync(d_centroid_type, hct.data(), hct.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  TCUDA(cudaMemcpyAsync(cbase_d, hcb.data(), hcb.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  TCUDA(cudaMemcpyAsync(kap_d, h_kappa, (size_t)n_types * sizeof(int32_t), cudaMemcpyHostToDevice, s));

  // 3. initial centroids, Lloyd rounds, the final assignment
  if (budget > 0) {
    k_tac_init<<<grid_for(budget, 8), 256, 0, s>>>(d_vectors, order, off, d_centroid_type, cbase_d, kap_d, budget,
                                                    d_centroids);
    TLAUNCH();
  }
  // the types assigned through the GEMM path, and its buffers
  const int32_t kmin = p->gemm_min_kappa == 0 ? GEMM_MIN_KAPPA : p->gemm_min_kappa;
  std::vector<int32_t> gtypes;
  std::vector<uint8_t> hgemm((size_t)n_types, 0);
  if (kmin > 0)
    for (int32_t j = 0; j < n_types; j++)
      if (h_kappa[j] >= kmin && hn[j] > 0) {
        gtypes.push_back(j);
        hgemm[(size_t)j] = 1;
      }
  uint8_t *gemm_d = nullptr;
  __nv_bfloat16 *Xb = nullptr, *Cb = nullptr;
  float *xn = nullptr, *cn2 = nullptr, *S = nullptr;
  unsigned *cmax_t = nullptr;
  Blas blas;
  if (!gtypes.empty()) {
    // best effort: without room for the BF16 copies every type takes the CUDA-core kernel
    TacBufs G;
    if (G.alloc(&gemm_d, (size_t)n_types) || G.alloc(&Xb, (size_t)N * DIM) || G.alloc(&xn, (size_t)N) ||
        G.alloc(&Cb, (size_t)budget * DIM) || G.alloc(&cn2, (size_t)budget) ||
        G.alloc(&cmax_t, (size_t)n_types) || G.alloc(&S, (size_t)GEMM_SCORES)) {
      gtypes.clear();  // G frees what it got
      gemm_d = nullptr;
    } else {
      B.p.insert(B.p.end(), G.p.begin(), G.p.end());  // owned by the call's buffers from here
      G.p.clear();
    }
  }
  if (!gtypes.empty()) {
    TCUDA(cudaMemcpyAsync(gemm_d, hgemm.data(), hgemm.size(), cudaMemcpyHostToDevice, s));
    k_tac_points_bf16<<<grid_for(N, 8), 256, 0, s>>>(d_vectors, order, N, Xb, xn);
    TLAUNCH();
    if (cublasCreate(&blas.h) != CUBLAS_STATUS_SUCCESS) {
      blas.h = nullptr;
      return fail(TACHIOM_ERR_CUDA, "tac_cluster: cublasCreate failed");
    }
    if (cublasSetStream(blas.h, s) != CUBLAS_STATUS_SUCCESS)
      return fail(TACHIOM_ERR_CUDA, "tac_cluster: cublasSetStream failed");
  }
  // every point of a GEMM-path type: S = X_j C_j^T in row chunks (column-major k_j x rows, so a
  // point's k_j products are contiguous), then the margin rescoring
  auto assign_gemm = [&]() -> tachiom_status {
    TCUDA(cudaMemsetAsync(cmax_t, 0, (size_t)n_types * sizeof(unsigned), s));
    k_tac_cent_prep<<<grid_for(budget, 8), 256, 0, s>>>(d_centroids, budget, d_centroid_type, Cb, cn2, cmax_t);
    TLAUNCH();
    const float one = 1.f, zero = 0.f;
    for (int32_t j : gtypes) {
      const int k = h_kappa[j];
      const int64_t rows_max = std::max<int64_t>(1, GEMM_SCORES / k);
      for (int64_t a0 = hoff[j]; a0 < hoff[j + 1]; a0 += rows_max) {
        const int R = (int)std::min<int64_t>(rows_max, hoff[j + 1] - a0);
        const cublasStatus_t cs =
            cublasGemmEx(blas.h, CUBLAS_OP_T, CUBLAS_OP_N, k, R, DIM, &one, Cb + hcb[j] * DIM, CUDA_R_16BF, DIM,
                         Xb + a0 * DIM, CUDA_R_16BF, DIM, &zero, S, CUDA_R_32F, k, CUBLAS_COMPUTE_32F,
                         CUBLAS_GEMM_DEFAULT);
        if (cs != CUBLAS_STATUS_SUCCESS) return fail(TACHIOM_ERR_CUDA, "tac_cluster: cublasGemmEx failed (%d)", (int)cs);
        k_tac_assign_gemm<<<(R + 7) / 8, 256, 0, s>>>(d_vectors, order, a0, R, S, k, hcb[j], d_centroids, cn2, xn,
                                                      cmax_t, j, lab);
        TLAUNCH();
      }
    }
    return TACHIOM_OK;
  };
  for (int32_t it = 0; it <= iters; it++) {
    if (N > 0) {
      if (!gtypes.empty()) TTRY(assign_gemm());
      k_tac_assign<<<grid_for(N, 8), 256, 0, s>>>(d_vectors, order, stype, N, d_centroids, cbase_d, kap_d, gemm_d,
                                                   lab);
      TLAUNCH();
    }
    if (it == iters || N == 0 || budget == 0) break;
    // members of every centroid in grouped order: a stable sort of (label, position)
    k_tac_iota<<<grid_for(N, 256), 256, 0, s>>>(idx, N);
    TLAUNCH();
    TCUDA(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, lab, labs, idx, mem, (int)N, 0, 32, s));
    k_tac_bounds<<<grid_for(budget + 1, 256), 256, 0, s>>>(labs, N, budget, moff);
    TLAUNCH();
    k_tac_means<<<(unsigned)budget, TC_WARPS * 32, 0, s>>>(d_vectors, order, mem, moff, d_centroids);
    TLAUNCH();
  }
  if (N > 0) {
    k_tac_scatter<<<grid_for(N, 256), 256, 0, s>>>(lab, order, N, d_labels);
    TLAUNCH();
  }
  TCUDA(cudaStreamSynchronize(s));
#undef TTRY
  return TACHIOM_OK;
}

// ---- residual compression (Sec. 2.1, "Residuals Compression") ----------------------------------
// Vector i with centroid c = C[label_i]: r = x - c, rho = ||r||, u = r / rho split into M contiguous
// subspaces of ds = 128 / M dims, each coded by its nearest codeword (squared L2 in FP32, ties to
// the lower code); rho is stored rounded to fp16. A zero residual, or a vector without a centroid
// (label < 0), gets rho = 0 and code 0 everywhere. One warp per vector, lane l on dims 4l .. 4l + 3;
// the codebook sits in shared memory code-major (codeword j of every subspace along the 128 dims),
// so the 32 lanes read 512 consecutive bytes per codeword.
namespace tachiom {
namespace {

constexpr int PQ_WARPS = 8;

// stage the codebook [M][256][DS] into shared memory code-major ([256][128]); all threads
template <int M>
__device__ __forceinline__ void pq_stage(const float *__restrict__ codebooks, float *cbs) {
  constexpr int DS = DIM / M;
  for (int x = threadIdx.x; x < 256 * DIM; x += blockDim.x) {
    const int j = x / DIM, d = x % DIM, m = d / DS, u = d % DS;
    cbs[x] = codebooks[((int64_t)m * 256 + j) * DS + u];
  }
}

// nearest codeword (squared L2 in FP32, ties to the lower code) of this lane's subspace for the
// unit vector whose dims 4 lane .. 4 lane + 3 are u; every lane of the subspace gets the answer
template <int M>
__device__ __forceinline__ int pq_nearest(const float4 u, const float *cbs, int lane) {
  constexpr int G = DIM / M / 4;  // lanes per subspace
  float best = INFINITY;
  int best_j = 0;
  for (int j = 0; j < 256; j++) {
    const float4 w = *reinterpret_cast<const float4 *>(cbs + j * DIM + 4 * lane);
    const float e0 = u.x - w.x, e1 = u.y - w.y, e2 = u.z - w.z, e3 = u.w - w.w;
    float d = fmaf(e3, e3, fmaf(e2, e2, fmaf(e1, e1, e0 * e0)));
#pragma unroll
    for (int o = 1; o < G; o <<= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (d < best) {
      best = d;
      best_j = j;
    }
  }
  return best_j;
}

// vector i's residual from its centroid (zero for a label < 0), this lane's 4 dims, and its norm
__device__ __forceinline__ float4 pq_residual(const float *__restrict__ X, const float *__restrict__ C, int32_t l,
                                              int64_t i, int lane, float &rho) {
  float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
  if (l >= 0) {
    const float4 x = *reinterpret_cast<const float4 *>(X + i * DIM + 4 * lane);
    const float4 c = *reinterpret_cast<const float4 *>(C + (int64_t)l * DIM + 4 * lane);
    r = make_float4(x.x - c.x, x.y - c.y, x.z - c.z, x.w - c.w);
  }
  float rr = fmaf(r.w, r.w, fmaf(r.z, r.z, fmaf(r.y, r.y, r.x * r.x)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) rr += __shfl_xor_sync(0xffffffffu, rr, o);
  rho = sqrtf(rr);
  return r;
}

template <int M>
__global__ void __launch_bounds__(PQ_WARPS * 32)
k_pq_encode(const float *__restrict__ X, const float *__restrict__ C, const int32_t *__restrict__ labels, int64_t n,
            const float *__restrict__ codebooks, uint8_t *__restrict__ codes, uint16_t *__restrict__ rnorm) {
  constexpr int G = DIM / M / 4;  // lanes per subspace
  extern __shared__ __align__(16) float cbs[];  // [256][128]
  pq_stage<M>(codebooks, cbs);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * PQ_WARPS;
  for (int64_t i = blockIdx.x * (int64_t)PQ_WARPS + (threadIdx.x >> 5); i < n; i += nw) {
    float rho;
    const float4 r = pq_residual(X, C, labels[i], i, lane, rho);
    int best_j = 0;
    if (rho > 0.f) best_j = pq_nearest<M>(make_float4(r.x / rho, r.y / rho, r.z / rho, r.w / rho), cbs, lane);
    if ((lane % G) == 0) codes[i * M + lane / G] = (uint8_t)best_j;
    if (lane == 0) rnorm[i] = __half_as_ushort(__float2half_rn(rho));
  }
}

// codebook training, sample r (one warp each): the normalised residual of vector
// floor((r + 1/2) n / S), the zero vector for a zero residual or a label < 0
__global__ void k_pq_sample(const float *__restrict__ X, const float *__restrict__ C,
                            const int32_t *__restrict__ labels, int64_t n, int32_t S, float *__restrict__ U) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < S; r += nw) {
    const int64_t i = ((2 * (int64_t)r + 1) * n) / (2 * (int64_t)S);  // floor((r + 1/2) n / S), exact
    float rho;
    const float4 v = pq_residual(X, C, labels[i], i, lane, rho);
    const float4 u = rho > 0.f ? make_float4(v.x / rho, v.y / rho, v.z / rho, v.w / rho) : make_float4(0.f, 0.f, 0.f, 0.f);
    *reinterpret_cast<float4 *>(U + r * DIM + 4 * lane) = u;
  }
}

// initial codeword (m, j): sub-vector m of sample point floor((j + 1/2) S / 256)
template <int M>
__global__ void k_pq_init(const float *__restrict__ U, int32_t S, float *__restrict__ books) {
  constexpr int DS = DIM / M;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < M * 256 * DS; x += gridDim.x * blockDim.x) {
    const int m = x / (256 * DS), j = (x / DS) % 256, u = x % DS;
    const int64_t p = ((2 * (int64_t)j + 1) * S) / 512;  // floor((j + 1/2) S / 256), exact
    books[x] = U[p * DIM + m * DS + u];
  }
}

// sample s (one warp each) to its nearest codeword of every subspace: key m * 256 + code at
// [m * S + s], value s
template <int M>
__global__ void __launch_bounds__(PQ_WARPS * 32)
k_pq_assign_unit(const float *__restrict__ U, int32_t S, const float *__restrict__ books, int32_t *__restrict__ keys,
                 int32_t *__restrict__ vals) {
  constexpr int G = DIM / M / 4;
  extern __shared__ __align__(16) float cbs[];
  pq_stage<M>(books, cbs);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * PQ_WARPS;
  for (int64_t s = blockIdx.x * (int64_t)PQ_WARPS + (threadIdx.x >> 5); s < S; s += nw) {
    const float4 u = *reinterpret_cast<const float4 *>(U + s * DIM + 4 * lane);
    const int j = pq_nearest<M>(u, cbs, lane);
    if ((lane % G) == 0) {
      const int m = lane / G;
      keys[(int64_t)m * S + s] = m * 256 + j;
      vals[(int64_t)m * S + s] = (int32_t)s;
    }
  }
}

// codeword k = m * 256 + j (one warp each) to the compensated FP32 mean of its members' sub-vectors m
// (lane l sums members l, l + 32, ...; the lanes are added by a fixed butterfly); a codeword without
// members keeps its place
template <int M>
__global__ void k_pq_means(const float *__restrict__ U, const int32_t *__restrict__ vals,
                           const int64_t *__restrict__ off, float *__restrict__ books) {
  constexpr int DS = DIM / M;
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t k = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); k < M * 256; k += nw) {
    const int64_t b = off[k], e1 = off[k + 1];
    if (b == e1) continue;
    const int m = (int)(k / 256);
    float acc[DS], cmp[DS];
#pragma unroll
    for (int u = 0; u < DS; u++) acc[u] = cmp[u] = 0.f;
    for (int64_t q = b + lane; q < e1; q += 32) {
      const float *src = U + (int64_t)vals[q] * DIM + m * DS;
#pragma unroll
      for (int u = 0; u < DS; u++) kadd(acc[u], cmp[u], src[u]);
    }
#pragma unroll
    for (int u = 0; u < DS; u++) {
      float t = acc[u], tc = cmp[u];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ot = __shfl_xor_sync(0xffffffffu, t, o), oc = __shfl_xor_sync(0xffffffffu, tc, o);
        kadd(t, tc, ot);
        tc += oc;
      }
      if (lane == 0) books[k * DS + u] = (t + tc) / (float)(e1 - b);
    }
  }
}

}  // namespace
}  // namespace tachiom

extern "C" tachiom_status tachiom_pq_encode(const float *d_vectors, const float *d_centroids, const int32_t *d_labels,
                                            int64_t n_vectors, const float *d_codebooks, int32_t pq_m,
                                            uint8_t *d_codes, uint16_t *d_rnorm, void *stream) {
  using namespace tachiom;
  if (n_vectors < 0 || (pq_m != 8 && pq_m != 16 && pq_m != 32))
    return fail(TACHIOM_ERR_INVALID, "pq_encode: n_vectors < 0 or pq_m not in {8, 16, 32}");
  if (n_vectors == 0) return TACHIOM_OK;
  if (!d_vectors || !d_centroids || !d_labels || !d_codebooks || !d_codes || !d_rnorm)
    return fail(TACHIOM_ERR_INVALID, "pq_encode: NULL argument");
  if (((uintptr_t)d_vectors & 15u) || ((uintptr_t)d_centroids & 15u))
    return fail(TACHIOM_ERR_INVALID, "pq_encode: vectors and centroids must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t smem = 256 * DIM * sizeof(float);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n_vectors + PQ_WARPS - 1) / PQ_WARPS;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms));
  switch (pq_m) {
    case 8:
      TCUDA(cudaFuncSetAttribute(k_pq_encode<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_pq_encode<8><<<grid, PQ_WARPS * 32, smem, s>>>(d_vectors, d_centroids, d_labels, n_vectors, d_codebooks,
                                                       d_codes, d_rnorm);
      break;
    case 16:
      TCUDA(cudaFuncSetAttribute(k_pq_encode<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_pq_encode<16><<<grid, PQ_WARPS * 32, smem, s>>>(d_vectors, d_centroids, d_labels, n_vectors, d_codebooks,
                                                        d_codes, d_rnorm);
      break;
    default:
      TCUDA(cudaFuncSetAttribute(k_pq_encode<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_pq_encode<32><<<grid, PQ_WARPS * 32, smem, s>>>(d_vectors, d_centroids, d_labels, n_vectors, d_codebooks,
                                                        d_codes, d_rnorm);
      break;
  }
  TLAUNCH();
  return TACHIOM_OK;
}

namespace {
template <int M>
tachiom_status pq_train_m(const float *X, const float *C, const int32_t *labels, int64_t n, int32_t S, int32_t iters,
                          float *books, cudaStream_t s) {
  using namespace tachiom;
  TacBufs B;
  tachiom_status st;
  float *U;
  int32_t *keys, *vals, *keys_s, *vals_s;
  int64_t *off;
  const int64_t nk = (int64_t)M * S;
  if ((st = B.alloc(&U, (size_t)S * DIM))) return st;
  if ((st = B.alloc(&keys, (size_t)nk))) return st;
  if ((st = B.alloc(&vals, (size_t)nk))) return st;
  if ((st = B.alloc(&keys_s, (size_t)nk))) return st;
  if ((st = B.alloc(&vals_s, (size_t)nk))) return st;
  if ((st = B.alloc(&off, (size_t)M * 256 + 1))) return st;
  size_t tmp_bytes = 0;
  TCUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, keys, keys_s, vals, vals_s, (int)nk, 0, 32, s));
  unsigned char *tmp;
  if ((st = B.alloc(&tmp, tmp_bytes))) return st;
  const size_t smem = 256 * DIM * sizeof(float);
  TCUDA(cudaFuncSetAttribute(k_pq_assign_unit<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_pq_sample<<<grid_for(S, 8), 256, 0, s>>>(X, C, labels, n, S, U);
  TLAUNCH();
  k_pq_init<M><<<grid_for((int64_t)M * 256 * (DIM / M), 256), 256, 0, s>>>(U, S, books);
  TLAUNCH();
  for (int32_t it = 0; it < iters; it++) {
    k_pq_assign_unit<M><<<grid_for(S, PQ_WARPS), PQ_WARPS * 32, smem, s>>>(U, S, books, keys, vals);
    TLAUNCH();
    TCUDA(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, keys, keys_s, vals, vals_s, (int)nk, 0, 32, s));
    k_tac_bounds<<<grid_for((int64_t)M * 256 + 1, 256), 256, 0, s>>>(keys_s, nk, (int64_t)M * 256, off);
    TLAUNCH();
    k_pq_means<M><<<grid_for((int64_t)M * 256, 8), 256, 0, s>>>(U, vals_s, off, books);
    TLAUNCH();
  }
  TCUDA(cudaStreamSynchronize(s));
  return TACHIOM_OK;
}
}  // namespace

extern "C" tachiom_status tachiom_pq_train(const float *d_vectors, const float *d_centroids, const int32_t *d_labels,
                                           int64_t n_vectors, int32_t pq_m, int32_t sample, int32_t iters,
                                           float *d_codebooks, void *stream) {
  using namespace tachiom;
  if (pq_m != 8 && pq_m != 16 && pq_m != 32)
    return fail(TACHIOM_ERR_INVALID, "pq_train: pq_m must be 8, 16 or 32");
  if (sample < 256 || sample > n_vectors || iters < 0 || (int64_t)sample * pq_m >= INT32_MAX)
    return fail(TACHIOM_ERR_INVALID, "pq_train: need 256 <= sample <= n_vectors, sample * pq_m < 2^31, iters >= 0");
  if (!d_vectors || !d_centroids || !d_labels || !d_codebooks)
    return fail(TACHIOM_ERR_INVALID, "pq_train: NULL argument");
  if (((uintptr_t)d_vectors & 15u) || ((uintptr_t)d_centroids & 15u))
    return fail(TACHIOM_ERR_INVALID, "pq_train: vectors and centroids must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (pq_m) {
    case 8: return pq_train_m<8>(d_vectors, d_centroids, d_labels, n_vectors, sample, iters, d_codebooks, s);
    case 16: return pq_train_m<16>(d_vectors, d_centroids, d_labels, n_vectors, sample, iters, d_codebooks, s);
    default: return pq_train_m<32>(d_vectors, d_centroids, d_labels, n_vectors, sample, iters, d_codebooks, s);
  }
}
