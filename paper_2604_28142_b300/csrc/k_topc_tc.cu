// Step (a) on the 5th-generation tensor cores: BF16 products, FP32 accumulation
// (Sec. 2.2, Gather step 1 in exhaustive form), with a rigorous FP32 repair.
//
// GEMM orientation: a tcgen05.mma tile is M = 128 centroids (TMEM lanes) by
// N = 256 query rows (TMEM columns) by K = 128. The CTA keeps its 256 query
// rows resident in shared memory (64 KB, loaded once by TMA) and streams
// 128-centroid tiles (32 KB) through a 4-stage TMA/mbarrier ring. Two
// 256-column FP32 accumulators (all 512 TMEM columns) let the MMA of tile t+1
// run while 8 epilogue warps drain tile t with tcgen05.ld. Warp roles: warp 0
// issues TMA, warp 1 owns TMEM and issues the MMAs, warps 2..9 are the
// epilogue (warp w reads TMEM lanes 32*(w%4).., column half (w-2)/4).
//
// Selection without any per-row state in the GEMM:
//   pass    every group of 32 consecutive centroids reports, per query row, its
//           maximum approximate score (one redux.sync per column) -> gmax;
//   select  tau'_r = a lower bound on the row's kappa_c-th largest group maximum
//           (two histogram levels, the second inside the bin the first finds);
//           every group whose maximum is >= tau'_r - margin_r is kept. A centroid of the row's exact FP32 top-kappa_c has
//           an approximate score >= (approximate kappa_c-th best) - 2 delta_r
//           >= tau'_r - margin_r (margin_r = 2 delta_r), so its group is kept:
//           about kappa_c groups per row survive;
//   rescore the centroids of the kept groups are scored exactly in FP32 (the
//           same fmaf chain as the FP32 path) and the exact top-kappa_c is kept.
// A row whose kept groups do not fit is recomputed by a full FP32 scan.
//
// Every wait on an mbarrier is bounded by %globaltimer; a wait that runs out
// raises TACHIOM_FLAG_TIMEOUT, every role leaves its loop, in-flight copies
// and MMAs are drained (again with a bound) and TMEM is freed before exit.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "tc_common.cuh"

namespace tachiom {

namespace tc {

constexpr int BM = 128;            // centroids per tile (MMA M)
constexpr int BN = 256;            // query rows per CTA (MMA N)
constexpr int KH = 64;             // K elements per 128-byte swizzled half
constexpr int STAGES = 4;
constexpr int A_HALF = BM * KH * 2;        // 16 KB
constexpr int A_STAGE = 2 * A_HALF;        // 32 KB
constexpr int B_HALF = BN * KH * 2;        // 32 KB
constexpr int B_BYTES = 2 * B_HALF;        // 64 KB
constexpr int TILE_BYTES = B_BYTES + STAGES * A_STAGE;  // 192 KB
constexpr int THREADS = 320;       // 10 warps
constexpr int EPI_WARPS = 8;
constexpr int TMEM_COLS = 512;

struct Ctl {
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t bfull;
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
};
constexpr int SMEM_BYTES = TILE_BYTES + (int)sizeof(Ctl) + 1024;

// MODE 1: maximum per group of 32 centroids -> (float) gmax[rb][tile * 4 + quarter][256]
// MODE 3: raw scores to (float *)cand [R x C] (diagnostics and tests)
template <int MODE>
__global__ void __launch_bounds__(THREADS, 1)
k_topc_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t C, int R,
          int ntiles, int tiles_per_split, int G, uint32_t *__restrict__ gmax, uint64_t *__restrict__ cand,
          uint32_t *__restrict__ flags) {
  extern __shared__ __align__(1024) unsigned char tsm_raw[];
  unsigned char *tsm = (unsigned char *)(((uintptr_t)tsm_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *Bs = tsm;                  // [2 halves][256 rows][128 B]
  unsigned char *As = tsm + B_BYTES;        // [STAGES][2 halves][128 rows][128 B]
  Ctl *ctl = reinterpret_cast<Ctl *>(tsm + TILE_BYTES);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rb = blockIdx.y;
  const int t0 = blockIdx.x * tiles_per_split;
  const int t1 = min(ntiles, t0 + tiles_per_split);
  const int nt = max(0, t1 - t0);
  volatile int *abort = &ctl->abort;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; s++) {
      mbar_init(&ctl->full[s], 1);
      mbar_init(&ctl->empty[s], 1);
    }
    for (int b = 0; b < 2; b++) {
      mbar_init(&ctl->tfull[b], 1);
      mbar_init(&ctl->tempty[b], EPI_WARPS);
    }
    mbar_init(&ctl->bfull, 1);
    mbar_init(&ctl->drain, 1);
    ctl->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem_base)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = ctl->tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0 && nt > 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
      mbar_expect_tx(&ctl->bfull, B_BYTES);
      tma_load_2d(Bs, &tmB, 0, rb * BN, &ctl->bfull);
      tma_load_2d(Bs + B_HALF, &tmB, KH, rb * BN, &ctl->bfull);
      int issued = 0;
      for (int it = 0; it < nt; it++) {
        const int s = it % STAGES;
        if (it >= STAGES && !mbar_wait(&ctl->empty[s], ((it / STAGES) & 1) ^ 1, abort, flags)) break;
        unsigned char *a = As + s * A_STAGE;
        mbar_expect_tx(&ctl->full[s], A_STAGE);
        tma_load_2d(a, &tmA, 0, (t0 + it) * BM, &ctl->full[s]);
        tma_load_2d(a + A_HALF, &tmA, KH, (t0 + it) * BM, &ctl->full[s]);
        issued = it + 1;
      }
      // drain: every copy this warp issued has landed before the CTA may exit
      mbar_drain(&ctl->bfull, 0);
      for (int it = max(0, issued - STAGES); it < issued; it++) mbar_drain(&ctl->full[it % STAGES], (it / STAGES) & 1);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0 && nt > 0) {
      bool ok = mbar_wait(&ctl->bfull, 0, abort, flags);
      const uint32_t b_base = smem_u32(Bs);
      for (int it = 0; ok && it < nt; it++) {
        const int s = it % STAGES, buf = it & 1;
        if (!mbar_wait(&ctl->full[s], (it / STAGES) & 1, abort, flags)) break;
        if (it >= 2 && !mbar_wait(&ctl->tempty[buf], ((it >> 1) - 1) & 1, abort, flags)) break;
        fence_after();
        const uint32_t a_base = smem_u32(As + s * A_STAGE);
#pragma unroll
        for (int kk = 0; kk < 8; kk++) {
          const uint32_t off = (uint32_t)((kk >> 2) * A_HALF + (kk & 3) * 32);
          const uint32_t boff = (uint32_t)((kk >> 2) * B_HALF + (kk & 3) * 32);
          mma_bf16(tmem + (uint32_t)(buf * BN), sdesc(a_base + off), sdesc(b_base + boff), idesc_bf16(BM, BN),
                   kk > 0 ? 1u : 0u);
        }
        mma_commit(&ctl->empty[s]);
        mma_commit(&ctl->tfull[buf]);
      }
      // drain: all MMAs issued by this thread are complete
      mma_commit(&ctl->drain);
      mbar_drain(&ctl->drain, 0);
    }
  } else {
    // ---------------- epilogue ----------------
    const int e = warp - 2;
    const int quarter = warp & 3;       // TMEM lane quarter this warp may access
    const int half = e >> 2;            // column half: query rows [half*128, +128)
    for (int it = 0; it < nt; it++) {
      const int buf = it & 1;
      // one lane waits, the whole warp follows its verdict (the TMEM loads below are warp-aligned)
      int ok = 0;
      if (lane == 0) ok = mbar_wait(&ctl->tfull[buf], (it >> 1) & 1, abort, flags) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      __syncwarp();
      fence_after();
      const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * BN + half * 128);
      const int tile = t0 + it;
      const int64_t j = (int64_t)tile * BM + quarter * 32 + lane;  // this thread's centroid
      const bool jv = j < C;
#pragma unroll 1
      for (int pr = 0; pr < 2; pr++) {
        uint32_t v[2][32];
        TC_LD32(ta + pr * 64, v[0]);
        TC_LD32(ta + pr * 64 + 32, v[1]);
        tmem_ld_wait();
        if (pr == 1) {
          // every column of this buffer has been read: hand it back to the MMA warp
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&ctl->tempty[buf]);
        }
#pragma unroll
        for (int cc = 0; cc < 2; cc++) {
          const int ch = pr * 2 + cc;
          if (MODE == 1) {
            // maximum score of the warp's 32 centroids, per query row (-inf: no valid centroid)
            float *dst = reinterpret_cast<float *>(gmax) + ((int64_t)rb * G + tile * 4 + quarter) * BN + half * 128;
            float mine = -INFINITY;
#pragma unroll
            for (int c = 0; c < 32; c++) {
              const float m = redux_fmax(jv ? __uint_as_float(v[cc][c]) : -INFINITY);
              mine = (c == lane) ? m : mine;
            }
            dst[ch * 32 + lane] = mine;
          } else if (MODE == 3) {
            // diagnostic: raw scores [R x C]
#pragma unroll
            for (int c = 0; c < 32; c++) {
              const int row = rb * BN + half * 128 + ch * 32 + c;
              if (jv && row < R) reinterpret_cast<float *>(cand)[(int64_t)row * C + j] = __uint_as_float(v[cc][c]);
            }
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

constexpr int SEL_BINS = 512;   // bins per histogram level
constexpr int SEL_PARTS = 16;   // slices of the groups, one block each
constexpr int GCAP = 256;       // groups a row may keep (8192 centroids)

// Histogram of the group maxima of 32 rows (lane = row) over one slice of the
// groups. Level 1 bins [-cmax, cmax]; level 2 bins the row's level-1 bin
// [lo_r, lo_r + w1) again. Counts are added to hist[row][SEL_BINS].
__global__ void __launch_bounds__(32)
k_gsel_hist(const float *__restrict__ gmax, int G, int R, float cmax, int level, const float *__restrict__ lo,
            uint32_t *__restrict__ hist) {
  __shared__ uint16_t h[32][SEL_BINS + 2];
  const int lane = threadIdx.x;
  const int rb = blockIdx.x >> 3, slab = blockIdx.x & 7;
  const int n = slab * 32 + lane;
  const int row = rb * BN + n;
  for (int b = 0; b < SEL_BINS; b++) h[lane][b] = 0;
  const float w1 = 2.f * cmax / SEL_BINS;
  const float base = (level == 1) ? -cmax : (row < R ? lo[row] : 0.f);
  const float scale = (level == 1) ? 1.f / w1 : SEL_BINS / w1;
  const bool skip = row >= R || (level == 2 && lo[row] == -INFINITY);
  const int per = (G + SEL_PARTS - 1) / SEL_PARTS;
  const int g0 = blockIdx.y * per, g1 = min(G, g0 + per);
  const float *src = gmax + (int64_t)rb * G * BN + n;
  if (!skip) {
    for (int g = g0; g < g1; g += 8) {
      float x[8];
#pragma unroll
      for (int u = 0; u < 8; u++) x[u] = (g + u < g1) ? src[(int64_t)(g + u) * BN] : -INFINITY;
#pragma unroll
      for (int u = 0; u < 8; u++) {
        if (x[u] == -INFINITY) continue;
        const float f = (x[u] - base) * scale;
        if (level == 2 && (f < 0.f || f >= (float)SEL_BINS)) continue;  // outside the row's level-1 bin
        const int b = max(0, min(SEL_BINS - 1, (int)floorf(f)));
        h[lane][b]++;
      }
    }
  }
  __syncwarp();
  if (skip) return;
  uint32_t *hq = hist + (int64_t)row * SEL_BINS;
  for (int b = 0; b < SEL_BINS; b++)
    if (h[lane][b]) atomicAdd(&hq[b], (uint32_t)h[lane][b]);
}

// Per row: the bin holding the kappa_c-th largest group maximum. Level 1 writes
// the bin's lower edge to lo[row] and the count strictly above it to above[row]
// (lo = -inf when fewer than kappa_c groups exist); level 2 narrows to a sub-bin
// and writes lim[row] = its lower edge - margin_r, a value no larger than the
// kappa_c-th largest group maximum minus the margin.
__global__ void k_gsel_tau(const uint32_t *__restrict__ hist, int R, int kc, float cmax, int level,
                           float *__restrict__ lo, uint32_t *__restrict__ above, const float *__restrict__ margins,
                           float *__restrict__ lim) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= R) return;
  const uint32_t *hq = hist + (int64_t)row * SEL_BINS;
  const float w1 = 2.f * cmax / SEL_BINS;
  if (level == 1) {
    uint32_t cum = 0;
    int b = SEL_BINS - 1;
    for (; b >= 0; b--) {
      if (cum + hq[b] >= (uint32_t)kc) break;
      cum += hq[b];
    }
    lo[row] = (b >= 0) ? -cmax + b * w1 : -INFINITY;
    above[row] = cum;
    if (b < 0) lim[row] = -INFINITY;
  } else {
    if (lo[row] == -INFINITY) return;
    uint32_t cum = above[row];
    int b = SEL_BINS - 1;
    for (; b >= 0; b--) {
      if (cum + hq[b] >= (uint32_t)kc) break;
      cum += hq[b];
    }
    const float w2 = w1 / SEL_BINS;
    // the bin edges are computed in FP32: step down by one more sub-bin for safety
    lim[row] = (b >= 0) ? lo[row] + b * w2 - w2 - margins[row] : -INFINITY;
  }
}

// Every group whose maximum is >= lim[row] goes to the row's list.
__global__ void __launch_bounds__(32)
k_gsel_collect(const float *__restrict__ gmax, int G, int R, const float *__restrict__ lim,
               int32_t *__restrict__ glist, int32_t *__restrict__ gcount) {
  const int lane = threadIdx.x;
  const int rb = blockIdx.x >> 3, slab = blockIdx.x & 7;
  const int n = slab * 32 + lane;
  const int row = rb * BN + n;
  if (row >= R) return;
  const float l = lim[row];
  const int per = (G + SEL_PARTS - 1) / SEL_PARTS;
  const int g0 = blockIdx.y * per, g1 = min(G, g0 + per);
  const float *src = gmax + (int64_t)rb * G * BN + n;
  int32_t *out = glist + (int64_t)row * GCAP;
  for (int g = g0; g < g1; g += 8) {
    float x[8];
#pragma unroll
    for (int u = 0; u < 8; u++) x[u] = (g + u < g1) ? src[(int64_t)(g + u) * BN] : -INFINITY;
#pragma unroll
    for (int u = 0; u < 8; u++) {
      if (x[u] != -INFINITY && x[u] >= l) {
        const int pos = atomicAdd(&gcount[row], 1);
        if (pos < GCAP) out[pos] = g + u;
      }
    }
  }
}

// exact FP32 score: fmaf chain over k = 0..127 (the FP32 path's arithmetic)
template <bool BF16C>
__device__ __forceinline__ float dot_exact(const float *__restrict__ q, const float *__restrict__ cf,
                                           const __nv_bfloat16 *__restrict__ cb, int64_t j) {
  float acc = 0.f;
  if (BF16C) {
    const uint4 *row = reinterpret_cast<const uint4 *>(cb + j * DIM);
#pragma unroll 4
    for (int k8 = 0; k8 < DIM / 8; k8++) {
      const uint4 u = row[k8];
      const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int h = 0; h < 4; h++) {
        acc = fmaf(q[k8 * 8 + 2 * h], __uint_as_float(w[h] << 16), acc);
        acc = fmaf(q[k8 * 8 + 2 * h + 1], __uint_as_float(w[h] & 0xffff0000u), acc);
      }
    }
  } else {
    const float4 *row = reinterpret_cast<const float4 *>(cf + j * DIM);
#pragma unroll 4
    for (int k4 = 0; k4 < DIM / 4; k4++) {
      const float4 c = row[k4];
      acc = fmaf(q[k4 * 4 + 0], c.x, acc);
      acc = fmaf(q[k4 * 4 + 1], c.y, acc);
      acc = fmaf(q[k4 * 4 + 2], c.z, acc);
      acc = fmaf(q[k4 * 4 + 3], c.w, acc);
    }
  }
  return acc;
}

// One block per query row: the centroids of the kept groups scored exactly in
// FP32. Only scores >= lim[row] are kept: kappa_c groups have a BF16 maximum
// >= lim + 2 margin, so kappa_c distinct centroids score >= lim + margin
// exactly and the kappa_c-th exact score (ties included) is above lim. The
// kept keys are sorted by (score desc, id asc); the first kappa_c are the
// answer. A row whose groups overflowed the list, or whose kept scores
// overflowed the buffer, is marked for the full FP32 scan.
constexpr int FCAP = 4096;  // kept exact scores per row

template <bool BF16C>
__global__ void __launch_bounds__(256)
k_group_rescore(const float *__restrict__ rows, int R, const float *__restrict__ cent_f32,
                const __nv_bfloat16 *__restrict__ cent_bf16, int64_t C, int kc, const int32_t *__restrict__ glist,
                const int32_t *__restrict__ gcount, const float *__restrict__ lim, int32_t *__restrict__ top_ids,
                float *__restrict__ top_s, int32_t *__restrict__ lossy_rows, uint32_t *__restrict__ flags) {
  extern __shared__ __align__(16) uint64_t rsm[];  // [FCAP] keys
  __shared__ float q[DIM];
  __shared__ int s_cnt;
  const int r = blockIdx.x;
  if (r >= R) return;
  const int ngr = gcount[r];
  const int n = min(ngr, GCAP) * 32;
  const float l = lim[r];
  for (int k = threadIdx.x; k < DIM; k += blockDim.x) q[k] = rows[(int64_t)r * DIM + k];
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  const int32_t *gl = glist + (int64_t)r * GCAP;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int64_t j = (int64_t)gl[i >> 5] * 32 + (i & 31);
    if (j >= C) continue;
    const float sc = dot_exact<BF16C>(q, cent_f32, cent_bf16, j);
    if (!(sc < l)) {
      const int pos = atomicAdd(&s_cnt, 1);
      if (pos < FCAP) rsm[pos] = comp_key(sc, (int32_t)j);
    }
  }
  __syncthreads();
  const int cnt = s_cnt;
  const int m = min(cnt, FCAP);
  const int np = next_pow2(max(m, 2));
  for (int i = m + threadIdx.x; i < np; i += blockDim.x) rsm[i] = 0ull;
  __syncthreads();
  block_sort_desc(rsm, np);
  for (int i = threadIdx.x; i < kc; i += blockDim.x) {
    const uint64_t v = i < m ? rsm[i] : 0ull;
    top_ids[(int64_t)r * kc + i] = v ? comp_id(v) : -1;
    top_s[(int64_t)r * kc + i] = v ? comp_score(v) : -INFINITY;
  }
  if (threadIdx.x == 0) {
    const bool lossy = ngr > GCAP || cnt > FCAP;
    lossy_rows[r] = lossy ? 1 : 0;
    if (lossy) atomicOr(flags, TACHIOM_FLAG_TOPC_RESCUED);
  }
}

// ---- host side ---------------------------------------------------------------------------
std::mutex g_encode_mu;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

tachiom_status get_encoder(PFN_cuTensorMapEncodeTiled_v12000 *out) {
  std::lock_guard<std::mutex> g(g_encode_mu);
  if (!g_encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return fail(TACHIOM_ERR_CUDA, "cuTensorMapEncodeTiled not available");
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  *out = g_encode;
  return TACHIOM_OK;
}

// bf16 [rows x 128], box of 64 K-elements by box_rows rows, 128-byte swizzle
tachiom_status encode_map(CUtensorMap *map, const void *base, int64_t rows, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc;
  tachiom_status st = get_encoder(&enc);
  if (st) return st;
  if (((uintptr_t)base & 15) != 0) return fail(TACHIOM_ERR_INVALID, "tensor map base not 16-byte aligned");
  cuuint64_t dims[2] = {(cuuint64_t)DIM, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)DIM * 2};
  cuuint32_t box[2] = {(cuuint32_t)KH, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(TACHIOM_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return TACHIOM_OK;
}

}  // namespace tc

tachiom_status encode_bf16_map(CUtensorMap *map, const void *base, int64_t rows, int box_rows) {
  return tc::encode_map(map, base, rows, box_rows);
}

int topc_tc_supported() {
  static int cached = -1;
  if (cached >= 0) return cached;
  int dev = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  cudaGetLastError();
  cached = (major == 10 && minor == 3) ? 1 : 0;
  return cached;
}



size_t topc_tc_gmax_elems(int64_t C, int rows) {
  const int64_t ntiles = (C + tc::BM - 1) / tc::BM;
  const int64_t rbs = (rows + tc::BN - 1) / tc::BN;
  return (size_t)(rbs * ntiles * 4 * tc::BN);
}

size_t topc_tc_glist_elems(int rows) { return (size_t)rows * (tc::GCAP + tc::SEL_BINS + 3); }

tachiom_status launch_topc_tc(const Index &ix, const __nv_bfloat16 *rows_bf16, const float *rows, int nrows, int kc,
                              const float *margins, uint32_t *gmax, int32_t *glist, int32_t *gcount,
                              int32_t *lossy_rows, int32_t *top_ids, float *top_s, uint32_t *flags, cudaStream_t s) {
  using namespace tc;
  if (nrows <= 0) return TACHIOM_OK;
  TPROF("topc_tc", s);
  CUtensorMap mA, mB;
  tachiom_status st;
  if ((st = encode_map(&mA, ix.cent_bf16, ix.C, BM))) return st;
  if ((st = encode_map(&mB, rows_bf16, nrows, BN))) return st;
  const int ntiles = (int)((ix.C + BM - 1) / BM);
  const int rbs = (nrows + BN - 1) / BN;
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix.device);
  int splits = std::max(1, sms / rbs);
  splits = std::min(splits, ntiles);
  const int per = (ntiles + splits - 1) / splits;
  splits = (ntiles + per - 1) / per;
  const int G = ntiles * 4;
  TCUDA(cudaFuncSetAttribute(k_topc_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
  k_topc_tc<1><<<dim3(splits, rbs), THREADS, SMEM_BYTES, s>>>(mA, mB, ix.C, nrows, ntiles, per, G, gmax, nullptr,
                                                               flags);
  TLAUNCH();
  {
    // selection workspace inside glist's tail: hist [rows x SEL_BINS] u32, lo, above, lim [rows]
    uint32_t *hist = reinterpret_cast<uint32_t *>(glist + (int64_t)nrows * GCAP);
    float *lo = reinterpret_cast<float *>(hist + (int64_t)nrows * SEL_BINS);
    uint32_t *above = reinterpret_cast<uint32_t *>(lo + nrows);
    float *lim = reinterpret_cast<float *>(above + nrows);
    const float cm = 1.0001f * ix.cnorm_max + 1e-6f;
    const dim3 sg(rbs * 8, SEL_PARTS);
    for (int level = 1; level <= 2; level++) {
      TCUDA(cudaMemsetAsync(hist, 0, (size_t)nrows * SEL_BINS * 4, s));
      k_gsel_hist<<<sg, 32, 0, s>>>(reinterpret_cast<const float *>(gmax), G, nrows, cm, level, lo, hist);
      TLAUNCH();
      k_gsel_tau<<<(nrows + 127) / 128, 128, 0, s>>>(hist, nrows, kc, cm, level, lo, above, margins, lim);
      TLAUNCH();
    }
    TCUDA(cudaMemsetAsync(gcount, 0, (size_t)nrows * 4, s));
    k_gsel_collect<<<sg, 32, 0, s>>>(reinterpret_cast<const float *>(gmax), G, nrows, lim, glist, gcount);
    TLAUNCH();
  }
  const float *lim = reinterpret_cast<const float *>(glist + (int64_t)nrows * GCAP) +
                     (int64_t)nrows * SEL_BINS + 2 * (int64_t)nrows;
  const size_t rsm = (size_t)FCAP * 8;
  if (ix.cdtype == TACHIOM_DTYPE_BF16) {
    TCUDA(cudaFuncSetAttribute(k_group_rescore<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
    k_group_rescore<true><<<nrows, 256, rsm, s>>>(rows, nrows, ix.cent_f32, ix.cent_bf16, ix.C, kc, glist, gcount,
                                                  lim, top_ids, top_s, lossy_rows, flags);
  } else {
    TCUDA(cudaFuncSetAttribute(k_group_rescore<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
    k_group_rescore<false><<<nrows, 256, rsm, s>>>(rows, nrows, ix.cent_f32, ix.cent_bf16, ix.C, kc, glist, gcount,
                                                   lim, top_ids, top_s, lossy_rows, flags);
  }
  TLAUNCH();
  return TACHIOM_OK;
}

// raw BF16 x BF16 -> FP32 tensor-core scores of the rows against every centroid
tachiom_status launch_topc_tc_raw(const Index &ix, const __nv_bfloat16 *rows, int nrows, float *out,
                                  uint32_t *flags, cudaStream_t s) {
  using namespace tc;
  if (nrows <= 0) return TACHIOM_OK;
  CUtensorMap mA, mB;
  tachiom_status st;
  if ((st = encode_map(&mA, ix.cent_bf16, ix.C, BM))) return st;
  if ((st = encode_map(&mB, rows, nrows, BN))) return st;
  const int ntiles = (int)((ix.C + BM - 1) / BM);
  const int rbs = (nrows + BN - 1) / BN;
  int splits = std::min(ntiles, 148);
  const int per = (ntiles + splits - 1) / splits;
  splits = (ntiles + per - 1) / per;
  TCUDA(cudaFuncSetAttribute(k_topc_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
  k_topc_tc<3><<<dim3(splits, rbs), THREADS, SMEM_BYTES, s>>>(mA, mB, ix.C, nrows, ntiles, per, ntiles * 4,
                                                               nullptr, reinterpret_cast<uint64_t *>(out), flags);
  TLAUNCH();
  return TACHIOM_OK;
}

}  // namespace tachiom

extern "C" int tachiom_tc_available(void) { return tachiom::topc_tc_supported(); }
