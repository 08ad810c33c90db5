// Step (a) on the 5th-generation tensor cores: BF16 products, FP32 accumulation
// (Sec. 2.2, Gather step 1 in exhaustive form), with a rigorous FP32 repair.
//
// GEMM orientation: a tcgen05.mma tile is M = 128 centroids (TMEM lanes) by
// N = 256 query rows (TMEM columns) by K = 128. The CTA keeps its 256 query
// rows resident in shared memory (64 KB, loaded once by TMA) and streams
// 128-centroid tiles (32 KB) through a 4-stage TMA/mbarrier ring. Two
// 256-column FP32 accumulators (all 512 TMEM columns) let the MMA of tile t+1
// run while 16 epilogue warps drain tile t with tcgen05.ld. Warp roles: warp 0
// issues TMA, warp 1 owns TMEM and issues the MMAs, warps 2..17 are the
// epilogue (warp w reads TMEM lanes 32*(w%4).., columns 64*((w-2)/4)..+64).
//
// Selection:
//   pass    every group of 32 consecutive centroids reports, per query row, its
//           maximum approximate score (one redux.sync per column), rounded up
//           to fp16 (so a group is never dropped by the rounding) -> gmax; each
//           epilogue lane also keeps, for each of its query rows, the TOPM
//           largest group maxima it has seen (a stream = one CTA's TMEM lane
//           quarter; tiles go to CTAs in a strided order, so the streams see
//           interleaved parts of the centroid table);
//   select  tau'_r = the kappa_c-th largest value in the union of the row's
//           streams, a lower bound on its kappa_c-th largest group maximum
//           (the union holds maxima of distinct groups); every group whose
//           maximum is >= tau'_r - margin_r is kept. A centroid of the row's
//           exact FP32 top-kappa_c has an approximate score >= (approximate
//           kappa_c-th best) - 2 delta_r >= tau'_r - margin_r (margin_r =
//           2 delta_r), so its group is kept: about kappa_c groups per row
//           survive;
//   rescore the centroids of the kept groups are scored exactly in FP32 (the
//           same fmaf chain as the FP32 path) and the exact top-kappa_c is kept.
// A row whose kept groups do not fit is recomputed by a full FP32 scan.
//
// Every wait on an mbarrier is bounded by %globaltimer; a wait that runs out
// raises TACHIOM_FLAG_TIMEOUT, every role leaves its loop, in-flight copies
// and MMAs are drained (again with a bound) and TMEM is freed before exit.
#include <cuda.h>
#include <cuda_fp16.h>
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
constexpr int EPI_WARPS = 16;      // 4 per TMEM lane quarter, 64 columns each
constexpr int THREADS = 64 + 32 * EPI_WARPS;  // TMA warp, MMA warp, epilogue
constexpr int TMEM_COLS = 512;
constexpr int TOPM = 8;            // group maxima kept per (query row, stream)

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

// CTA (x, rb) takes the tiles x, x + splits, x + 2 splits, ... against query rows [rb * 256, +256).
// MODE 1: maximum per group of 32 centroids, rounded up to fp16 -> gmax[rb][tile * 4 + quarter][256], and per
//         query row the TOPM largest of its stream -> tops[row][x * 4 + quarter][TOPM] (descending)
// MODE 3: raw scores to (float *)cand [R x C] (diagnostics and tests)
template <int MODE>
__global__ void __launch_bounds__(THREADS, 1)
k_topc_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t C, int R,
          int ntiles, int G, uint32_t *__restrict__ gmax, float *__restrict__ tops, uint64_t *__restrict__ cand,
          uint32_t *__restrict__ flags) {
  extern __shared__ __align__(1024) unsigned char tsm_raw[];
  unsigned char *tsm = (unsigned char *)(((uintptr_t)tsm_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *Bs = tsm;                  // [2 halves][256 rows][128 B]
  unsigned char *As = tsm + B_BYTES;        // [STAGES][2 halves][128 rows][128 B]
  Ctl *ctl = reinterpret_cast<Ctl *>(tsm + TILE_BYTES);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rb = blockIdx.y;
  const int splits = gridDim.x;
  const int nt = max(0, (ntiles - (int)blockIdx.x + splits - 1) / splits);
  auto tile_of = [&](int it) { return (int)blockIdx.x + it * splits; };
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
        tma_load_2d(a, &tmA, 0, tile_of(it) * BM, &ctl->full[s]);
        tma_load_2d(a + A_HALF, &tmA, KH, tile_of(it) * BM, &ctl->full[s]);
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
    const int cblk = e >> 2;            // column block: query rows [cblk * 64, +64)
    // running TOPM largest group maxima of this lane's rows cblk * 64 + ch * 32 + lane (descending)
    float tm[2][TOPM];
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
      for (int k = 0; k < TOPM; k++) tm[a][k] = -INFINITY;
    auto insert = [](float (&t)[TOPM], float x) {
      x = (x == x) ? x : -INFINITY;
#pragma unroll
      for (int k = 0; k < TOPM; k++) {
        const float hi = fmaxf(t[k], x);
        x = fminf(t[k], x);
        t[k] = hi;
      }
    };
    for (int it = 0; it < nt; it++) {
      const int buf = it & 1;
      // one lane waits, the whole warp follows its verdict (the TMEM loads below are warp-aligned)
      int ok = 0;
      if (lane == 0) ok = mbar_wait(&ctl->tfull[buf], (it >> 1) & 1, abort, flags) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      __syncwarp();
      fence_after();
      const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * BN + cblk * 64);
      const int tile = tile_of(it);
      const int64_t j = (int64_t)tile * BM + quarter * 32 + lane;  // this thread's centroid
      const bool jv = j < C;
      const bool full_tile = (int64_t)(tile + 1) * BM <= C;  // uniform: no centroid past C
#pragma unroll
      for (int ch = 0; ch < 2; ch++) {
        uint32_t v[32];
        TC_LD32(ta + ch * 32, v);
        tmem_ld_wait();
        if (ch == 1) {
          // every column of this warp's share of the buffer has been read: hand it back
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&ctl->tempty[buf]);
        }
        if (MODE == 1) {
          // maximum score of the warp's 32 centroids, per query row (-inf: no valid centroid):
          // one redux per column gives every lane all 32 maxima, a 5-level select tree
          // leaves lane l the one of its row
          __half *dst = reinterpret_cast<__half *>(gmax) + ((int64_t)rb * G + tile * 4 + quarter) * BN + cblk * 64;
          float m[32];
          if (full_tile) {
#pragma unroll
            for (int c = 0; c < 32; c++) m[c] = redux_fmax(__uint_as_float(v[c]));
          } else {
#pragma unroll
            for (int c = 0; c < 32; c++) m[c] = redux_fmax(jv ? __uint_as_float(v[c]) : -INFINITY);
          }
#pragma unroll
          for (int w = 16; w >= 1; w >>= 1) {
            const bool hi = (lane & w) != 0;
#pragma unroll
            for (int c = 0; c < w; c++) m[c] = hi ? m[c + w] : m[c];
          }
          const float mine = m[0];
          dst[ch * 32 + lane] = __float2half_ru(mine);  // rounded up: the filter stays conservative
          // most values fall below every lane's current 8th largest: skip the insertion then
          if (__any_sync(0xffffffffu, !(mine <= tm[ch][TOPM - 1]))) insert(tm[ch], mine);
        } else if (MODE == 3) {
          // diagnostic: raw scores [R x C]
#pragma unroll
          for (int c = 0; c < 32; c++) {
            const int row = rb * BN + cblk * 64 + ch * 32 + c;
            if (jv && row < R) reinterpret_cast<float *>(cand)[(int64_t)row * C + j] = __uint_as_float(v[c]);
          }
        }
      }
    }
    if (MODE == 1) {
#pragma unroll
      for (int ch = 0; ch < 2; ch++) {
        const int row = rb * BN + cblk * 64 + ch * 32 + lane;
        if (row < R) {
          float4 *d = reinterpret_cast<float4 *>(tops + ((int64_t)row * splits * 4 + blockIdx.x * 4 + quarter) * TOPM);
          const float *t = tm[ch];
#pragma unroll
          for (int k = 0; k < TOPM / 4; k++) d[k] = make_float4(t[4 * k], t[4 * k + 1], t[4 * k + 2], t[4 * k + 3]);
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

constexpr int GCAP = 256;       // groups a row may keep (8192 centroids)
constexpr int LIM_THREADS = 128;
constexpr int LIM_VPT = 37;     // values per thread: up to 148 CTAs x 4 streams x TOPM per row

// Per row: tau' = the kappa_c-th largest value of the union of its streams'
// TOPM lists (bitwise search for the largest key with at least kappa_c keys
// >= it), lim[row] = tau' - margin_r; -inf when the union has fewer than
// kappa_c finite values.
__global__ void __launch_bounds__(LIM_THREADS)
k_gsel_lim(const float *__restrict__ tops, int R, int nvals, int kc, const float *__restrict__ margins,
           float *__restrict__ lim) {
  __shared__ int cnt[3];
  const int row = blockIdx.x;
  if (row >= R) return;
  const float *src = tops + (int64_t)row * nvals;
  uint32_t key[LIM_VPT];
#pragma unroll
  for (int u = 0; u < LIM_VPT; u++) {
    const int i = threadIdx.x + u * LIM_THREADS;
    key[u] = i < nvals ? fkey(src[i]) : 0u;
  }
  if (threadIdx.x < 3) cnt[threadIdx.x] = 0;
  __syncthreads();
  uint32_t T = 0u;
  for (int bit = 31, it = 0; bit >= 0; bit--, it++) {
    // buffer it % 3 is counted now; buffer (it + 1) % 3 was last read two iterations ago
    if (threadIdx.x == 0) cnt[(it + 1) % 3] = 0;
    const uint32_t cand = T | (1u << bit);
    int c = 0;
#pragma unroll
    for (int u = 0; u < LIM_VPT; u++) c += key[u] >= cand ? 1 : 0;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&cnt[it % 3], c);
    __syncthreads();
    if (cnt[it % 3] >= kc) T = cand;
  }
  if (threadIdx.x == 0) {
    const float v = funkey(T);
    lim[row] = (nvals >= kc && T > fkey(-INFINITY) && v == v) ? v - margins[row] : -INFINITY;
  }
}

// Same, one warp per row when the union holds at most 32 x LIM_VPL values (no barriers).
constexpr int LIM_VPL = 24;
__global__ void __launch_bounds__(128)
k_gsel_lim_warp(const float *__restrict__ tops, int R, int nvals, int kc, const float *__restrict__ margins,
                float *__restrict__ lim) {
  const int row = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= R) return;
  const float *src = tops + (int64_t)row * nvals;
  uint32_t key[LIM_VPL];
#pragma unroll
  for (int u = 0; u < LIM_VPL; u++) {
    const int i = lane + u * 32;
    key[u] = i < nvals ? fkey(src[i]) : 0u;
  }
  uint32_t T = 0u;
  for (int bit = 31; bit >= 0; bit--) {
    const uint32_t cand = T | (1u << bit);
    int c = 0;
#pragma unroll
    for (int u = 0; u < LIM_VPL; u++) c += key[u] >= cand ? 1 : 0;
    if (__reduce_add_sync(0xffffffffu, c) >= kc) T = cand;
  }
  if (lane == 0) {
    const float v = funkey(T);
    lim[row] = (nvals >= kc && T > fkey(-INFINITY) && v == v) ? v - margins[row] : -INFINITY;
  }
}

// Every group whose maximum is >= lim[row] goes to the row's list. Block =
// 8 warps on the same 32 rows (lane = row), each warp a strided share of
// one slice of the groups.
constexpr int COL_PARTS = 16;
__global__ void __launch_bounds__(256)
k_gsel_collect(const __half *__restrict__ gmax, int G, int R, const float *__restrict__ lim,
               int32_t *__restrict__ glist, int32_t *__restrict__ gcount) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rb = blockIdx.x >> 3, slab = blockIdx.x & 7;
  const int n = slab * 32 + lane;
  const int row = rb * BN + n;
  const bool live = row < R;
  const float l = live ? lim[row] : INFINITY;
  const int per = (G + COL_PARTS - 1) / COL_PARTS;
  const int g0 = blockIdx.y * per, g1 = min(G, g0 + per);
  const __half *src = gmax + (int64_t)rb * G * BN + n;
  int32_t *out = glist + (int64_t)row * GCAP;
  for (int g = g0 + warp * 8; g < g1; g += 64) {
    float x[8];
#pragma unroll
    for (int u = 0; u < 8; u++) x[u] = (g + u < g1) ? __half2float(src[(int64_t)(g + u) * BN]) : -INFINITY;
#pragma unroll
    for (int u = 0; u < 8; u++) {
      if (live && x[u] != -INFINITY && x[u] >= l) {
        const int pos = atomicAdd(&gcount[row], 1);
        if (pos < GCAP) out[pos] = g + u;
      }
    }
  }
}

// One block per query row: the centroids of the kept groups scored exactly in
// FP32 (a warp stages a group's 32 centroid rows in shared memory with
// coalesced loads; lane l scores centroid l with the FP32 path's arithmetic,
// the fmaf chain over k = 0..127). Only scores >= lim[row] are kept: kappa_c
// groups have a BF16 maximum >= lim + 2 margin, so kappa_c distinct centroids
// score >= lim + margin exactly and the kappa_c-th exact score (ties
// included) is above lim. The kept keys are sorted by (score desc, id asc);
// the first kappa_c are the answer. A row whose groups overflowed the list,
// or whose kept scores overflowed the buffer, is marked for the full FP32 scan.
constexpr int FCAP = 2048;       // kept exact scores per row
constexpr int RS_WARPS = 8;

template <bool BF16C>
constexpr int rs_row_bytes() { return BF16C ? DIM * 2 + 16 : DIM * 4 + 16; }
template <bool BF16C>
constexpr size_t rs_smem() { return (size_t)FCAP * 8 + (size_t)RS_WARPS * 32 * rs_row_bytes<BF16C>(); }

template <bool BF16C>
__global__ void __launch_bounds__(RS_WARPS * 32)
k_group_rescore(const float *__restrict__ rows, int R, const float *__restrict__ cent_f32,
                const __nv_bfloat16 *__restrict__ cent_bf16, int64_t C, int kc, const int32_t *__restrict__ glist,
                const int32_t *__restrict__ gcount, const float *__restrict__ lim, int32_t *__restrict__ top_ids,
                float *__restrict__ top_s, int32_t *__restrict__ lossy_rows, uint32_t *__restrict__ flags) {
  constexpr int RB = rs_row_bytes<BF16C>();
  constexpr int CH = BF16C ? DIM * 2 / 16 : DIM * 4 / 16;  // 16-byte chunks per centroid row
  extern __shared__ __align__(16) unsigned char rsm_raw[];
  uint64_t *keys = reinterpret_cast<uint64_t *>(rsm_raw);  // [FCAP]
  __shared__ float q[DIM];
  __shared__ int s_cnt;
  const int r = blockIdx.x;
  if (r >= R) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char *st = rsm_raw + FCAP * 8 + warp * 32 * RB;
  const int ngr = gcount[r];
  const int ng = min(ngr, GCAP);
  const float l = lim[r];
  for (int k = threadIdx.x; k < DIM; k += blockDim.x) q[k] = rows[(int64_t)r * DIM + k];
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  const int32_t *gl = glist + (int64_t)r * GCAP;
  // the group's rows in registers, loaded one group ahead (a row past C reads row C - 1: unused)
  uint4 v[CH];
  auto load_group = [&](int g) {
    const int64_t j0 = (int64_t)gl[g] * 32;
#pragma unroll
    for (int u = 0; u < CH; u++) {
      const int c = u * 32 + lane, row = c / CH, pc = c % CH;
      const int64_t jr = min(j0 + row, C - 1);
      v[u] = BF16C ? reinterpret_cast<const uint4 *>(cent_bf16 + jr * DIM)[pc]
                   : reinterpret_cast<const uint4 *>(cent_f32 + jr * DIM)[pc];
    }
  };
  if (warp < ng) load_group(warp);
  for (int g = warp; g < ng; g += RS_WARPS) {
    const int64_t j0 = (int64_t)gl[g] * 32;
#pragma unroll
    for (int u = 0; u < CH; u++) {
      const int c = u * 32 + lane, row = c / CH, pc = c % CH;
      *reinterpret_cast<uint4 *>(st + row * RB + pc * 16) = v[u];
    }
    __syncwarp();
    if (g + RS_WARPS < ng) load_group(g + RS_WARPS);  // in flight while this group is scored
    const int64_t j = j0 + lane;
    if (j < C) {
      float acc = 0.f;
      const uint4 *cr = reinterpret_cast<const uint4 *>(st + lane * RB);
      if (BF16C) {
#pragma unroll
        for (int k8 = 0; k8 < DIM / 8; k8++) {
          const uint4 u = cr[k8];
          const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
          for (int h = 0; h < 4; h++) {
            acc = fmaf(q[k8 * 8 + 2 * h], __uint_as_float(w[h] << 16), acc);
            acc = fmaf(q[k8 * 8 + 2 * h + 1], __uint_as_float(w[h] & 0xffff0000u), acc);
          }
        }
      } else {
#pragma unroll
        for (int k4 = 0; k4 < DIM / 4; k4++) {
          const uint4 u = cr[k4];
          acc = fmaf(q[k4 * 4 + 0], __uint_as_float(u.x), acc);
          acc = fmaf(q[k4 * 4 + 1], __uint_as_float(u.y), acc);
          acc = fmaf(q[k4 * 4 + 2], __uint_as_float(u.z), acc);
          acc = fmaf(q[k4 * 4 + 3], __uint_as_float(u.w), acc);
        }
      }
      if (!(acc < l)) {
        const int pos = atomicAdd(&s_cnt, 1);
        if (pos < FCAP) keys[pos] = comp_key(acc, (int32_t)j);
      }
    }
    __syncwarp();
  }
  __syncthreads();
  const int cnt = s_cnt;
  const int m = min(cnt, FCAP);
  const int np = next_pow2(max(m, 2));
  for (int i = m + threadIdx.x; i < np; i += blockDim.x) keys[i] = 0ull;
  __syncthreads();
  block_sort_desc(keys, np);
  for (int i = threadIdx.x; i < kc; i += blockDim.x) {
    const uint64_t v = i < m ? keys[i] : 0ull;
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



static int tc_sms(int device) {
  int sms = 148;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    sms = 148;
  }
  return sms;
}

// CTAs along the centroid axis: enough to fill the SMs, at least enough streams
// for a row's union to hold kappa_c values, at most what k_gsel_lim holds
static int tc_splits(int ntiles, int rbs, int kc, int sms) {
  using namespace tc;
  int sp = std::max(1, sms / rbs);
  sp = std::max(sp, (kc + 4 * TOPM - 1) / (4 * TOPM));
  sp = std::min(sp, LIM_VPT * LIM_THREADS / (4 * TOPM));
  return std::max(1, std::min(sp, ntiles));
}

// 32-bit words of: gmax [rbs][groups][256] fp16, then tops [rows][streams][TOPM] fp32
size_t topc_tc_gmax_elems(const Index &ix, int rows) {
  using namespace tc;
  const int ntiles = (int)((ix.C + BM - 1) / BM);
  const int rbs = (rows + BN - 1) / BN;
  const int splits = tc_splits(ntiles, rbs, MAX_KC, tc_sms(ix.device));
  return (size_t)rbs * ntiles * 4 * BN / 2 + (size_t)rows * splits * 4 * TOPM;
}

// glist [rows][GCAP] followed by lim [rows]
size_t topc_tc_glist_elems(int rows) { return (size_t)rows * (tc::GCAP + 1); }

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
  const int splits = tc_splits(ntiles, rbs, kc, tc_sms(ix.device));
  const int G = ntiles * 4;
  float *tops = reinterpret_cast<float *>(reinterpret_cast<__half *>(gmax) + (int64_t)rbs * G * BN);
  float *lim = reinterpret_cast<float *>(glist + (int64_t)nrows * GCAP);
  TCUDA(cudaFuncSetAttribute(k_topc_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
  k_topc_tc<1><<<dim3(splits, rbs), THREADS, SMEM_BYTES, s>>>(mA, mB, ix.C, nrows, ntiles, G, gmax, tops, nullptr,
                                                               flags);
  TLAUNCH();
  if (splits * 4 * TOPM <= 32 * LIM_VPL)
    k_gsel_lim_warp<<<(nrows + 3) / 4, 128, 0, s>>>(tops, nrows, splits * 4 * TOPM, kc, margins, lim);
  else
    k_gsel_lim<<<nrows, LIM_THREADS, 0, s>>>(tops, nrows, splits * 4 * TOPM, kc, margins, lim);
  TLAUNCH();
  TCUDA(cudaMemsetAsync(gcount, 0, (size_t)nrows * 4, s));
  k_gsel_collect<<<dim3(rbs * 8, COL_PARTS), 256, 0, s>>>(reinterpret_cast<const __half *>(gmax), G, nrows, lim,
                                                          glist, gcount);
  TLAUNCH();
  if (ix.cdtype == TACHIOM_DTYPE_BF16) {
    const size_t rsm = rs_smem<true>();
    TCUDA(cudaFuncSetAttribute(k_group_rescore<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
    k_group_rescore<true><<<nrows, RS_WARPS * 32, rsm, s>>>(rows, nrows, ix.cent_f32, ix.cent_bf16, ix.C, kc,
                                                            glist, gcount, lim, top_ids, top_s, lossy_rows, flags);
  } else {
    const size_t rsm = rs_smem<false>();
    TCUDA(cudaFuncSetAttribute(k_group_rescore<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
    k_group_rescore<false><<<nrows, RS_WARPS * 32, rsm, s>>>(rows, nrows, ix.cent_f32, ix.cent_bf16, ix.C, kc,
                                                             glist, gcount, lim, top_ids, top_s, lossy_rows, flags);
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
  const int splits = std::min(ntiles, 148);
  TCUDA(cudaFuncSetAttribute(k_topc_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
  k_topc_tc<3><<<dim3(splits, rbs), THREADS, SMEM_BYTES, s>>>(mA, mB, ix.C, nrows, ntiles, ntiles * 4, nullptr,
                                                               nullptr, reinterpret_cast<uint64_t *>(out), flags);
  TLAUNCH();
  return TACHIOM_OK;
}

}  // namespace tachiom

extern "C" int tachiom_tc_available(void) { return tachiom::topc_tc_supported(); }
