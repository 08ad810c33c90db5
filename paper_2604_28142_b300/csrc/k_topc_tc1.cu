// Step (a) on the tensor cores in one pass: BF16 products, FP32 accumulation,
// a per-row running top-kappa_c in the epilogue (Sec. 2.2, Gather step 1 in
// exhaustive form).
//
// Orientation: a tcgen05.mma tile is M = 128 query rows (TMEM lanes) by
// N = 128 centroids (TMEM columns) by K = 128, so an epilogue thread owns one
// query row. The CTA keeps its 128 rows resident (32 KB, one TMA load) and
// streams the centroids of its slice in 128-row tiles through a 3-stage
// TMA/mbarrier ring; two 128-column FP32 accumulators in TMEM let the MMA of
// tile t+1 overlap the epilogue of tile t. Warp 0 issues TMA, warp 1 owns TMEM
// and issues the MMAs, warps 2..5 (one per TMEM lane quarter) are the epilogue.
//
// Per row, the owning thread keeps a threshold thr in a register (the
// kappa_c-th best approximate score it has seen, -inf before kappa_c) and a
// private 96-entry buffer in shared memory. A score s is kept when
// s >= thr - margin; a full buffer is compacted by a quickselect of its
// kappa_c-th entry, which raises thr, and keeps every entry >= thr - margin.
// margin = 2 * delta_row, delta_row a bound on |BF16 score - FP32 score| for the
// row (from its own rounding error, k_quantize_rows), so the
// survivors of all slices contain the row's exact FP32 top-kappa_c and the
// merge (k_topc_merge) rescoring that window in FP32 returns it exactly. A
// row whose kept set cannot fit is marked and recomputed in FP32.
//
// Every mbarrier wait is bounded by %globaltimer; on a timeout every role
// leaves its loop, copies and MMAs in flight are drained, TMEM is freed.
#include "tc_common.cuh"

namespace tachiom {
namespace tc1 {

using namespace tc;

constexpr int BM = 128;        // query rows per CTA (MMA M)
constexpr int BN = 128;        // centroids per tile (MMA N)
constexpr int KH = 64;         // K elements per 128-byte swizzled half
constexpr int STAGES = 3;
constexpr int A_HALF = BM * KH * 2;      // 16 KB
constexpr int A_BYTES = 2 * A_HALF;      // 32 KB (resident queries)
constexpr int B_HALF = BN * KH * 2;      // 16 KB
constexpr int B_STAGE = 2 * B_HALF;      // 32 KB
constexpr int CAP = 96;                  // candidates a row keeps between compactions
constexpr int THREADS = 192;             // 6 warps
constexpr int EPI_WARPS = 4;
constexpr int TMEM_COLS = 256;
constexpr int MAX_KC1 = 64;              // larger kappa_c takes the two-pass kernel

struct Ctl {
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t afull;
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
};
constexpr int TILE_BYTES = A_BYTES + STAGES * B_STAGE;           // 128 KB
constexpr int BUF_BYTES = CAP * BM * 8;                          // 96 KB
constexpr int SMEM_BYTES = TILE_BYTES + BUF_BYTES + (int)sizeof(Ctl) + 1024;

// k-th largest (1 <= k <= n) of the n keys buf[i * BM] by quickselect (Hoare
// partition); reorders them so that the k largest come first
__device__ __noinline__ uint64_t kth_largest(uint64_t *buf, int n, int k) {
  int lo = 0, hi = n - 1;
  const int want = k - 1;  // index in descending order
  while (lo < hi) {
    const uint64_t pivot = buf[((lo + hi) >> 1) * BM];
    int i = lo, j = hi;
    while (i <= j) {
      while (i < hi && buf[i * BM] > pivot) i++;
      while (j > lo && buf[j * BM] < pivot) j--;
      if (i <= j) {
        const uint64_t t = buf[i * BM];
        buf[i * BM] = buf[j * BM];
        buf[j * BM] = t;
        i++;
        j--;
      }
    }
    if (want <= j) hi = j;
    else if (want >= i) lo = i;
    else break;
  }
  return buf[want * BM];
}

// Raise thr to the kappa_c-th best and keep every entry >= thr - margin.
// Returns the new count; sets *lossy when that set leaves no room.
__device__ __noinline__ int compact(uint64_t *buf, int n, int kc, float margin, float *thr, bool *lossy) {
  if (n < kc) return n;
  const float t = comp_score(kth_largest(buf, n, kc));
  *thr = t;
  const float lim = t - margin;
  int m = 0;
  for (int i = 0; i < n; i++) {
    const uint64_t v = buf[i * BM];
    if (comp_score(v) >= lim) buf[(m++) * BM] = v;
  }
  if (m > CAP - 8) {
    // too many entries within the window: keep the best CAP - 8, the row is recomputed exactly
    kth_largest(buf, m, CAP - 8);
    m = CAP - 8;
    *lossy = true;
  }
  return m;
}

__global__ void __launch_bounds__(THREADS, 1)
k_topc_tc1(const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmC, int64_t C, int R,
           int ntiles, int tiles_per_split, int kc, const float *__restrict__ margins, uint64_t *__restrict__ split_out,
           int32_t *__restrict__ split_cnt, uint32_t *__restrict__ flags) {
  extern __shared__ __align__(1024) unsigned char tsm_raw[];
  unsigned char *tsm = (unsigned char *)(((uintptr_t)tsm_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *As = tsm;                            // queries: [2 halves][128 rows][128 B]
  unsigned char *Bs = tsm + A_BYTES;                  // centroid tiles: [STAGES][2 halves][128 rows][128 B]
  uint64_t *cbuf = reinterpret_cast<uint64_t *>(tsm + TILE_BYTES);  // [CAP][128 rows]
  Ctl *ctl = reinterpret_cast<Ctl *>(tsm + TILE_BYTES + BUF_BYTES);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rb = blockIdx.y, split = blockIdx.x, nsplit = gridDim.x;
  const int t0 = split * tiles_per_split;
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
    mbar_init(&ctl->afull, 1);
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
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmQ) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmC) : "memory");
      mbar_expect_tx(&ctl->afull, A_BYTES);
      tma_load_2d(As, &tmQ, 0, rb * BM, &ctl->afull);
      tma_load_2d(As + A_HALF, &tmQ, KH, rb * BM, &ctl->afull);
      int issued = 0;
      for (int it = 0; it < nt; it++) {
        const int s = it % STAGES;
        if (it >= STAGES && !mbar_wait(&ctl->empty[s], ((it / STAGES) & 1) ^ 1, abort, flags)) break;
        unsigned char *b = Bs + s * B_STAGE;
        mbar_expect_tx(&ctl->full[s], B_STAGE);
        tma_load_2d(b, &tmC, 0, (t0 + it) * BN, &ctl->full[s]);
        tma_load_2d(b + B_HALF, &tmC, KH, (t0 + it) * BN, &ctl->full[s]);
        issued = it + 1;
      }
      mbar_drain(&ctl->afull, 0);
      for (int it = max(0, issued - STAGES); it < issued; it++) mbar_drain(&ctl->full[it % STAGES], (it / STAGES) & 1);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0 && nt > 0) {
      bool ok = mbar_wait(&ctl->afull, 0, abort, flags);
      const uint32_t a_base = smem_u32(As);
      for (int it = 0; ok && it < nt; it++) {
        const int s = it % STAGES, buf = it & 1;
        if (!mbar_wait(&ctl->full[s], (it / STAGES) & 1, abort, flags)) break;
        if (it >= 2 && !mbar_wait(&ctl->tempty[buf], ((it >> 1) - 1) & 1, abort, flags)) break;
        fence_after();
        const uint32_t b_base = smem_u32(Bs + s * B_STAGE);
#pragma unroll
        for (int kk = 0; kk < 8; kk++) {
          const uint32_t aoff = (uint32_t)((kk >> 2) * A_HALF + (kk & 3) * 32);
          const uint32_t boff = (uint32_t)((kk >> 2) * B_HALF + (kk & 3) * 32);
          mma_bf16(tmem + (uint32_t)(buf * BN), sdesc(a_base + aoff), sdesc(b_base + boff), idesc_bf16(BM, BN),
                   kk > 0 ? 1u : 0u);
        }
        mma_commit(&ctl->empty[s]);
        mma_commit(&ctl->tfull[buf]);
      }
      mma_commit(&ctl->drain);
      mbar_drain(&ctl->drain, 0);
    }
  } else {
    // ---------------- epilogue: one thread per query row ----------------
    const int quarter = warp & 3;
    const int rloc = quarter * 32 + lane;             // TMEM lane = row within the CTA
    const int row = rb * BM + rloc;
    const bool rv = row < R;
    const float margin = rv ? margins[row] : 0.f;
    uint64_t *mybuf = cbuf + rloc;                    // entry i at mybuf[i * BM]
    int cnt = 0;
    float thr = -INFINITY;
    bool lossy = false;
    for (int it = 0; it < nt; it++) {
      const int buf = it & 1;
      int ok = 0;
      if (lane == 0) ok = mbar_wait(&ctl->tfull[buf], (it >> 1) & 1, abort, flags) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      __syncwarp();
      fence_after();
      const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * BN);
      const int64_t jbase = (int64_t)(t0 + it) * BN;
#pragma unroll 1
      for (int pr = 0; pr < 2; pr++) {
        uint32_t v[2][32];
        TC_LD32(ta + pr * 64, v[0]);
        TC_LD32(ta + pr * 64 + 32, v[1]);
        tmem_ld_wait();
        if (pr == 1) {
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&ctl->tempty[buf]);
        }
        if (!rv) continue;
#pragma unroll
        for (int cc = 0; cc < 2; cc++) {
#pragma unroll
          for (int c = 0; c < 32; c++) {
            const float sc = __uint_as_float(v[cc][c]);
            if (sc >= thr - margin) {
              const int64_t j = jbase + pr * 64 + cc * 32 + c;
              if (j < C) {
                mybuf[(cnt++) * BM] = comp_key(sc, (int32_t)j);
                if (cnt == CAP) cnt = compact(mybuf, cnt, kc, margin, &thr, &lossy);
              }
            }
          }
        }
      }
    }
    if (rv) {
      cnt = compact(mybuf, cnt, kc, margin, &thr, &lossy);
      uint64_t *dst = split_out + ((int64_t)row * nsplit + split) * CAP;
      for (int i = 0; i < cnt; i++) dst[i] = mybuf[i * BM];
      split_cnt[(int64_t)row * nsplit + split] = cnt | (lossy ? (1 << 30) : 0);
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

}  // namespace tc1

int topc_tc1_capout() { return tc1::CAP; }
int topc_tc1_max_kc() { return tc1::MAX_KC1; }

// number of centroid slices per 128-row block (one CTA each)
int topc_tc1_splits(const Index &ix, int nrows) {
  const int ntiles = (int)((ix.C + tc1::BN - 1) / tc1::BN);
  const int rbs = (nrows + tc1::BM - 1) / tc1::BM;
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix.device);
  int splits = std::max(1, sms / rbs);
  splits = std::min(splits, ntiles);
  const int per = (ntiles + splits - 1) / splits;
  return (ntiles + per - 1) / per;
}

tachiom_status encode_bf16_map(CUtensorMap *map, const void *base, int64_t rows, int box_rows);

tachiom_status launch_topc_tc1(const Index &ix, const __nv_bfloat16 *rows, int nrows, int kc, const float *margins,
                               uint64_t *split_out, int32_t *split_cnt, uint32_t *flags, cudaStream_t s) {
  using namespace tc1;
  if (nrows <= 0) return TACHIOM_OK;
  if (kc > MAX_KC1) return fail(TACHIOM_ERR_INVALID, "single-pass tensor-core scan takes kappa_c <= %d", MAX_KC1);
  TPROF("topc_tc1", s);
  CUtensorMap mQ, mC;
  tachiom_status st;
  if ((st = encode_bf16_map(&mQ, rows, nrows, BM))) return st;
  if ((st = encode_bf16_map(&mC, ix.cent_bf16, ix.C, BN))) return st;
  const int ntiles = (int)((ix.C + BN - 1) / BN);
  const int rbs = (nrows + BM - 1) / BM;
  const int splits = topc_tc1_splits(ix, nrows);
  const int per = (ntiles + splits - 1) / splits;
  TCUDA(cudaFuncSetAttribute(k_topc_tc1, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
  k_topc_tc1<<<dim3(splits, rbs), THREADS, SMEM_BYTES, s>>>(mQ, mC, ix.C, nrows, ntiles, per, kc, margins, split_out,
                                                            split_cnt, flags);
  TLAUNCH();
  return TACHIOM_OK;
}

}  // namespace tachiom
