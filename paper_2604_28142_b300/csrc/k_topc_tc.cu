// Step (a) on the 5th-generation tensor cores (Sec. 2.2, Gather step 1 in
// exhaustive form): BF16 or FP8-E4M3 products with FP32 accumulation, then an
// exact FP32 repair of the candidates near each row's kappa_c-th score.
//
// GEMM orientation: a tcgen05.mma tile is M = 128 centroids (TMEM lanes) by
// N = 256 query rows (TMEM columns) by K = 128. The CTA keeps its 256 query
// rows resident in shared memory (one TMA load) and streams 128-centroid tiles
// through a TMA/mbarrier ring; two 256-column FP32 accumulators (all 512 TMEM
// columns) let the MMA of tile t+1 run while 16 epilogue warps drain tile t
// with tcgen05.ld. Warp 0 issues TMA, warp 1 owns TMEM and issues the MMAs,
// warps 2..17 are the epilogue (warp w reads TMEM lanes 32*(w%4).., columns
// 64*((w-2)/4)..+64).
//   BF16: a 128-element row is two 128-byte swizzled halves; 8 MMAs of
//         kind::f16 (K = 16) per tile; 4 pipeline stages (192 KB).
//   E4M3: a row is one 128-byte swizzled row; 4 MMAs of kind::f8f6f4 (K = 32)
//         per tile; 8 stages (160 KB). Every centroid and every query row is
//         stored as x * 2^k with max |x| * 2^k in (224, 448] (a power of two, so
//         the scaling is exact) and the epilogue undoes both scales:
//         score = acc * 2^-k_j * 2^-k_i.
//
// The same kernel runs three epilogues:
//   sample  (MODE_SAMPLE) the CTAs walk every S-th centroid tile; per query row,
//           each epilogue lane keeps the TOPM largest maxima over groups of 32
//           centroids it has seen (a stream = one CTA's TMEM lane quarter) ->
//           tops. k_gsel_lim then takes tau'_r = the kappa_c-th largest value of
//           the union of the row's streams: the union holds maxima of distinct
//           groups, so kappa_c distinct centroids score >= tau'_r approximately
//           and >= tau'_r - delta_r exactly, and every centroid of the row's exact
//           top-kappa_c scores >= tau'_r - 2 delta_r =: lim_r approximately;
//   emit    (MODE_EMIT) every tile; each (row, centroid) whose approximate score
//           is >= lim_r is appended to the row's candidate list;
//   raw     (MODE_RAW) diagnostics: every approximate score.
// k_cand_rescore then scores a row's candidates exactly in FP32 (the FP32
// path's fmaf chain) and keeps the first kappa_c by (score desc, id asc). A
// row whose list overflows is recomputed by the full FP32 scan.
// delta_r is the rigorous bound of the row's rounding errors for BF16 (the
// result is then the FP32 path's, bit for bit); for E4M3 it is lambda times
// the same Cauchy-Schwarz bound (lambda = 1: rigorous; lambda < 1: a window
// sized to the typical error, the path's accuracy then measured against the
// FP64 oracle).
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
constexpr int EPI_WARPS = 16;      // 4 per TMEM lane quarter, 64 columns each
constexpr int THREADS = 64 + 32 * EPI_WARPS;  // TMA warp, MMA warp, epilogue
constexpr int TMEM_COLS = 512;
constexpr int TOPM = 4;            // group maxima kept per (query row, stream): any subset of distinct
                                   // groups gives a valid threshold; 4 of the 4 x 148 streams of a row
                                   // nearly always hold its top kappa_c groups
constexpr int ECAP = 16384;        // E4M3: candidates a row may emit (over all CTAs of its row block)
constexpr int SAMPLE_STRIDE = 16;  // the sample pass walks at most every 16th tile
constexpr int GCAP = 256;          // groups of 32 centroids a row may keep (group selection)

enum { MODE_SAMPLE = 1, MODE_EMIT = 2, MODE_RAW = 3 };

// shared-memory geometry of the two operand types
template <bool F8>
struct Geo {
  static constexpr int HALVES = F8 ? 1 : 2;            // 128-byte swizzled column blocks per row
  static constexpr int KBOX = F8 ? 128 : 64;           // K elements per block
  static constexpr int STAGES = F8 ? 8 : 4;
  static constexpr int A_HALF = BM * 128;              // 16 KB
  static constexpr int A_STAGE = HALVES * A_HALF;
  static constexpr int B_HALF = BN * 128;              // 32 KB
  static constexpr int B_BYTES = HALVES * B_HALF;
  static constexpr int KSTEPS = F8 ? 4 : 8;            // MMAs per tile (32 bytes of K each)
  static constexpr int TILE_BYTES = B_BYTES + STAGES * A_STAGE;
};

template <bool F8>
struct Ctl {
  uint64_t full[Geo<F8>::STAGES];
  uint64_t empty[Geo<F8>::STAGES];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t bfull;
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
  float lim[BN];  // MODE_EMIT: per query row, the emission threshold in the accumulator's scale
  int ecnt[BN];   // MODE_EMIT: per query row, the candidates this CTA has emitted
  alignas(16) float stage[EPI_WARPS][2][32];  // MODE_SAMPLE: a warp's 32 column maxima, lane 0 -> lane c
};
template <bool F8>
constexpr int smem_bytes() { return Geo<F8>::TILE_BYTES + (int)sizeof(Ctl<F8>) + 1024; }

// instruction descriptor: kind::f8f6f4 with A = B = E4M3 (format 0), D = F32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_e4m3(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

struct TcArgs {
  int64_t C;
  int R;
  int ntiles;        // centroid tiles of the table
  int tstride;       // the CTA walks tiles (x + it * splits) * tstride
  const float *inv_sc;   // E4M3: [C] 2^-k of every centroid
  const float *inv_sq;   // E4M3: [R] 2^-k of every query row
  const float *lim;      // MODE_EMIT: [R] emission threshold (score scale)
  float *tops;           // MODE_SAMPLE: [R][splits * 4][TOPM]
  uint32_t *gmax;        // MODE_SAMPLE, optional: [rbs][G][256] fp16 group maxima, rounded up
  int G;                 // groups of the table (4 per tile)
  int32_t *elist;        // MODE_EMIT: [R][splits][scap] each CTA's candidates of each row
  int32_t *ecnt;         // MODE_EMIT: [R][splits] their counts (may exceed scap: overflow)
  int scap;
  float *raw;            // MODE_RAW: [R][C]
  uint64_t wait_ns;      // limit of every mbarrier wait (0: TIMEOUT_NS)
  int withhold;          // diagnostics: the producer issues no copy, so the first wait runs out
  uint32_t *flags;
};

// CTA (x, rb) takes the tiles (x + it * splits) * tstride against query rows [rb * 256, +256).
template <int MODE, bool F8>
__global__ void __launch_bounds__(THREADS, 1)
k_topc_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcArgs A) {
  using G = Geo<F8>;
  extern __shared__ __align__(1024) unsigned char tsm_raw[];
  unsigned char *tsm = (unsigned char *)(((uintptr_t)tsm_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *Bs = tsm;                  // [halves][256 rows][128 B]
  unsigned char *As = tsm + G::B_BYTES;     // [STAGES][halves][128 rows][128 B]
  Ctl<F8> *ctl = reinterpret_cast<Ctl<F8> *>(tsm + G::TILE_BYTES);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the row block is the fastest grid index, so the CTAs resident at once share centroid tiles in L2
  const int rb = blockIdx.x;
  const int sx = blockIdx.y, splits = gridDim.y;
  const int nts = (A.ntiles + A.tstride - 1) / A.tstride;  // tiles of the walk
  const int nt = max(0, (nts - sx + splits - 1) / splits);
  auto tile_of = [&](int it) { return (sx + it * splits) * A.tstride; };
  volatile int *abort = &ctl->abort;

  if (threadIdx.x == 0) {
    for (int s = 0; s < G::STAGES; s++) {
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
  if (MODE == MODE_EMIT) {
    // per row, the threshold in the accumulator's scale: lim / inv_sq (E4M3), +inf past the last row
    for (int i = threadIdx.x; i < BN; i += THREADS) {
      const int row = rb * BN + i;
      float l = INFINITY;
      if (row < A.R) l = F8 ? A.lim[row] / A.inv_sq[row] : A.lim[row];
      ctl->lim[i] = l;
      ctl->ecnt[i] = 0;
    }
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
    if (lane == 0 && nt > 0 && !A.withhold) {
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
      mbar_expect_tx(&ctl->bfull, G::B_BYTES);
#pragma unroll
      for (int h = 0; h < G::HALVES; h++) tma_load_2d(Bs + h * G::B_HALF, &tmB, h * G::KBOX, rb * BN, &ctl->bfull);
      int issued = 0;
      for (int it = 0; it < nt; it++) {
        const int s = it % G::STAGES;
        if (it >= G::STAGES && !mbar_wait(&ctl->empty[s], ((it / G::STAGES) & 1) ^ 1, abort, A.flags, A.wait_ns)) break;
        unsigned char *a = As + s * G::A_STAGE;
        mbar_expect_tx(&ctl->full[s], G::A_STAGE);
#pragma unroll
        for (int h = 0; h < G::HALVES; h++)
          tma_load_2d(a + h * G::A_HALF, &tmA, h * G::KBOX, tile_of(it) * BM, &ctl->full[s]);
        issued = it + 1;
      }
      // drain: every copy this warp issued has landed before the CTA may exit
      mbar_drain(&ctl->bfull, 0, A.wait_ns);
      for (int it = max(0, issued - G::STAGES); it < issued; it++)
        mbar_drain(&ctl->full[it % G::STAGES], (it / G::STAGES) & 1, A.wait_ns);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0 && nt > 0) {
      bool ok = mbar_wait(&ctl->bfull, 0, abort, A.flags, A.wait_ns);
      const uint32_t b_base = smem_u32(Bs);
      for (int it = 0; ok && it < nt; it++) {
        const int s = it % G::STAGES, buf = it & 1;
        if (!mbar_wait(&ctl->full[s], (it / G::STAGES) & 1, abort, A.flags, A.wait_ns)) break;
        if (it >= 2 && !mbar_wait(&ctl->tempty[buf], ((it >> 1) - 1) & 1, abort, A.flags, A.wait_ns)) break;
        fence_after();
        const uint32_t a_base = smem_u32(As + s * G::A_STAGE);
#pragma unroll
        for (int kk = 0; kk < G::KSTEPS; kk++) {
          // 32 bytes of K per MMA inside a 128-byte swizzled block
          const uint32_t off = (uint32_t)((kk >> 2) * G::A_HALF + (kk & 3) * 32);
          const uint32_t boff = (uint32_t)((kk >> 2) * G::B_HALF + (kk & 3) * 32);
          if (F8)
            mma_e4m3(tmem + (uint32_t)(buf * BN), sdesc(a_base + off), sdesc(b_base + boff), idesc_e4m3(BM, BN),
                     kk > 0 ? 1u : 0u);
          else
            mma_bf16(tmem + (uint32_t)(buf * BN), sdesc(a_base + off), sdesc(b_base + boff), idesc_bf16(BM, BN),
                     kk > 0 ? 1u : 0u);
        }
        mma_commit(&ctl->empty[s]);
        mma_commit(&ctl->tfull[buf]);
      }
      // drain: all MMAs issued by this thread are complete
      mma_commit(&ctl->drain);
      mbar_drain(&ctl->drain, 0, A.wait_ns);
    }
  } else {
    // ---------------- epilogue ----------------
    const int e = warp - 2;
    const int quarter = warp & 3;       // TMEM lane quarter this warp may access
    const int cblk = e >> 2;            // column block: query rows [cblk * 64, +64)
    float tm[2][TOPM];                  // MODE_SAMPLE: running TOPM largest of this lane's two rows
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
    float isq[2] = {1.f, 1.f};  // MODE_SAMPLE, E4M3: the scale of this lane's two rows
    if (F8 && MODE == MODE_SAMPLE) {
#pragma unroll
      for (int ch = 0; ch < 2; ch++) {
        const int row = rb * BN + cblk * 64 + ch * 32 + lane;
        isq[ch] = row < A.R ? A.inv_sq[row] : 1.f;
      }
    }
    for (int it = 0; it < nt; it++) {
      const int buf = it & 1;
      // one lane waits, the whole warp follows its verdict (the TMEM loads below are warp-aligned)
      int ok = 0;
      if (lane == 0) ok = mbar_wait(&ctl->tfull[buf], (it >> 1) & 1, abort, A.flags, A.wait_ns) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      __syncwarp();
      fence_after();
      const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * BN + cblk * 64);
      const int tile = tile_of(it);
      const int64_t j = (int64_t)tile * BM + quarter * 32 + lane;  // this thread's centroid
      const bool jv = j < A.C;
      const bool full_tile = (int64_t)(tile + 1) * BM <= A.C;  // uniform: no centroid past C
      const float isc = F8 ? (jv ? __ldg(A.inv_sc + j) : 0.f) : 1.f;
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
        if (MODE == MODE_SAMPLE) {
          // maximum score of the warp's 32 centroids, per query row (-inf: no valid centroid):
          // one redux per column gives every lane all 32 maxima; lane 0 stages them in shared
          // memory and lane l reads the one of its row (two 16-byte stores per 8 columns'
          // worth of selects otherwise spent on the ALU pipe)
          float m[32];
          if (full_tile) {
#pragma unroll
            for (int c = 0; c < 32; c++) m[c] = redux_fmax(F8 ? __uint_as_float(v[c]) * isc : __uint_as_float(v[c]));
          } else {
#pragma unroll
            for (int c = 0; c < 32; c++)
              m[c] = redux_fmax(jv ? (F8 ? __uint_as_float(v[c]) * isc : __uint_as_float(v[c])) : -INFINITY);
          }
          float *stg = ctl->stage[e][ch];
          if (lane == 0) {
#pragma unroll
            for (int u = 0; u < 8; u++)
              reinterpret_cast<float4 *>(stg)[u] = make_float4(m[4 * u], m[4 * u + 1], m[4 * u + 2], m[4 * u + 3]);
          }
          __syncwarp();
          const float mcol = stg[lane];
          __syncwarp();  // read before lane 0 stages the next tile's maxima
          const float mine = F8 ? mcol * isq[ch] : mcol;
          if (A.gmax) {
            __half *dst = reinterpret_cast<__half *>(A.gmax) + ((int64_t)rb * A.G + tile * 4 + quarter) * BN + cblk * 64;
            dst[ch * 32 + lane] = __float2half_ru(mine);  // rounded up: the filter stays conservative
          }
          // most values fall below every lane's current 8th largest: skip the insertion then
          if (__any_sync(0xffffffffu, !(mine <= tm[ch][TOPM - 1]))) insert(tm[ch], mine);
        } else if (MODE == MODE_EMIT) {
          // the rare (row, centroid) pairs at or above the row's threshold go to its list
          const float *lim = ctl->lim + cblk * 64 + ch * 32;
          uint32_t hit = 0u;
#pragma unroll
          for (int c = 0; c < 32; c++) {
            const float sv = F8 ? __uint_as_float(v[c]) * isc : __uint_as_float(v[c]);
            hit |= (sv >= lim[c]) ? (1u << c) : 0u;
          }
          if (!jv) hit = 0u;
          // the rare hits; the row's count lives in shared memory (no global round trip here)
          while (hit) {
            const int c = __ffs(hit) - 1;
            hit &= hit - 1u;
            const int lr = cblk * 64 + ch * 32 + c;
            const int pos = atomicAdd(&ctl->ecnt[lr], 1);
            if (pos < A.scap) A.elist[((int64_t)(rb * BN + lr) * splits + sx) * A.scap + pos] = (int32_t)j;
          }
        } else if (MODE == MODE_RAW) {
#pragma unroll
          for (int c = 0; c < 32; c++) {
            const int row = rb * BN + cblk * 64 + ch * 32 + c;
            if (jv && row < A.R) {
              float sv = __uint_as_float(v[c]);
              if (F8) sv = sv * isc * A.inv_sq[row];
              A.raw[(int64_t)row * A.C + j] = sv;
            }
          }
        }
      }
    }
    if (MODE == MODE_SAMPLE) {
#pragma unroll
      for (int ch = 0; ch < 2; ch++) {
        const int row = rb * BN + cblk * 64 + ch * 32 + lane;
        if (row < A.R) {
          float4 *d = reinterpret_cast<float4 *>(A.tops + ((int64_t)row * splits * 4 + sx * 4 + quarter) * TOPM);
          const float *t = tm[ch];
#pragma unroll
          for (int k = 0; k < TOPM / 4; k++) d[k] = make_float4(t[4 * k], t[4 * k + 1], t[4 * k + 2], t[4 * k + 3]);
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (MODE == MODE_EMIT) {
    for (int i = threadIdx.x; i < BN; i += THREADS) {
      const int row = rb * BN + i;
      if (row < A.R) A.ecnt[(int64_t)row * splits + sx] = ctl->ecnt[i];
    }
  }
  if (warp == 1) {
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

constexpr int LIM_THREADS = 128;
constexpr int LIM_VPT = 37;     // values per thread: up to 148 CTAs x 4 streams x 8 per row

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
constexpr int GRS_WARPS = 8;

template <bool BF16C>
constexpr int grs_row_bytes() { return BF16C ? DIM * 2 + 16 : DIM * 4 + 16; }
template <bool BF16C>
constexpr size_t grs_smem() { return (size_t)FCAP * 8 + (size_t)GRS_WARPS * 32 * grs_row_bytes<BF16C>(); }

template <bool BF16C>
__global__ void __launch_bounds__(GRS_WARPS * 32)
k_group_rescore(const float *__restrict__ rows, int R, const float *__restrict__ cent_f32,
                const __nv_bfloat16 *__restrict__ cent_bf16, int64_t C, int kc, const int32_t *__restrict__ glist,
                const int32_t *__restrict__ gcount, const float *__restrict__ lim, int32_t *__restrict__ top_ids,
                float *__restrict__ top_s, int32_t *__restrict__ lossy_rows, uint32_t *__restrict__ flags) {
  constexpr int RB = grs_row_bytes<BF16C>();
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
  for (int g = warp; g < ng; g += GRS_WARPS) {
    const int64_t j0 = (int64_t)gl[g] * 32;
#pragma unroll
    for (int u = 0; u < CH; u++) {
      const int c = u * 32 + lane, row = c / CH, pc = c % CH;
      *reinterpret_cast<uint4 *>(st + row * RB + pc * 16) = v[u];
    }
    __syncwarp();
    if (g + GRS_WARPS < ng) load_group(g + GRS_WARPS);  // in flight while this group is scored
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

// One block per query row: the row's candidates (the emit pass's per-CTA lists)
// scored exactly in FP32 with the FP32 path's arithmetic, the fmaf chain over
// k = 0..127; each lane loads its candidate's centroid row into registers
// (16-byte loads). Only scores >= lim[row] are kept: kappa_c centroids score
// >= lim + margin / 2 exactly, so the kappa_c-th exact score (ties included) is
// above lim. The kappa_c-th largest key is found by a radix select, the kappa_c
// keys at or above it are sorted by (score desc, id asc). A row whose lists
// overflowed is marked for the full FP32 scan.
constexpr int RS_THREADS = 256;
constexpr size_t rs_smem() { return (size_t)ECAP * 8; }

template <bool BF16C>
__global__ void __launch_bounds__(RS_THREADS)
k_cand_rescore(const float *__restrict__ rows, int R, const float *__restrict__ cent_f32,
               const __nv_bfloat16 *__restrict__ cent_bf16, int64_t C, int kc, const int32_t *__restrict__ elist,
               const int32_t *__restrict__ ecnt, int splits, int scap, const float *__restrict__ lim,
               int32_t *__restrict__ ncand, int32_t *__restrict__ top_ids, float *__restrict__ top_s,
               int32_t *__restrict__ lossy_rows, uint32_t *__restrict__ flags) {
  extern __shared__ __align__(16) unsigned char rsm_raw[];
  uint64_t *keys = reinterpret_cast<uint64_t *>(rsm_raw);  // [ECAP]
  __shared__ float q[DIM];
  __shared__ uint32_t hist[1 << KSEL_BITS];
  __shared__ uint64_t small[64];
  __shared__ uint64_t kept[MAX_KC];
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t sh[8];
  __shared__ int s_cnt, s_tot, s_lossy;
  const int r = blockIdx.x;
  if (r >= R) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float l = lim[r];
  for (int k = tid; k < DIM; k += RS_THREADS) q[k] = rows[(int64_t)r * DIM + k];
  if (tid == 0) {
    s_cnt = 0;
    s_tot = 0;
    s_lossy = 0;
  }
  __syncthreads();
  for (int x = tid; x < splits; x += RS_THREADS) {
    const int c = ecnt[(int64_t)r * splits + x];
    atomicAdd(&s_tot, c);
    if (c > scap) s_lossy = 1;
  }
  __syncthreads();
  const bool lossy = s_lossy != 0;
  if (!lossy) {
    // warp w takes the lists of CTAs w, w + 8, ...; a lane per candidate
    for (int x = warp; x < splits; x += RS_THREADS / 32) {
      const int c = ecnt[(int64_t)r * splits + x];
      const int32_t *el = elist + ((int64_t)r * splits + x) * scap;
      for (int b = 0; b < c; b += 32) {
        const int i = b + lane;
        const int32_t j = i < c ? el[i] : -1;
        if (j >= 0 && j < C) {
          float acc = 0.f;
          if (BF16C) {
            const uint4 *cr = reinterpret_cast<const uint4 *>(cent_bf16 + (int64_t)j * DIM);
            uint4 v[16];
#pragma unroll
            for (int u = 0; u < 16; u++) v[u] = __ldg(cr + u);
#pragma unroll
            for (int k8 = 0; k8 < 16; k8++) {
              const uint32_t w[4] = {v[k8].x, v[k8].y, v[k8].z, v[k8].w};
#pragma unroll
              for (int h = 0; h < 4; h++) {
                acc = fmaf(q[k8 * 8 + 2 * h], __uint_as_float(w[h] << 16), acc);
                acc = fmaf(q[k8 * 8 + 2 * h + 1], __uint_as_float(w[h] & 0xffff0000u), acc);
              }
            }
          } else {
            const uint4 *cr = reinterpret_cast<const uint4 *>(cent_f32 + (int64_t)j * DIM);
#pragma unroll
            for (int half = 0; half < 2; half++) {
              uint4 v[16];
#pragma unroll
              for (int u = 0; u < 16; u++) v[u] = __ldg(cr + half * 16 + u);
#pragma unroll
              for (int k4 = 0; k4 < 16; k4++) {
                const int k = half * 64 + k4 * 4;
                acc = fmaf(q[k + 0], __uint_as_float(v[k4].x), acc);
                acc = fmaf(q[k + 1], __uint_as_float(v[k4].y), acc);
                acc = fmaf(q[k + 2], __uint_as_float(v[k4].z), acc);
                acc = fmaf(q[k + 3], __uint_as_float(v[k4].w), acc);
              }
            }
          }
          if (!(acc < l)) keys[atomicAdd(&s_cnt, 1)] = comp_key(acc, j);
        } else if (j >= C) {
          atomicOr(flags, TACHIOM_FLAG_BAD_INPUT);
        }
      }
    }
  }
  __syncthreads();
  const int m = lossy ? 0 : s_cnt;
  uint64_t *best = keys;
  int nb = m;
  if (m > kc) {
    // the kappa_c largest keys (distinct: the id is part of the key)
    const uint64_t T = block_kth_largest(keys, m, kc, hist, small, wsum, sh);
    if (tid == 0) sh[6] = 0u;
    __syncthreads();
    for (int i = tid; i < m; i += RS_THREADS)
      if (keys[i] >= T) {
        const uint32_t d = atomicAdd(&sh[6], 1u);
        if (d < (uint32_t)kc) kept[d] = keys[i];
      }
    __syncthreads();
    best = kept;
    nb = kc;
  }
  const int np = next_pow2(max(nb, 2));
  for (int i = nb + tid; i < np; i += RS_THREADS) best[i] = 0ull;
  __syncthreads();
  block_sort_desc(best, np);
  for (int i = tid; i < kc; i += RS_THREADS) {
    const uint64_t vv = i < nb ? best[i] : 0ull;
    top_ids[(int64_t)r * kc + i] = vv ? comp_id(vv) : -1;
    top_s[(int64_t)r * kc + i] = vv ? comp_score(vv) : -INFINITY;
  }
  if (tid == 0) {
    lossy_rows[r] = lossy ? 1 : 0;
    ncand[r] = s_tot;
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
  cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(TACHIOM_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return TACHIOM_OK;
}

// uint8 (E4M3) [rows x 128], box of 128 K-elements (128 bytes) by box_rows rows, 128-byte swizzle
tachiom_status encode_map_u8(CUtensorMap *map, const void *base, int64_t rows, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc;
  tachiom_status st = get_encoder(&enc);
  if (st) return st;
  if (((uintptr_t)base & 15) != 0) return fail(TACHIOM_ERR_INVALID, "tensor map base not 16-byte aligned");
  cuuint64_t dims[2] = {(cuuint64_t)DIM, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)DIM};
  cuuint32_t box[2] = {(cuuint32_t)DIM, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(base), dims, strides, box, estr,
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

static int gcd_int(int a, int b) {
  while (b) {
    const int t = a % b;
    a = b;
    b = t;
  }
  return a;
}

// CTAs along the centroid axis for a walk of nts tiles: splits x row blocks a multiple of the
// SM count (one CTA per SM, every SM busy in every wave), at least enough streams for a row's
// union to hold kappa_c values, at most what k_gsel_lim holds.
static int tc_splits(int nts, int rbs, int kc, int sms) {
  using namespace tc;
  int sp = std::max(1, sms / gcd_int(sms, std::max(1, rbs)));
  sp = std::max(sp, (kc + 4 * TOPM - 1) / (4 * TOPM));
  sp = std::min(sp, std::min(148, LIM_VPT * LIM_THREADS / (4 * TOPM)));  // the per-CTA count layout holds 148
  return std::max(1, std::min(sp, nts));
}

// stride S of the sample pass: at most SAMPLE_STRIDE, the sample keeps >= 8 kappa_c groups, and
// S kappa_c <= 640. The sample's kappa_c-th score sits near the (S kappa_c)-th of the full row, so
// the emission pass passes about S kappa_c centroids plus the window's: a large kappa_c takes a
// denser sample to keep the lists inside ECAP.
static int tc_sample_stride(int ntiles, int kc) {
  const int k = std::max(1, kc);
  return std::max(1, std::min(std::min(tc::SAMPLE_STRIDE, ntiles / (2 * k)), 640 / k));
}

// 32-bit words of: gmax [rbs][groups][256] fp16 (BF16 group selection), then tops
// [rows][streams <= 148 x 4][TOPM] fp32
size_t topc_tc_gmax_elems(const Index &ix, int rows) {
  using namespace tc;
  const int64_t ntiles = (ix.C + BM - 1) / BM;
  const int64_t rbs = (rows + BN - 1) / BN;
  return (size_t)(rbs * ntiles * 4 * BN / 2) + (size_t)rows * (LIM_VPT * LIM_THREADS);
}

// BF16: glist [rows][GCAP], then lim [rows]; E4M3: elist [rows][ECAP] (per row [splits][ECAP /
// splits]), then lim [rows], then the per-CTA counts [rows][splits <= 148]
size_t topc_tc_glist_elems(int rows) {
  return (size_t)rows * std::max<size_t>(tc::GCAP + 1, tc::ECAP + 1 + 148);
}

// the operand maps of one precision: centroids (box 128 rows) and query rows (box 256 rows)
static tachiom_status tc_maps(const Index &ix, const void *rows_q, int nrows, bool f8, CUtensorMap *mA,
                              CUtensorMap *mB) {
  using namespace tc;
  tachiom_status st;
  if (f8) {
    if ((st = encode_map_u8(mA, ix.cent_e4m3, ix.C, BM))) return st;
    return encode_map_u8(mB, rows_q, nrows, BN);
  }
  if ((st = encode_map(mA, ix.cent_bf16, ix.C, BM))) return st;
  return encode_map(mB, rows_q, nrows, BN);
}

template <int MODE, bool F8>
static tachiom_status tc_launch(const CUtensorMap &mA, const CUtensorMap &mB, const tc::TcArgs &a, int splits, int rbs,
                                cudaStream_t s) {
  using namespace tc;
  constexpr int SM = smem_bytes<F8>();
  TCUDA(cudaFuncSetAttribute(k_topc_tc<MODE, F8>, cudaFuncAttributeMaxDynamicSharedMemorySize, SM));
  k_topc_tc<MODE, F8><<<dim3(rbs, splits), THREADS, SM, s>>>(mA, mB, a);
  TLAUNCH();
  return TACHIOM_OK;
}

tachiom_status launch_topc_tc(const Index &ix, const void *rows_q, const float *inv_sq, bool f8, const float *rows,
                              int nrows, int kc, const float *margins, float *gmax_tops, int32_t *glist, int32_t *gcount,
                              int32_t *lossy_rows, int32_t *top_ids, float *top_s, uint32_t *flags, cudaStream_t s) {
  using namespace tc;
  if (nrows <= 0) return TACHIOM_OK;
  TPROF("topc_tc", s);
  if (f8 && !ix.cent_e4m3) return fail(TACHIOM_ERR_INVALID, "the index has no E4M3 centroid copy");
  CUtensorMap mA, mB;
  tachiom_status st;
  if ((st = tc_maps(ix, rows_q, nrows, f8, &mA, &mB))) return st;
  const int ntiles = (int)((ix.C + BM - 1) / BM);
  const int rbs = (nrows + BN - 1) / BN;
  const int sms = tc_sms(ix.device);
  const int G = ntiles * 4;
  TcArgs a{};
  a.C = ix.C;
  a.R = nrows;
  a.ntiles = ntiles;
  a.inv_sc = ix.cent_inv_sc;
  a.inv_sq = inv_sq;
  a.flags = flags;
  a.G = G;
  if (!f8) {
    // BF16: every tile; per (row, group of 32) the maximum -> gmax, per (row, stream) the TOPM largest
    // -> tops; lim = tau' - margin; the groups >= lim; their centroids scored exactly
    uint32_t *gmax = reinterpret_cast<uint32_t *>(gmax_tops);
    float *tops = reinterpret_cast<float *>(reinterpret_cast<__half *>(gmax) + (int64_t)rbs * G * BN);
    float *lim = reinterpret_cast<float *>(glist + (int64_t)nrows * GCAP);
    a.tstride = 1;
    a.tops = tops;
    a.gmax = gmax;
    const int sp = tc_splits(ntiles, rbs, kc, sms);
    if ((st = tc_launch<MODE_SAMPLE, false>(mA, mB, a, sp, rbs, s))) return st;
    if (sp * 4 * TOPM <= 32 * LIM_VPL)
      k_gsel_lim_warp<<<(nrows + 3) / 4, 128, 0, s>>>(tops, nrows, sp * 4 * TOPM, kc, margins, lim);
    else
      k_gsel_lim<<<nrows, LIM_THREADS, 0, s>>>(tops, nrows, sp * 4 * TOPM, kc, margins, lim);
    TLAUNCH();
    TCUDA(cudaMemsetAsync(gcount, 0, (size_t)nrows * 4, s));
    k_gsel_collect<<<dim3(rbs * 8, COL_PARTS), 256, 0, s>>>(reinterpret_cast<const __half *>(gmax), G, nrows, lim,
                                                            glist, gcount);
    TLAUNCH();
    if (ix.cdtype == TACHIOM_DTYPE_BF16) {
      const size_t rsm = grs_smem<true>();
      TCUDA(cudaFuncSetAttribute(k_group_rescore<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
      k_group_rescore<true><<<nrows, GRS_WARPS * 32, rsm, s>>>(rows, nrows, ix.cent_f32, ix.cent_bf16, ix.C, kc,
                                                               glist, gcount, lim, top_ids, top_s, lossy_rows, flags);
    } else {
      const size_t rsm = grs_smem<false>();
      TCUDA(cudaFuncSetAttribute(k_group_rescore<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
      k_group_rescore<false><<<nrows, GRS_WARPS * 32, rsm, s>>>(rows, nrows, ix.cent_f32, ix.cent_bf16, ix.C, kc,
                                                                glist, gcount, lim, top_ids, top_s, lossy_rows, flags);
    }
    TLAUNCH();
    return TACHIOM_OK;
  }
  // E4M3: a sample pass over every S-th tile gives the per-row threshold before the full pass, which
  // emits the candidates above it; their exact scores give the answer
  float *tops = gmax_tops;
  int32_t *elist = glist;
  float *lim = reinterpret_cast<float *>(elist + (int64_t)nrows * ECAP);
  int32_t *scnt = elist + (int64_t)nrows * (ECAP + 1);
  a.tstride = tc_sample_stride(ntiles, kc);
  const int nts = (ntiles + a.tstride - 1) / a.tstride;
  const int sp1 = tc_splits(nts, rbs, kc, sms);
  a.tops = tops;
  if ((st = tc_launch<MODE_SAMPLE, true>(mA, mB, a, sp1, rbs, s))) return st;
  if (sp1 * 4 * TOPM <= 32 * LIM_VPL)
    k_gsel_lim_warp<<<(nrows + 3) / 4, 128, 0, s>>>(tops, nrows, sp1 * 4 * TOPM, kc, margins, lim);
  else
    k_gsel_lim<<<nrows, LIM_THREADS, 0, s>>>(tops, nrows, sp1 * 4 * TOPM, kc, margins, lim);
  TLAUNCH();
  a.tstride = 1;
  a.tops = nullptr;
  a.lim = lim;
  a.elist = elist;
  a.ecnt = scnt;
  const int sp2 = tc_splits(ntiles, rbs, kc, sms);
  a.scap = ECAP / sp2;
  if ((st = tc_launch<MODE_EMIT, true>(mA, mB, a, sp2, rbs, s))) return st;
  const size_t rsm = rs_smem();
  if (ix.cdtype == TACHIOM_DTYPE_BF16) {
    TCUDA(cudaFuncSetAttribute(k_cand_rescore<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
    k_cand_rescore<true><<<nrows, RS_THREADS, rsm, s>>>(rows, nrows, ix.cent_f32, ix.cent_bf16, ix.C, kc, elist, scnt,
                                                        sp2, a.scap, lim, gcount, top_ids, top_s, lossy_rows, flags);
  } else {
    TCUDA(cudaFuncSetAttribute(k_cand_rescore<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
    k_cand_rescore<false><<<nrows, RS_THREADS, rsm, s>>>(rows, nrows, ix.cent_f32, ix.cent_bf16, ix.C, kc, elist,
                                                         scnt, sp2, a.scap, lim, gcount, top_ids, top_s, lossy_rows,
                                                         flags);
  }
  TLAUNCH();
  return TACHIOM_OK;
}

// Diagnostics of the bounded waits: one CTA of the BF16 sample pass whose producer issues no
// copy, every mbarrier wait limited to wait_ns. The MMA warp's first wait runs out: it raises
// TACHIOM_FLAG_TIMEOUT and the abort word, every role leaves its loop, the drains end within
// the same limit, TMEM is freed and the kernel returns. rows_q: any BF16 [>= 256 x 128] buffer
// (nothing is read from it).
tachiom_status launch_topc_tc_wait_test(const Index &ix, const void *rows_q, uint64_t wait_ns, float *tops,
                                        uint32_t *flags, cudaStream_t s) {
  using namespace tc;
  CUtensorMap mA, mB;
  tachiom_status st;
  if ((st = tc_maps(ix, rows_q, BN, false, &mA, &mB))) return st;
  TcArgs a{};
  a.C = ix.C;
  a.R = BN;
  a.ntiles = (int)((ix.C + BM - 1) / BM);
  a.tstride = 1;
  a.tops = tops;
  a.wait_ns = wait_ns;
  a.withhold = 1;
  a.flags = flags;
  return tc_launch<MODE_SAMPLE, false>(mA, mB, a, 1, 1, s);
}

// raw approximate tensor-core scores of the rows against every centroid (BF16 x BF16 or
// E4M3 x E4M3 with the scales undone) -> out [nrows x C]
tachiom_status launch_topc_tc_raw(const Index &ix, const void *rows_q, const float *inv_sq, bool f8, int nrows,
                                  float *out, uint32_t *flags, cudaStream_t s) {
  using namespace tc;
  if (nrows <= 0) return TACHIOM_OK;
  if (f8 && !ix.cent_e4m3) return fail(TACHIOM_ERR_INVALID, "the index has no E4M3 centroid copy");
  CUtensorMap mA, mB;
  tachiom_status st;
  if ((st = tc_maps(ix, rows_q, nrows, f8, &mA, &mB))) return st;
  const int ntiles = (int)((ix.C + BM - 1) / BM);
  const int rbs = (nrows + BN - 1) / BN;
  tc::TcArgs a{};
  a.C = ix.C;
  a.R = nrows;
  a.ntiles = ntiles;
  a.tstride = 1;
  a.inv_sc = ix.cent_inv_sc;
  a.inv_sq = inv_sq;
  a.raw = out;
  a.flags = flags;
  const int splits = std::min(ntiles, 148);
  return f8 ? tc_launch<MODE_RAW, true>(mA, mB, a, splits, rbs, s) : tc_launch<MODE_RAW, false>(mA, mB, a, splits, rbs, s);
}

}  // namespace tachiom

extern "C" int tachiom_tc_available(void) { return tachiom::topc_tc_supported(); }
