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
// Selection without per-row buffers, in two passes over the same products:
//   pass 1  every group of 32 consecutive centroids reports, per query row, its
//           two largest scores (redux.sync per column);
//   tau     tau_r = a lower bound on the row's kappa_c-th largest of those
//           2 x G scores, which are scores of distinct centroids, so tau_r <=
//           the row's kappa_c-th best approximate score (k_topc_tau);
//   pass 2  every score >= tau_r - margin is appended to the row's list.
// With margin = 2 * delta, delta a bound on |BF16 score - FP32 score|, the
// list holds every centroid of the row's exact FP32 top-kappa_c; the merge
// kernel rescores the window in FP32 and keeps the exact top-kappa_c, so the
// result equals the FP32 path's. A row whose list overflows is recomputed in
// FP32 (k_topc_rescue).
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
constexpr int CAPG = 4096;         // candidates per row after pass 2

struct Ctl {
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t bfull;
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
  float thrf[BN];    // pass 2: tau - margin per row of the CTA (+inf for rows past R)
};
constexpr int SMEM_BYTES = TILE_BYTES + (int)sizeof(Ctl) + 1024;

// MODE 1: two largest per group -> gmax[rb][tile*4 + quarter][2][256]
// MODE 2: append scores >= thr to cand[row][CAPG], cnt[row]
// MODE 3: raw scores to (float *)cand [R x C] (diagnostics and tests)
template <int MODE>
__global__ void __launch_bounds__(THREADS, 1)
k_topc_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t C, int R,
          int ntiles, int tiles_per_split, int G, uint32_t *__restrict__ gmax, const uint32_t *__restrict__ tau,
          const float *__restrict__ margins, int32_t *__restrict__ cnt, uint64_t *__restrict__ cand,
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
  if (MODE == 2) {
    for (int n = threadIdx.x; n < BN; n += THREADS) {
      const int row = rb * BN + n;
      const uint32_t t = (row < R) ? tau[row] : 0u;
      // tau == 0: fewer than kappa_c groups, keep everything
      ctl->thrf[n] = (row >= R) ? INFINITY : (t == 0 ? -INFINITY : funkey(t) - margins[row]);
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
            // the two largest scores of the warp's 32 centroids, per query row
            uint32_t *dst = gmax + (((int64_t)rb * G + tile * 4 + quarter) * 2) * BN + half * 128;
            float m1l = -INFINITY, m2l = -INFINITY;
#pragma unroll
            for (int c = 0; c < 32; c++) {
              const float x = jv ? __uint_as_float(v[cc][c]) : -INFINITY;
              const float m1 = redux_fmax(x);
              const unsigned eq = __ballot_sync(0xffffffffu, x == m1);
              const float m2 = (__popc(eq) > 1) ? m1 : redux_fmax(x == m1 ? -INFINITY : x);
              m1l = (c == lane) ? m1 : m1l;
              m2l = (c == lane) ? m2 : m2l;
            }
            dst[ch * 32 + lane] = (m1l == -INFINITY) ? 0u : fkey(m1l);
            dst[BN + ch * 32 + lane] = (m2l == -INFINITY) ? 0u : fkey(m2l);
          } else if (MODE == 3) {
            // diagnostic: raw scores [R x C]
#pragma unroll
            for (int c = 0; c < 32; c++) {
              const int row = rb * BN + half * 128 + ch * 32 + c;
              if (jv && row < R) reinterpret_cast<float *>(cand)[(int64_t)row * C + j] = __uint_as_float(v[cc][c]);
            }
          } else {
            // the warp's max per column decides (uniformly) whether any lane has a candidate
#pragma unroll
            for (int c = 0; c < 32; c++) {
              const int n = half * 128 + ch * 32 + c;
              const float sc = jv ? __uint_as_float(v[cc][c]) : -INFINITY;
              const float lim = ctl->thrf[n];
              if (redux_fmax(sc) >= lim) {
                if (sc >= lim) {
                  const int row = rb * BN + n;
                  const int pos = atomicAdd(&cnt[row], 1);
                  if (pos < CAPG) cand[(int64_t)row * CAPG + pos] = comp_key(sc, (int32_t)j);
                }
              }
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

// tau_r: a lower bound on the row's kappa_c-th largest score, from the two
// largest scores of every group (2 x G actual scores of distinct centroids):
// a saturating 8-bit histogram per row over [-cmax, cmax] (TAU_BINS bins; a
// score above the range counts in the top bin), then the lower edge of the
// highest bin at which the count from the top reaches kappa_c. At least
// kappa_c scores lie at or above that edge, so it cannot exceed the
// kappa_c-th largest score; the work per value does not depend on the order
// in which the values arrive. A block owns 32 rows; its 4 warps histogram one
// quarter of the groups each, lane = row.
constexpr int TAU_WARPS = 4;
constexpr int TAU_BINS = 1024;
__global__ void __launch_bounds__(TAU_WARPS * 32)
k_topc_tau(const uint32_t *__restrict__ gmax, int G, int R, int kc, float cmax, uint32_t *__restrict__ tau) {
  extern __shared__ unsigned char hsm[];  // [TAU_WARPS][TAU_BINS][32] saturating counts
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rb = blockIdx.x >> 3, slab = blockIdx.x & 7;
  const int n = slab * 32 + lane;
  for (int i = threadIdx.x; i < TAU_WARPS * TAU_BINS * 32 / 4; i += blockDim.x)
    reinterpret_cast<uint32_t *>(hsm)[i] = 0u;
  __syncthreads();
  unsigned char *h = hsm + (size_t)warp * TAU_BINS * 32 + lane;
  const float scale = TAU_BINS / (2.f * cmax);
  const int per = (G + TAU_WARPS - 1) / TAU_WARPS;
  const int g0 = warp * per, g1 = min(G, g0 + per);
  const uint32_t *src = gmax + (int64_t)rb * G * 2 * BN + n;
  for (int g = g0; g < g1; g += 4) {
    uint32_t x[8];
#pragma unroll
    for (int u = 0; u < 8; u++) x[u] = (g + (u >> 1) < g1) ? src[((int64_t)(g + (u >> 1)) * 2 + (u & 1)) * BN] : 0u;
#pragma unroll
    for (int u = 0; u < 8; u++) {
      if (!x[u]) continue;
      const float sc = funkey(x[u]);
      const int b = max(0, min(TAU_BINS - 1, (int)floorf((sc + cmax) * scale)));
      unsigned char *p = h + b * 32;
      const unsigned char c = *p;
      if (c != 255) *p = c + 1;
    }
  }
  __syncthreads();
  if (warp == 0) {
    int cum = 0, b = TAU_BINS - 1;
    for (; b >= 0; b--) {
      int c = 0;
#pragma unroll
      for (int w = 0; w < TAU_WARPS; w++) c += hsm[((size_t)w * TAU_BINS + b) * 32 + lane];
      cum += c;
      if (cum >= kc) break;
    }
    const int row = rb * BN + n;
    // bin b's lower edge; fewer than kappa_c scores in all: no bound (keep everything)
    const float edge = (b > 0) ? (b / scale - cmax) : -INFINITY;
    if (row < R) tau[row] = (b >= 0 && edge > -INFINITY) ? fkey(edge) : 0u;
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

int topc_tc_capg() { return tc::CAPG; }

size_t topc_tc_gmax_elems(int64_t C, int rows) {
  const int64_t ntiles = (C + tc::BM - 1) / tc::BM;
  const int64_t rbs = (rows + tc::BN - 1) / tc::BN;
  return (size_t)(rbs * ntiles * 4 * 2 * tc::BN);
}

tachiom_status launch_topc_tc(const Index &ix, const __nv_bfloat16 *rows, int nrows, int kc, const float *margins,
                              uint32_t *gmax, uint32_t *tau, int32_t *cnt, uint64_t *cand, uint32_t *flags,
                              cudaStream_t s) {
  using namespace tc;
  if (nrows <= 0) return TACHIOM_OK;
  TPROF("topc_tc", s);
  CUtensorMap mA, mB;
  tachiom_status st;
  if ((st = encode_map(&mA, ix.cent_bf16, ix.C, BM))) return st;
  if ((st = encode_map(&mB, rows, nrows, BN))) return st;
  const int ntiles = (int)((ix.C + BM - 1) / BM);
  const int rbs = (nrows + BN - 1) / BN;
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix.device);
  int splits = std::max(1, sms / rbs);
  splits = std::min(splits, ntiles);
  const int per = (ntiles + splits - 1) / splits;
  splits = (ntiles + per - 1) / per;
  const int G = ntiles * 4;
  dim3 grid(splits, rbs);
  TCUDA(cudaFuncSetAttribute(k_topc_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
  TCUDA(cudaFuncSetAttribute(k_topc_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
  k_topc_tc<1><<<grid, THREADS, SMEM_BYTES, s>>>(mA, mB, ix.C, nrows, ntiles, per, G, gmax, nullptr, nullptr, nullptr,
                                                  nullptr, flags);
  TLAUNCH();
  const size_t tsm = (size_t)TAU_WARPS * TAU_BINS * 32;
  TCUDA(cudaFuncSetAttribute(k_topc_tau, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm));
  k_topc_tau<<<rbs * 8, TAU_WARPS * 32, tsm, s>>>(gmax, G, nrows, kc, 1.0001f * ix.cnorm_max + 1e-6f, tau);
  TLAUNCH();
  TCUDA(cudaMemsetAsync(cnt, 0, (size_t)nrows * 4, s));
  k_topc_tc<2><<<grid, THREADS, SMEM_BYTES, s>>>(mA, mB, ix.C, nrows, ntiles, per, G, nullptr, tau, margins, cnt,
                                                  cand, flags);
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
                                                               nullptr, nullptr, nullptr, nullptr,
                                                               reinterpret_cast<uint64_t *>(out), flags);
  TLAUNCH();
  return TACHIOM_OK;
}

}  // namespace tachiom

extern "C" int tachiom_tc_available(void) { return tachiom::topc_tc_supported(); }
