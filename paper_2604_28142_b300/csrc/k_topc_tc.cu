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
//           maximum score (one redux.sync per column);
//   tau     tau_r = the kappa_c-th largest group maximum of row r. Those kappa_c
//           maxima are kappa_c distinct scores, so tau_r <= the row's
//           kappa_c-th best approximate score;
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

#include "tachiom_internal.cuh"

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
constexpr uint64_t TIMEOUT_NS = 2000000000ull;

struct Ctl {
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t bfull;
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
  uint32_t thr[BN];  // pass 2: fkey(tau - margin) per row of the CTA
};
constexpr int SMEM_BYTES = TILE_BYTES + (int)sizeof(Ctl) + 1024;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false when the CTA is aborting or the time limit passed
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, volatile int *abort, uint32_t *flags) {
  uint64_t t0 = 0;
  for (uint32_t i = 0;; i++) {
    if (mbar_test(b, parity)) return true;
    if ((i & 63) == 0) {
      if (*abort) return false;
      uint64_t t = gtimer();
      if (i == 0) t0 = t;
      else if (t - t0 > TIMEOUT_NS) {
        *abort = 1;
        atomicOr(flags, TACHIOM_FLAG_TIMEOUT);
        return false;
      }
    }
  }
}
// wait with a bound and no abort check (drain at exit)
__device__ __forceinline__ void mbar_drain(uint64_t *b, uint32_t parity) {
  uint64_t t0 = gtimer();
  while (!mbar_test(b, parity))
    if (gtimer() - t0 > TIMEOUT_NS) break;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}

// instruction descriptor: kind::f16, A = B = BF16, D = F32, K-major both, M = 128, N = 256
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(IDESC), "r"(accum));
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

#define TC_LD32(taddr, v)                                                                                    \
  asm volatile(                                                                                              \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"      \
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                             \
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),      \
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), \
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),           \
        "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),           \
        "=r"(v[30]), "=r"(v[31])                                                                             \
      : "r"(taddr))

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t redux_max(uint32_t x) {
  uint32_t r;
  asm volatile("redux.sync.max.u32 %0, %1, 0xffffffff;" : "=r"(r) : "r"(x));
  return r;
}

// MODE 1: group maxima -> gmax[rb][tile*4 + quarter][256]
// MODE 2: append scores >= thr to cand[row][CAPG], cnt[row]
// MODE 3: raw scores to (float *)cand [R x C] (diagnostics and tests)
template <int MODE>
__global__ void __launch_bounds__(THREADS, 1)
k_topc_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t C, int R,
          int ntiles, int tiles_per_split, int G, uint32_t *__restrict__ gmax, const uint32_t *__restrict__ tau,
          float margin, int32_t *__restrict__ cnt, uint64_t *__restrict__ cand, uint32_t *__restrict__ flags) {
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
      int row = rb * BN + n;
      uint32_t t = (row < R) ? tau[row] : 0xFFFFFFFFu;
      // tau == 0: fewer than kappa_c groups, keep everything
      ctl->thr[n] = (row >= R) ? 0xFFFFFFFFu : (t == 0 ? 0u : fkey(funkey(t) - margin));
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
          mma_bf16(tmem + (uint32_t)(buf * BN), sdesc(a_base + off), sdesc(b_base + boff), kk > 0 ? 1u : 0u);
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
      if (!mbar_wait(&ctl->tfull[buf], (it >> 1) & 1, abort, flags)) break;
      fence_after();
      uint32_t v[4][32];
      const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * BN + half * 128);
      TC_LD32(ta + 0, v[0]);
      TC_LD32(ta + 32, v[1]);
      TC_LD32(ta + 64, v[2]);
      TC_LD32(ta + 96, v[3]);
      tmem_ld_wait();
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl->tempty[buf]);
      const int tile = t0 + it;
      const int64_t j = (int64_t)tile * BM + quarter * 32 + lane;  // this thread's centroid
      const bool jv = j < C;
      if (MODE == 1) {
        uint32_t *dst = gmax + ((int64_t)rb * G + tile * 4 + quarter) * BN + half * 128;
#pragma unroll
        for (int ch = 0; ch < 4; ch++) {
          uint32_t mine = 0;
#pragma unroll
          for (int c = 0; c < 32; c++) {
            uint32_t k = jv ? fkey(__uint_as_float(v[ch][c])) : 0u;
            uint32_t m = redux_max(k);
            if (c == lane) mine = m;
          }
          dst[ch * 32 + lane] = mine;
        }
      } else if (MODE == 3) {
        // diagnostic: raw scores [R x C]
#pragma unroll
        for (int ch = 0; ch < 4; ch++) {
#pragma unroll
          for (int c = 0; c < 32; c++) {
            const int row = rb * BN + half * 128 + ch * 32 + c;
            if (jv && row < R) reinterpret_cast<float *>(cand)[(int64_t)row * C + j] = __uint_as_float(v[ch][c]);
          }
        }
      } else {
#pragma unroll
        for (int ch = 0; ch < 4; ch++) {
#pragma unroll
          for (int c = 0; c < 32; c++) {
            const int n = half * 128 + ch * 32 + c;
            const float sc = __uint_as_float(v[ch][c]);
            if (jv && rb * BN + n < R && fkey(sc) >= ctl->thr[n]) {
              const int row = rb * BN + n;
              const int pos = atomicAdd(&cnt[row], 1);
              if (pos < CAPG) cand[(int64_t)row * CAPG + pos] = comp_key(sc, (int32_t)j);
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

// tau_r = kappa_c-th largest group maximum of row r over one part of the groups;
// the parts combine by max (each part's value is itself a valid lower bound).
__global__ void __launch_bounds__(128)
k_topc_tau(const uint32_t *__restrict__ gmax, int G, int gpart, int R, int kc, uint32_t *__restrict__ tau) {
  extern __shared__ uint32_t top[];  // [kc][128]
  const int rb = blockIdx.x >> 1, n = (blockIdx.x & 1) * 128 + threadIdx.x;
  const int row = rb * BN + n;
  const int tid = threadIdx.x;
  for (int i = 0; i < kc; i++) top[i * 128 + tid] = 0u;
  const int g0 = blockIdx.y * gpart, g1 = min(G, g0 + gpart);
  const uint32_t *src = gmax + (int64_t)rb * G * BN + n;
  uint32_t last = 0u;
  for (int g = g0; g < g1; g++) {
    const uint32_t x = src[(int64_t)g * BN];
    if (x > last) {
      int i = kc - 1;
      while (i > 0 && top[(i - 1) * 128 + tid] < x) {
        top[i * 128 + tid] = top[(i - 1) * 128 + tid];
        i--;
      }
      top[i * 128 + tid] = x;
      last = top[(kc - 1) * 128 + tid];
    }
  }
  if (row < R && last) atomicMax(&tau[row], last);
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
  return (size_t)(rbs * ntiles * 4 * tc::BN);
}

tachiom_status launch_topc_tc(const Index &ix, const __nv_bfloat16 *rows, int nrows, int kc, float margin,
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
  k_topc_tc<1><<<grid, THREADS, SMEM_BYTES, s>>>(mA, mB, ix.C, nrows, ntiles, per, G, gmax, nullptr, 0.f, nullptr,
                                                  nullptr, flags);
  TLAUNCH();
  TCUDA(cudaMemsetAsync(tau, 0, (size_t)nrows * 4, s));
  const int parts = std::max(1, std::min(8, G / std::max(1, 64 * kc)));
  const int gpart = (G + parts - 1) / parts;
  TCUDA(cudaFuncSetAttribute(k_topc_tau, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_KC * 128 * 4));
  k_topc_tau<<<dim3(rbs * 2, parts), 128, (size_t)kc * 128 * 4, s>>>(gmax, G, gpart, nrows, kc, tau);
  TLAUNCH();
  TCUDA(cudaMemsetAsync(cnt, 0, (size_t)nrows * 4, s));
  k_topc_tc<2><<<grid, THREADS, SMEM_BYTES, s>>>(mA, mB, ix.C, nrows, ntiles, per, G, nullptr, tau, margin, cnt,
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
                                                               nullptr, nullptr, 0.f, nullptr,
                                                               reinterpret_cast<uint64_t *>(out), flags);
  TLAUNCH();
  return TACHIOM_OK;
}

}  // namespace tachiom

extern "C" int tachiom_tc_available(void) { return tachiom::topc_tc_supported(); }
