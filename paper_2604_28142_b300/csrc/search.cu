// Search orchestration: per-stream scratch, launch plans, and the C-ABI
// entry points that run steps (a)-(d) of Sec. 2.2 on one stream.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "tachiom_internal.cuh"

namespace tachiom {

// ---- workspace ---------------------------------------------------------------------
void ws_destroy(Workspace *w) {
  if (!w) return;
  for (void *p : w->blocks) cudaFree(p);
  if (w->h_meta) cudaFreeHost(w->h_meta);
  if (w->h_rows) cudaFreeHost(w->h_rows);
  if (w->h_out_ids) cudaFreeHost(w->h_out_ids);
  if (w->h_out_s) cudaFreeHost(w->h_out_s);
  if (w->meta_done) cudaEventDestroy(w->meta_done);
  delete w;
}

tachiom_status ws_get(Index *ix, cudaStream_t stream, Workspace **out) {
  std::lock_guard<std::mutex> g(ix->mu);
  auto it = ix->ws.find(stream);
  if (it != ix->ws.end()) {
    *out = it->second;
    return TACHIOM_OK;
  }
  Workspace *w = new Workspace();
  w->stream = stream;
  w->device = ix->device;
  if (cudaEventCreateWithFlags(&w->meta_done, cudaEventDisableTiming) != cudaSuccess) {
    delete w;
    return fail(TACHIOM_ERR_CUDA, "cudaEventCreate failed");
  }
  if (cudaMalloc(&w->d_flags, 4) != cudaSuccess || cudaMemset(w->d_flags, 0, 4) != cudaSuccess) {
    cudaGetLastError();
    ws_destroy(w);
    return fail(TACHIOM_ERR_OOM, "cudaMalloc of the status word failed");
  }
  w->blocks.push_back(w->d_flags);
  ix->ws[stream] = w;
  *out = w;
  return TACHIOM_OK;
}

void ws_release(Index *ix, cudaStream_t stream) {
  std::lock_guard<std::mutex> g(ix->mu);
  auto it = ix->ws.find(stream);
  if (it == ix->ws.end()) return;
  ws_destroy(it->second);
  ix->ws.erase(it);
}

struct Need {
  int64_t nq = 0, rows = 0, kc = 0, kd = 0, split_entries = 0, pool = 0, gmax = 0;
};

// (Re)allocate the device scratch for a batch. Growth synchronises the stream
// first, so memory still in use by earlier work on it is never freed early.
static tachiom_status ws_reserve(Index *ix, Workspace *w, const Need &n) {
  bool grow = n.nq > w->cap_q || n.rows > w->cap_rows || n.kc > w->cap_kc || n.kd > w->cap_kd ||
              n.split_entries > w->cap_split_entries || n.pool > w->cap_pool || n.gmax > w->cap_gmax;
  if (!grow) return TACHIOM_OK;
  TCUDA(cudaStreamSynchronize(w->stream));
  for (void *p : w->blocks)
    if (p != w->d_flags) cudaFree(p);
  w->blocks.clear();
  w->blocks.push_back(w->d_flags);
  int64_t nq = std::max<int64_t>(n.nq, w->cap_q), rows = std::max<int64_t>(n.rows, w->cap_rows);
  int64_t kc = std::max<int64_t>(n.kc, w->cap_kc), kd = std::max<int64_t>(n.kd, w->cap_kd);
  int64_t se = std::max<int64_t>(n.split_entries, w->cap_split_entries);
  int64_t pl = std::max<int64_t>(n.pool, w->cap_pool);
  int64_t gm = std::max<int64_t>(n.gmax, w->cap_gmax);
  const int groups = refine_groups(32);  // the largest group count of any pq_m
  auto al = [&](void **p, size_t bytes) -> tachiom_status {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(TACHIOM_ERR_OOM, "scratch allocation of %zu bytes failed", bytes);
    }
    w->blocks.push_back(*p);
    return TACHIOM_OK;
  };
  tachiom_status st;
#define AL(ptr, bytes)                               \
  if ((st = al((void **)&(ptr), (size_t)(bytes)))) { \
    w->cap_q = w->cap_rows = 0;                      \
    return st;                                       \
  }
  AL(w->d_meta, (5 * nq + 2) * 4);
  AL(w->d_rows_f32, rows * DIM * 4);
  AL(w->d_rows_bf16, rows * DIM * 2);
  AL(w->d_rows_f8, rows * DIM);
  AL(w->d_inv_sq, rows * 4);
  AL(w->d_split, se * 8);
  AL(w->d_split_cnt, (se + rows) * 4);
  AL(w->d_top_ids, rows * kc * 4);
  AL(w->d_top_s, rows * kc * 4);
  AL(w->d_pool, pl * 8);
  AL(w->d_pool_n, (int64_t)nq * 64 * 4);
  AL(w->d_gmax, gm * 4);
  AL(w->d_tau, rows * 4);
  AL(w->d_margin, rows * 4);
  AL(w->d_glist, (int64_t)topc_tc_glist_elems((int)rows) * 4);
  AL(w->d_gcount, rows * 4);
  AL(w->d_lossy, rows * 4);
  AL(w->d_cand, nq * kd * 4);
  AL(w->d_cand_s, nq * kd * 4);
  AL(w->d_ncand, nq * 4);
  AL(w->d_part, nq * groups * kd * 4);
  AL(w->d_win, nq * kd * 4);
  AL(w->d_win_slot, nq * kd * 4);
  AL(w->d_thr, nq * kd * 32 * 4);
  AL(w->d_wl, nq * (int64_t)WL_PER_QUERY * 8);
  AL(w->d_wl_n, 16);
  AL(w->d_emx, nq * kd * 32 * 4);
  AL(w->d_wovf, nq * kd * 4);
  AL(w->d_out_ids, nq * kd * 4);
  AL(w->d_out_s, nq * kd * 4);
#undef AL
  w->cap_q = nq;
  w->cap_rows = rows;
  w->cap_kc = kc;
  w->cap_kd = kd;
  w->cap_split_entries = se;
  w->cap_pool = pl;
  w->cap_gmax = gm;
  return TACHIOM_OK;
}

static tachiom_status host_reserve(Workspace *w, int64_t meta_ints) {
  if (meta_ints <= w->cap_meta) return TACHIOM_OK;
  if (w->h_meta) {
    cudaEventSynchronize(w->meta_done);
    cudaFreeHost(w->h_meta);
  }
  w->h_meta = nullptr;
  w->cap_meta = 0;
  if (cudaMallocHost((void **)&w->h_meta, (size_t)meta_ints * 4) != cudaSuccess) {
    cudaGetLastError();
    return fail(TACHIOM_ERR_OOM, "pinned host allocation failed");
  }
  w->cap_meta = meta_ints;
  return TACHIOM_OK;
}

// ---- plan -----------------------------------------------------------------------------
struct Plan {
  int splits;   // centroid slices of step (a)
  int capout;   // survivors a slice hands to the merge, per row
};

static int sm_count(int dev) {
  static int cached[64] = {0};
  if (dev >= 0 && dev < 64 && cached[dev]) return cached[dev];
  int n = 148;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  if (dev >= 0 && dev < 64) cached[dev] = n;
  return n;
}

static Plan make_plan(const Index &ix, int rows, int kc, int precision, int plan_id) {
  Plan p;
  const int sms = sm_count(ix.device);
  const int row_tiles = (rows + 31) / 32;
  // enough CTAs for two waves, each slice at least one 128-centroid tile
  int splits = std::max(1, (2 * sms + row_tiles - 1) / row_tiles);
  int64_t max_splits = (ix.C + 127) / 128;
  splits = (int)std::min<int64_t>(splits, max_splits);
  p.capout = kc + 64;
  splits = std::min(splits, std::max(1, 16384 / p.capout));
  const int forced = plan_id >= 0 ? ((plan_id >> 4) & 0xfffff) : 0;  // bits 4-23
  if (forced > 0) {
    // an explicit slice count of the FP32 scan (autotuner)
    splits = std::max(1, std::min(forced, (int)std::min<int64_t>(max_splits, 16384 / p.capout)));
  }
  p.splits = splits;
  (void)precision;
  return p;
}

struct Batch {
  int nq = 0;
  int rows = 0;
  int max_k = 0;
  int64_t total_k = 0;
};

static tachiom_status check_batch(const int32_t *h_ntok, const int32_t *h_k, int nq, int kd_limit,
                                  Batch *b) {
  if (nq < 0) return fail(TACHIOM_ERR_INVALID, "nq < 0");
  if (nq > 0 && !h_ntok) return fail(TACHIOM_ERR_INVALID, "h_ntok is NULL");
  b->nq = nq;
  int64_t rows = 0, tk = 0;
  int mk = 0;
  for (int i = 0; i < nq; i++) {
    if (h_ntok[i] < 1 || h_ntok[i] > MAX_NTOK)
      return fail(TACHIOM_ERR_INVALID, "ntok[%d] = %d out of [1, %d]", i, h_ntok[i], MAX_NTOK);
    rows += h_ntok[i];
    if (h_k) {
      if (h_k[i] < 1 || (kd_limit > 0 && h_k[i] > kd_limit))
        return fail(TACHIOM_ERR_INVALID, "k[%d] = %d out of [1, kappa_d]", i, h_k[i]);
      tk += h_k[i];
      mk = std::max(mk, h_k[i]);
    }
  }
  if (rows > (1 << 30) || tk > (1LL << 31) - 1) return fail(TACHIOM_ERR_CAPACITY, "batch too large");
  b->rows = (int)rows;
  b->total_k = tk;
  b->max_k = mk;
  return TACHIOM_OK;
}

static tachiom_status check_params(const tachiom_search_params *p) {
  if (!p) return fail(TACHIOM_ERR_INVALID, "params is NULL");
  if (p->kappa_c < 1 || p->kappa_c > MAX_KC)
    return fail(TACHIOM_ERR_INVALID, "kappa_c = %d out of [1, %d]", p->kappa_c, MAX_KC);
  if (p->kappa_d < 0 || p->kappa_d > MAX_KD)
    return fail(TACHIOM_ERR_INVALID, "kappa_d = %d out of [0, %d]", p->kappa_d, MAX_KD);
  if (p->precision != TACHIOM_PREC_FP32 && p->precision != TACHIOM_PREC_BF16 && p->precision != TACHIOM_PREC_FP8)
    return fail(TACHIOM_ERR_INVALID, "unknown precision %d", p->precision);
  if (!(p->rescore_margin == p->rescore_margin) || p->rescore_margin > 64.f)
    return fail(TACHIOM_ERR_INVALID, "rescore_margin out of range");
  return TACHIOM_OK;
}

static int resolve_kd(const tachiom_search_params *p, int max_k) {
  if (p->kappa_d > 0) return p->kappa_d;
  return std::min(MAX_KD, std::max(1000, 4 * max_k));
}

// upload qoff | koff | k | ntok through pinned staging
// qoff [nq+1] | koff [nq+1] | k [nq] | ntok [nq] | kappa_d of each query [nq]
static tachiom_status upload_meta(Workspace *w, const tachiom_search_params *p, const int32_t *h_ntok,
                                  const int32_t *h_k, int nq) {
  tachiom_status st = host_reserve(w, 5 * (int64_t)nq + 2);
  if (st) return st;
  TCUDA(cudaEventSynchronize(w->meta_done));
  int32_t *m = w->h_meta;
  m[0] = 0;
  m[nq + 1] = 0;
  for (int i = 0; i < nq; i++) {
    m[i + 1] = m[i] + h_ntok[i];
    int k = h_k ? h_k[i] : 0;
    m[nq + 2 + i] = m[nq + 1 + i] + k;
    m[2 * nq + 2 + i] = k;
    m[3 * nq + 2 + i] = h_ntok[i];
    m[4 * nq + 2 + i] = resolve_kd(p, k);  // per query, so a result never depends on its batch
  }
  TCUDA(cudaMemcpyAsync(w->d_meta, m, (size_t)(5 * nq + 2) * 4, cudaMemcpyHostToDevice, w->stream));
  TCUDA(cudaEventRecord(w->meta_done, w->stream));
  return TACHIOM_OK;
}

static bool use_tc(const tachiom_search_params *p) {
  return (p->precision == TACHIOM_PREC_BF16 || p->precision == TACHIOM_PREC_FP8) && topc_tc_supported();
}
static bool use_fp8(const tachiom_search_params *p) { return p->precision == TACHIOM_PREC_FP8 && topc_tc_supported(); }
// the E4M3 repair window as a multiple of the rigorous bound (1: rigorous)
constexpr float kFp8DefaultLambda = 0.1f;
static float fp8_lambda(const tachiom_search_params *p) {
  return p->rescore_margin > 0.f ? p->rescore_margin : kFp8DefaultLambda;
}

// plan_id >= 0 overrides the library's choices (all choices give the same results):
//   bits 0-1  step (a) kernel: 0 default (2), 1 single-pass tensor-core scan with per-row
//             selection in the epilogue, 2 tensor-core group maxima + exact rescoring of the
//             kept groups, 3 FP32 CUDA-core scan
//   bits 2-3  step (c) kernel: 0 default (3), 1 tensor-core centroid term + lookup tables, then the
//             FP32 window, 2 FP32 refine only, 3 decode + tensor cores, then the FP32 window
//   bits 4-23 slices of the FP32 scan (0: default)
//   bit 24    step (b): every document range cut into pieces of at most 256 list entries, the
//             path the gather takes for a range whose entries exceed its buffers (default:
//             pieces only where a range does not fit)
//   bit 25    step (c), decode path: the window rescored over every (query token, document
//             token) pair in FP32 (default: only the pairs that can hold a maximum)
//   bits 26-28 step (b): range groups per query (0: the default, about 8 CTAs per SM over the
//             batch; g: 2 g groups, within the selection's capacity)
enum { SCAN_DEFAULT = 0, SCAN_TC1 = 1, SCAN_TC2 = 2, SCAN_F32 = 3 };
constexpr int32_t PLAN_GATHER_SPLIT = 1 << 24;
constexpr int32_t PLAN_WINDOW_ALL = 1 << 25;
static bool gather_split(const tachiom_search_params *p) { return p->plan_id >= 0 && (p->plan_id & PLAN_GATHER_SPLIT); }
static int gather_groups_of(const tachiom_search_params *p) { return p->plan_id >= 0 ? (p->plan_id >> 26) & 7 : 0; }
enum { REFINE_DEFAULT = 0, REFINE_TC = 1, REFINE_F32 = 2, REFINE_DEC = 3 };

static int scan_kind(const tachiom_search_params *p) {
  const int forced = p->plan_id >= 0 ? (p->plan_id & 3) : SCAN_DEFAULT;
  if (!use_tc(p)) return SCAN_F32;
  if (forced == SCAN_F32) return SCAN_F32;
  if (forced == SCAN_TC1 && p->kappa_c <= topc_tc1_max_kc() && !use_fp8(p)) return SCAN_TC1;
  return SCAN_TC2;
}

static int refine_kind(const tachiom_search_params *p) {
  const int forced = p->plan_id >= 0 ? ((p->plan_id >> 2) & 3) : REFINE_DEFAULT;
  if (!use_tc(p)) return REFINE_F32;
  if (forced == REFINE_F32 || forced == REFINE_TC) return forced;
  return REFINE_DEC;
}

// scratch sizes of step (a) for a batch
static void need_topc(const Index &ix, const tachiom_search_params *p, int rows, const Plan &plan, Need *n) {
  const int kind = scan_kind(p);
  if (kind == SCAN_TC1) {
    n->split_entries = (int64_t)rows * topc_tc1_splits(ix, rows) * topc_tc1_capout();
  } else if (kind == SCAN_TC2) {
    n->split_entries = rows;
    n->gmax = (int64_t)topc_tc_gmax_elems(ix, rows);
  } else {
    n->split_entries = (int64_t)rows * plan.splits * plan.capout;
  }
}

// step (a) into w->d_top_ids / d_top_s
static tachiom_status run_topc(Index *ix, Workspace *w, const tachiom_search_params *p, const float *rows,
                               int nrows, const Plan &plan) {
  const int kc = p->kappa_c;
  tachiom_status st;
  const int kind = scan_kind(p);
  if (kind == SCAN_TC1) {
    // one pass, per-row running top-kappa_c in the epilogue
    if ((st = launch_quantize_rows(*ix, rows, w->d_rows_bf16, nrows, w->d_margin, w->stream))) return st;
    const int splits = topc_tc1_splits(*ix, nrows);
    if ((st = launch_topc_tc1(*ix, w->d_rows_bf16, nrows, kc, w->d_margin, w->d_split, w->d_split_cnt, w->d_flags,
                              w->stream)))
      return st;
    return launch_topc_merge(*ix, rows, nrows, kc, splits, topc_tc1_capout(), w->d_split, w->d_split_cnt, w->d_margin, 1,
                             w->d_top_ids, w->d_top_s, w->d_flags, w->stream);
  }
  if (kind == SCAN_TC2) {
    // tensor-core sample pass, emission of the candidates above each row's threshold, exact FP32
    // top-kappa_c of the candidates
    const bool f8 = use_fp8(p);
    if (f8) {
      if ((st = launch_quantize_e4m3(*ix, rows, nrows, w->d_rows_f8, w->d_inv_sq, fp8_lambda(p), w->d_margin,
                                     w->stream)))
        return st;
    } else if ((st = launch_quantize_rows(*ix, rows, w->d_rows_bf16, nrows, w->d_margin, w->stream))) {
      return st;
    }
    const void *rq = f8 ? (const void *)w->d_rows_f8 : (const void *)w->d_rows_bf16;
    if ((st = launch_topc_tc(*ix, rq, w->d_inv_sq, f8, rows, nrows, kc, w->d_margin,
                             reinterpret_cast<float *>(w->d_gmax), w->d_glist, w->d_gcount, w->d_lossy, w->d_top_ids,
                             w->d_top_s, w->d_flags, w->stream)))
      return st;
    return launch_topc_rescue(*ix, rows, nrows, kc, w->d_lossy, w->d_top_ids, w->d_top_s, w->stream);
  }
  if ((st = launch_topc_f32(*ix, rows, nrows, kc, plan.splits, plan.capout, w->d_split, w->d_split_cnt,
                            w->d_flags, w->stream)))
    return st;
  return launch_topc_merge(*ix, rows, nrows, kc, plan.splits, plan.capout, w->d_split, w->d_split_cnt, nullptr, 0,
                           w->d_top_ids, w->d_top_s, w->d_flags, w->stream);
}

// Bound on |tensor-core centroid term - FP32 centroid term| for one (query token,
// document token): the query split q_hi + q_lo leaves 2^-18 |q_k| per component,
// the bf16 table is exact when the centroids are stored in bf16 (a rounded
// copy otherwise: 2^-9); the bound used is 16x those for the accumulation.
static float refine_tc_delta(const Index &ix) {
  const float rel = ix.cdtype == TACHIOM_DTYPE_BF16 ? ldexpf(1.f, -14) : ldexpf(1.f, -5);
  return rel * ix.cnorm_max;
}

// steps (c)-(d): FP32 refine, or the tensor-core refine plus the FP32 repair of the
// top-k window, into the caller's outputs
static tachiom_status run_refine(Index *ix, Workspace *w, const tachiom_search_params *p, const float *queries,
                                 int nq, const int32_t *cand, int kd, int32_t *out_ids, float *out_s,
                                 cudaStream_t stream) {
  tachiom_status st;
  const int rk = refine_kind(p);
  if (rk == REFINE_DEC) {
    float *sa = w->d_part, *da = w->d_part + (int64_t)nq * kd;  // consumed before the FP32 pass reuses d_part
    if ((st = launch_refine_dec(*ix, queries, w->d_meta, nq, cand, kd, sa, da, w->d_thr, w->d_flags, stream)))
      return st;
    if ((st = launch_refine_window_b(*ix, w->d_meta, nq, cand, kd, sa, da, w->d_win, w->d_win_slot, stream)))
      return st;
    if (p->plan_id >= 0 && (p->plan_id & PLAN_WINDOW_ALL)) {
      // every pair of the window's documents in FP32
      if ((st = launch_refine_win(*ix, queries, w->d_meta, nq, w->d_win, kd, w->d_part, w->d_flags, stream)))
        return st;
    } else {
      // the window's documents: the decode pass again, and the FP32 path's numbers for the pairs
      // that can hold a maximum
      WinScratch ws{w->d_wl, w->d_wl_n, (int)std::min<int64_t>((int64_t)nq * WL_PER_QUERY, INT32_MAX), w->d_emx,
                    w->d_wovf};
      if ((st = launch_refine_dec_win(*ix, queries, w->d_meta, nq, w->d_win, w->d_win_slot, kd, w->d_thr,
                                      w->d_part, ws, w->d_flags, stream)))
        return st;
      // the documents whose pairs did not fit the list (normally none): every pair in FP32
      if ((st = launch_refine_win_only(*ix, queries, w->d_meta, nq, w->d_win, kd, w->d_wovf, w->d_part, w->d_flags,
                                       stream)))
        return st;
    }
    return launch_final_topk(*ix, w->d_meta, nq, w->d_win, kd, w->d_part, out_ids, out_s, stream);
  } else if (rk == REFINE_TC) {
    if ((st = launch_refine_tc(*ix, queries, w->d_meta, nq, cand, kd, w->d_part, w->d_flags, stream))) return st;
    if ((st = launch_refine_window(*ix, w->d_meta, nq, cand, kd, w->d_part, refine_tc_delta(*ix), w->d_win,
                                   stream)))
      return st;
    cand = w->d_win;
  }
  if ((st = launch_refine(*ix, queries, w->d_meta, nq, cand, kd, w->d_part, w->d_flags, stream))) return st;
  return launch_final_topk(*ix, w->d_meta, nq, cand, kd, w->d_part, out_ids, out_s, stream);
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

static tachiom_status search_device(Index *ix, const tachiom_search_params *p, const float *d_queries,
                                    const int32_t *h_ntok, const int32_t *h_k, int nq, int32_t *d_out_ids,
                                    float *d_out_scores, cudaStream_t stream, Workspace **wout) {
  tachiom_status st;
  if ((st = check_params(p))) return st;
  Batch b;
  if ((st = check_batch(h_ntok, h_k, nq, 0, &b))) return st;
  if (nq > 0 && !h_k) return fail(TACHIOM_ERR_INVALID, "h_k is NULL");
  const int kd = resolve_kd(p, b.max_k);
  if (b.max_k > kd) return fail(TACHIOM_ERR_INVALID, "k (%d) > kappa_d (%d)", b.max_k, kd);
  if (nq > 0 && (!d_queries || !d_out_ids || !d_out_scores))
    return fail(TACHIOM_ERR_INVALID, "NULL device buffer");
  Workspace *w;
  if ((st = ws_get(ix, stream, &w))) return st;
  if (wout) *wout = w;
  if (nq == 0) return TACHIOM_OK;
  Plan plan = make_plan(*ix, b.rows, p->kappa_c, p->precision, p->plan_id);
  Need n;
  n.nq = nq;
  n.rows = b.rows;
  n.kc = p->kappa_c;
  n.kd = kd;
  need_topc(*ix, p, b.rows, plan, &n);
  n.pool = (int64_t)gather_pool_elems(*ix, nq, kd);
  if ((st = ws_reserve(ix, w, n))) return st;
  if ((st = upload_meta(w, p, h_ntok, h_k, nq))) return st;
  if ((st = run_topc(ix, w, p, d_queries, b.rows, plan))) return st;
  if ((st = launch_gather(*ix, w->d_meta, nq, w->d_top_ids, w->d_top_s, p->kappa_c, kd, w->d_pool, w->d_pool_n,
                          gather_split(p), gather_groups_of(p), w->d_flags, stream)))
    return st;
  if ((st = launch_select_kd(*ix, w->d_meta, nq, kd, w->d_pool, w->d_pool_n, gather_groups_of(p), w->d_cand,
                             w->d_cand_s, w->d_ncand, stream)))
    return st;
  return run_refine(ix, w, p, d_queries, nq, w->d_cand, kd, d_out_ids, d_out_scores, stream);
}

}  // namespace tachiom

using namespace tachiom;

static Index *as_index(tachiom_index *p) { return reinterpret_cast<Index *>(p); }

extern "C" tachiom_status tachiom_search(tachiom_index *index, const tachiom_search_params *params,
                                         const float *d_queries, const int32_t *h_ntok, const int32_t *h_k,
                                         int32_t nq, int32_t *d_out_ids, float *d_out_scores, void *stream) {
  Index *ix = as_index(index);
  if (!ix) return fail(TACHIOM_ERR_INVALID, "index is NULL");
  DeviceGuard g(ix->device);
  return search_device(ix, params, d_queries, h_ntok, h_k, nq, d_out_ids, d_out_scores,
                       (cudaStream_t)stream, nullptr);
}

extern "C" tachiom_status tachiom_search_host(tachiom_index *index, const tachiom_search_params *params,
                                              const float *h_queries, const int32_t *h_ntok,
                                              const int32_t *h_k, int32_t nq, int32_t *h_out_ids,
                                              float *h_out_scores, void *stream) {
  Index *ix = as_index(index);
  if (!ix) return fail(TACHIOM_ERR_INVALID, "index is NULL");
  DeviceGuard g(ix->device);
  tachiom_status st;
  if ((st = check_params(params))) return st;
  Batch b;
  if ((st = check_batch(h_ntok, h_k, nq, 0, &b))) return st;
  if (nq == 0) return TACHIOM_OK;
  if (!h_queries || !h_k || !h_out_ids || !h_out_scores) return fail(TACHIOM_ERR_INVALID, "NULL host buffer");
  cudaStream_t s = (cudaStream_t)stream;
  Workspace *w;
  if ((st = ws_get(ix, s, &w))) return st;
  const int kd = resolve_kd(params, b.max_k);
  Plan plan = make_plan(*ix, b.rows, params->kappa_c, params->precision, params->plan_id);
  Need n;
  n.nq = nq;
  n.rows = b.rows;
  n.kc = params->kappa_c;
  n.kd = std::max<int64_t>(kd, (b.total_k + nq - 1) / nq + 1);
  need_topc(*ix, params, b.rows, plan, &n);
  n.pool = (int64_t)gather_pool_elems(*ix, nq, kd);
  if ((st = ws_reserve(ix, w, n))) return st;
  if (b.total_k > w->cap_q * w->cap_kd) return fail(TACHIOM_ERR_CAPACITY, "sum(k) beyond scratch");
  // pinned staging for queries and results
  int64_t qbytes = (int64_t)b.rows * DIM;
  if (qbytes > w->cap_h_rows) {
    TCUDA(cudaStreamSynchronize(s));
    if (w->h_rows) cudaFreeHost(w->h_rows);
    w->h_rows = nullptr;
    w->cap_h_rows = 0;
    if (cudaMallocHost((void **)&w->h_rows, (size_t)qbytes * 4) != cudaSuccess) {
      cudaGetLastError();
      return fail(TACHIOM_ERR_OOM, "pinned host allocation failed");
    }
    w->cap_h_rows = qbytes;
  }
  if (b.total_k > w->cap_h_out) {
    TCUDA(cudaStreamSynchronize(s));
    if (w->h_out_ids) cudaFreeHost(w->h_out_ids);
    if (w->h_out_s) cudaFreeHost(w->h_out_s);
    w->h_out_ids = nullptr;
    w->h_out_s = nullptr;
    w->cap_h_out = 0;
    if (cudaMallocHost((void **)&w->h_out_ids, (size_t)b.total_k * 4) != cudaSuccess ||
        cudaMallocHost((void **)&w->h_out_s, (size_t)b.total_k * 4) != cudaSuccess) {
      cudaGetLastError();
      return fail(TACHIOM_ERR_OOM, "pinned host allocation failed");
    }
    w->cap_h_out = b.total_k;
  }
  TCUDA(cudaStreamSynchronize(s));
  memcpy(w->h_rows, h_queries, (size_t)qbytes * 4);
  TCUDA(cudaMemcpyAsync(w->d_rows_f32, w->h_rows, (size_t)qbytes * 4, cudaMemcpyHostToDevice, s));
  if ((st = search_device(ix, params, w->d_rows_f32, h_ntok, h_k, nq, w->d_out_ids, w->d_out_s, s, nullptr)))
    return st;
  TCUDA(cudaMemcpyAsync(w->h_out_ids, w->d_out_ids, (size_t)b.total_k * 4, cudaMemcpyDeviceToHost, s));
  TCUDA(cudaMemcpyAsync(w->h_out_s, w->d_out_s, (size_t)b.total_k * 4, cudaMemcpyDeviceToHost, s));
  TCUDA(cudaStreamSynchronize(s));
  memcpy(h_out_ids, w->h_out_ids, (size_t)b.total_k * 4);
  memcpy(h_out_scores, w->h_out_s, (size_t)b.total_k * 4);
  return TACHIOM_OK;
}

extern "C" tachiom_status tachiom_top_centroids(tachiom_index *index, const tachiom_search_params *params,
                                                const float *d_rows, int32_t nrows, int32_t *d_top_ids,
                                                float *d_top_scores, void *stream) {
  Index *ix = as_index(index);
  if (!ix) return fail(TACHIOM_ERR_INVALID, "index is NULL");
  DeviceGuard g(ix->device);
  tachiom_status st;
  if ((st = check_params(params))) return st;
  if (nrows < 0) return fail(TACHIOM_ERR_INVALID, "nrows < 0");
  if (nrows == 0) return TACHIOM_OK;
  if (!d_rows || !d_top_ids || !d_top_scores) return fail(TACHIOM_ERR_INVALID, "NULL device buffer");
  cudaStream_t s = (cudaStream_t)stream;
  Workspace *w;
  if ((st = ws_get(ix, s, &w))) return st;
  Plan plan = make_plan(*ix, nrows, params->kappa_c, params->precision, params->plan_id);
  Need n;
  n.nq = 1;
  n.rows = nrows;
  n.kc = params->kappa_c;
  n.kd = 1;
  need_topc(*ix, params, nrows, plan, &n);
  if ((st = ws_reserve(ix, w, n))) return st;
  if ((st = run_topc(ix, w, params, d_rows, nrows, plan))) return st;
  TCUDA(cudaMemcpyAsync(d_top_ids, w->d_top_ids, (size_t)nrows * params->kappa_c * 4, cudaMemcpyDeviceToDevice, s));
  TCUDA(cudaMemcpyAsync(d_top_scores, w->d_top_s, (size_t)nrows * params->kappa_c * 4, cudaMemcpyDeviceToDevice, s));
  return TACHIOM_OK;
}

extern "C" tachiom_status tachiom_gather(tachiom_index *index, const tachiom_search_params *params,
                                         const float *d_queries, const int32_t *h_ntok, int32_t nq,
                                         const int32_t *d_top_ids, int32_t *d_cand_ids, float *d_cand_scores,
                                         int32_t *d_ncand, void *stream) {
  Index *ix = as_index(index);
  if (!ix) return fail(TACHIOM_ERR_INVALID, "index is NULL");
  DeviceGuard g(ix->device);
  tachiom_status st;
  if ((st = check_params(params))) return st;
  Batch b;
  if ((st = check_batch(h_ntok, nullptr, nq, 0, &b))) return st;
  if (nq == 0) return TACHIOM_OK;
  if (!d_queries || !d_top_ids || !d_cand_ids || !d_cand_scores || !d_ncand)
    return fail(TACHIOM_ERR_INVALID, "NULL device buffer");
  const int kd = resolve_kd(params, 0);
  cudaStream_t s = (cudaStream_t)stream;
  Workspace *w;
  if ((st = ws_get(ix, s, &w))) return st;
  Need n;
  n.nq = nq;
  n.rows = b.rows;
  n.kc = params->kappa_c;
  n.kd = kd;
  n.pool = (int64_t)gather_pool_elems(*ix, nq, kd);
  if ((st = ws_reserve(ix, w, n))) return st;
  if ((st = upload_meta(w, params, h_ntok, nullptr, nq))) return st;
  if ((st = launch_score_pairs(*ix, d_queries, b.rows, d_top_ids, params->kappa_c, w->d_top_ids, w->d_top_s,
                                w->d_flags, s)))
    return st;
  if ((st = launch_gather(*ix, w->d_meta, nq, w->d_top_ids, w->d_top_s, params->kappa_c, kd, w->d_pool, w->d_pool_n,
                          gather_split(params), gather_groups_of(params), w->d_flags, s)))
    return st;
  return launch_select_kd(*ix, w->d_meta, nq, kd, w->d_pool, w->d_pool_n, gather_groups_of(params), d_cand_ids,
                          d_cand_scores, d_ncand, s);
}

extern "C" tachiom_status tachiom_refine(tachiom_index *index, const tachiom_search_params *params,
                                         const float *d_queries, const int32_t *h_ntok, const int32_t *h_k,
                                         int32_t nq, const int32_t *d_cand_ids, int32_t *d_out_ids,
                                         float *d_out_scores, void *stream) {
  Index *ix = as_index(index);
  if (!ix) return fail(TACHIOM_ERR_INVALID, "index is NULL");
  DeviceGuard g(ix->device);
  tachiom_status st;
  if ((st = check_params(params))) return st;
  Batch b;
  if ((st = check_batch(h_ntok, h_k, nq, 0, &b))) return st;
  if (nq == 0) return TACHIOM_OK;
  if (!h_k) return fail(TACHIOM_ERR_INVALID, "h_k is NULL");
  const int kd = resolve_kd(params, b.max_k);
  if (b.max_k > kd) return fail(TACHIOM_ERR_INVALID, "k > kappa_d");
  if (!d_queries || !d_cand_ids || !d_out_ids || !d_out_scores) return fail(TACHIOM_ERR_INVALID, "NULL device buffer");
  cudaStream_t s = (cudaStream_t)stream;
  Workspace *w;
  if ((st = ws_get(ix, s, &w))) return st;
  Need n;
  n.nq = nq;
  n.rows = b.rows;
  n.kc = params->kappa_c;
  n.kd = kd;
  if ((st = ws_reserve(ix, w, n))) return st;
  if ((st = upload_meta(w, params, h_ntok, h_k, nq))) return st;
  return run_refine(ix, w, params, d_queries, nq, d_cand_ids, kd, d_out_ids, d_out_scores, s);
}

extern "C" tachiom_status tachiom_centroid_interaction(tachiom_index *index, const tachiom_search_params *params,
                                                       const float *d_queries, const int32_t *h_ntok,
                                                       const int32_t *h_k, int32_t nq, const int32_t *d_cand_ids,
                                                       int32_t *d_out_ids, float *d_out_scores, void *stream) {
  Index *ix = as_index(index);
  if (!ix) return fail(TACHIOM_ERR_INVALID, "index is NULL");
  DeviceGuard g(ix->device);
  tachiom_status st;
  if ((st = check_params(params))) return st;
  Batch b;
  if ((st = check_batch(h_ntok, h_k, nq, 0, &b))) return st;
  if (nq == 0) return TACHIOM_OK;
  if (!h_k) return fail(TACHIOM_ERR_INVALID, "h_k is NULL");
  const int kd = resolve_kd(params, b.max_k);
  if (b.max_k > kd) return fail(TACHIOM_ERR_INVALID, "k > kappa_d");
  if (!d_queries || !d_cand_ids || !d_out_ids || !d_out_scores) return fail(TACHIOM_ERR_INVALID, "NULL device buffer");
  cudaStream_t s = (cudaStream_t)stream;
  Workspace *w;
  if ((st = ws_get(ix, s, &w))) return st;
  Need n;
  n.nq = nq;
  n.rows = b.rows;
  n.kc = params->kappa_c;
  n.kd = kd;
  if ((st = ws_reserve(ix, w, n))) return st;
  if ((st = upload_meta(w, params, h_ntok, h_k, nq))) return st;
  // the FP32 refine with every residual norm taken as 0, then the top-k
  if ((st = launch_refine(*ix, d_queries, w->d_meta, nq, d_cand_ids, kd, w->d_part, w->d_flags, s, true))) return st;
  return launch_final_topk(*ix, w->d_meta, nq, d_cand_ids, kd, w->d_part, d_out_ids, d_out_scores, s);
}

extern "C" tachiom_status tachiom_stream_status(tachiom_index *index, void *stream, uint32_t *h_flags) {
  Index *ix = as_index(index);
  if (!ix || !h_flags) return fail(TACHIOM_ERR_INVALID, "NULL argument");
  DeviceGuard g(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  Workspace *w;
  tachiom_status st;
  if ((st = ws_get(ix, s, &w))) return st;
  TCUDA(cudaStreamSynchronize(s));
  TCUDA(cudaMemcpy(h_flags, w->d_flags, 4, cudaMemcpyDeviceToHost));
  TCUDA(cudaMemset(w->d_flags, 0, 4));
  return TACHIOM_OK;
}

extern "C" tachiom_status tachiom_debug_tc_scores(tachiom_index *index, const float *d_rows, int32_t nrows,
                                                  float *d_out, void *stream) {
  Index *ix = as_index(index);
  if (!ix) return fail(TACHIOM_ERR_INVALID, "index is NULL");
  if (!topc_tc_supported()) return fail(TACHIOM_ERR_INVALID, "no tensor-core step (a) on this device");
  if (nrows < 0 || (nrows > 0 && (!d_rows || !d_out))) return fail(TACHIOM_ERR_INVALID, "bad arguments");
  if (nrows == 0) return TACHIOM_OK;
  DeviceGuard g(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  Workspace *w;
  tachiom_status st;
  if ((st = ws_get(ix, s, &w))) return st;
  Need n;
  n.nq = 1;
  n.rows = nrows;
  n.kc = 1;
  n.kd = 1;
  if ((st = ws_reserve(ix, w, n))) return st;
  if ((st = launch_quantize_bf16(d_rows, w->d_rows_bf16, (int64_t)nrows * DIM, s))) return st;
  return launch_topc_tc_raw(*ix, w->d_rows_bf16, nullptr, false, nrows, d_out, w->d_flags, s);
}

extern "C" tachiom_status tachiom_debug_wait_timeout(tachiom_index *index, int32_t timeout_us, void *stream) {
  Index *ix = as_index(index);
  if (!ix) return fail(TACHIOM_ERR_INVALID, "index is NULL");
  if (!topc_tc_supported()) return fail(TACHIOM_ERR_INVALID, "no tensor-core step (a) on this device");
  if (timeout_us < 1 || timeout_us > 2000000) return fail(TACHIOM_ERR_INVALID, "timeout_us out of [1, 2e6]");
  DeviceGuard g(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  Workspace *w;
  tachiom_status st;
  if ((st = ws_get(ix, s, &w))) return st;
  Need n;
  n.nq = 1;
  n.rows = 256;
  n.kc = 1;
  n.kd = 1;
  n.gmax = (int64_t)topc_tc_gmax_elems(*ix, 256);
  if ((st = ws_reserve(ix, w, n))) return st;
  return launch_topc_tc_wait_test(*ix, w->d_rows_bf16, (uint64_t)timeout_us * 1000ull,
                                  reinterpret_cast<float *>(w->d_gmax), w->d_flags, s);
}

extern "C" tachiom_status tachiom_debug_tc_scores_fp8(tachiom_index *index, const float *d_rows, int32_t nrows,
                                                      float *d_out, float *d_margins, void *stream) {
  Index *ix = as_index(index);
  if (!ix) return fail(TACHIOM_ERR_INVALID, "index is NULL");
  if (!topc_tc_supported()) return fail(TACHIOM_ERR_INVALID, "no tensor-core step (a) on this device");
  if (nrows < 0 || (nrows > 0 && (!d_rows || !d_out))) return fail(TACHIOM_ERR_INVALID, "bad arguments");
  if (nrows == 0) return TACHIOM_OK;
  DeviceGuard g(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  Workspace *w;
  tachiom_status st;
  if ((st = ws_get(ix, s, &w))) return st;
  Need n;
  n.nq = 1;
  n.rows = nrows;
  n.kc = 1;
  n.kd = 1;
  if ((st = ws_reserve(ix, w, n))) return st;
  if ((st = launch_quantize_e4m3(*ix, d_rows, nrows, w->d_rows_f8, w->d_inv_sq, 1.f, w->d_margin, s))) return st;
  if ((st = launch_topc_tc_raw(*ix, w->d_rows_f8, w->d_inv_sq, true, nrows, d_out, w->d_flags, s))) return st;
  if (d_margins) TCUDA(cudaMemcpyAsync(d_margins, w->d_margin, (size_t)nrows * 4, cudaMemcpyDeviceToDevice, s));
  return TACHIOM_OK;
}

extern "C" tachiom_status tachiom_debug_refine_scores(tachiom_index *index, const tachiom_search_params *params,
                                                     const float *d_queries, const int32_t *h_ntok, int32_t nq,
                                                     const int32_t *d_cand_ids, float *d_scores, float *d_bounds,
                                                     void *stream) {
  Index *ix = as_index(index);
  if (!ix) return fail(TACHIOM_ERR_INVALID, "index is NULL");
  DeviceGuard g(ix->device);
  tachiom_status st;
  if ((st = check_params(params))) return st;
  if (params->kappa_d < 1) return fail(TACHIOM_ERR_INVALID, "kappa_d must be given");
  Batch b;
  if ((st = check_batch(h_ntok, nullptr, nq, 0, &b))) return st;
  if (nq == 0) return TACHIOM_OK;
  if (!d_queries || !d_cand_ids || !d_scores) return fail(TACHIOM_ERR_INVALID, "NULL device buffer");
  const int kd = params->kappa_d;
  cudaStream_t s = (cudaStream_t)stream;
  Workspace *w;
  if ((st = ws_get(ix, s, &w))) return st;
  Need n;
  n.nq = nq;
  n.rows = b.rows;
  n.kc = params->kappa_c;
  n.kd = kd;
  if ((st = ws_reserve(ix, w, n))) return st;
  if ((st = upload_meta(w, params, h_ntok, nullptr, nq))) return st;
  if (use_tc(params) && refine_kind(params) == REFINE_DEC) {
    // approximate S and its per-document bound
    float *bounds = d_bounds ? d_bounds : w->d_part;
    return launch_refine_dec(*ix, d_queries, w->d_meta, nq, d_cand_ids, kd, d_scores, bounds, w->d_thr, w->d_flags,
                             s);
  } else if (use_tc(params)) {
    if ((st = launch_refine_tc(*ix, d_queries, w->d_meta, nq, d_cand_ids, kd, w->d_part, w->d_flags, s))) return st;
  } else {
    if ((st = launch_refine(*ix, d_queries, w->d_meta, nq, d_cand_ids, kd, w->d_part, w->d_flags, s))) return st;
  }
  return launch_refine_sum(*ix, w->d_meta, nq, d_cand_ids, kd, w->d_part, d_scores, s);
}

// ---- CUDA graphs of a fixed batch shape --------------------------------------------------
namespace tachiom {
struct Graph {
  Index *ix = nullptr;
  cudaStream_t stream = nullptr;  // capture stream; its workspace holds the graph's scratch
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  float *d_in = nullptr;
  int32_t *d_ids = nullptr;
  float *d_s = nullptr;
  int64_t rows = 0, total_k = 0;
};

// Warm-up input of a graph's sizing run: components uniform in [-1/2, 1/2) from a hash of their
// index (splitmix64), so the run takes the path an ordinary batch takes. All-zero rows would tie
// every score at every stage, the slowest input of the cascade.
__global__ void k_fill_warmup(float *__restrict__ x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = (uint64_t)i + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    x[i] = (float)(z >> 40) * (1.f / 16777216.f) - 0.5f;
  }
}

static void graph_free(Graph *g) {
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->d_in) cudaFree(g->d_in);
  if (g->d_ids) cudaFree(g->d_ids);
  if (g->d_s) cudaFree(g->d_s);
  if (g->stream) {
    ws_release(g->ix, g->stream);
    cudaStreamDestroy(g->stream);
  }
  delete g;
}
}  // namespace tachiom

extern "C" tachiom_status tachiom_graph_create(tachiom_index *index, const tachiom_search_params *params,
                                               const int32_t *h_ntok, const int32_t *h_k, int32_t nq,
                                               tachiom_graph **out) {
  Index *ix = as_index(index);
  if (!ix || !out) return fail(TACHIOM_ERR_INVALID, "NULL argument");
  *out = nullptr;
  tachiom_status st;
  if ((st = check_params(params))) return st;
  Batch b;
  if ((st = check_batch(h_ntok, h_k, nq, 0, &b))) return st;
  if (nq < 1 || !h_k) return fail(TACHIOM_ERR_INVALID, "a graph needs at least one query and its k");
  DeviceGuard dg(ix->device);
  Graph *g = new Graph();
  g->ix = ix;
  g->rows = b.rows;
  g->total_k = b.total_k;
  if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&g->d_in, (size_t)b.rows * DIM * 4) != cudaSuccess ||
      cudaMalloc(&g->d_ids, (size_t)b.total_k * 4) != cudaSuccess ||
      cudaMalloc(&g->d_s, (size_t)b.total_k * 4) != cudaSuccess) {
    cudaGetLastError();
    graph_free(g);
    return fail(TACHIOM_ERR_OOM, "graph buffers");
  }
  k_fill_warmup<<<256, 256, 0, g->stream>>>(g->d_in, (int64_t)b.rows * DIM);
  // first run outside the capture: scratch grows, kernel attributes are set
  if ((st = search_device(ix, params, g->d_in, h_ntok, h_k, nq, g->d_ids, g->d_s, g->stream, nullptr))) {
    graph_free(g);
    return st;
  }
  if (cudaStreamSynchronize(g->stream) != cudaSuccess) {
    graph_free(g);
    return fail(TACHIOM_ERR_CUDA, "graph warm-up failed: %s", cudaGetErrorString(cudaGetLastError()));
  }
  if (cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    graph_free(g);
    return fail(TACHIOM_ERR_CUDA, "cudaStreamBeginCapture failed");
  }
  st = search_device(ix, params, g->d_in, h_ntok, h_k, nq, g->d_ids, g->d_s, g->stream, nullptr);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(g->stream, &graph);
  g->graph = graph;
  if (st || e != cudaSuccess) {
    cudaGetLastError();
    graph_free(g);
    return st ? st : fail(TACHIOM_ERR_CUDA, "capture failed: %s", cudaGetErrorString(e));
  }
  if (cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) {
    cudaGetLastError();
    graph_free(g);
    return fail(TACHIOM_ERR_CUDA, "cudaGraphInstantiate failed");
  }
  *out = reinterpret_cast<tachiom_graph *>(g);
  return TACHIOM_OK;
}

extern "C" tachiom_status tachiom_graph_launch(tachiom_graph *graph, const float *d_queries, int32_t *d_out_ids,
                                               float *d_out_scores, void *stream) {
  Graph *g = reinterpret_cast<Graph *>(graph);
  if (!g || !d_queries || !d_out_ids || !d_out_scores) return fail(TACHIOM_ERR_INVALID, "NULL argument");
  DeviceGuard dg(g->ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  TCUDA(cudaMemcpyAsync(g->d_in, d_queries, (size_t)g->rows * DIM * 4, cudaMemcpyDeviceToDevice, s));
  TCUDA(cudaGraphLaunch(g->exec, s));
  TCUDA(cudaMemcpyAsync(d_out_ids, g->d_ids, (size_t)g->total_k * 4, cudaMemcpyDeviceToDevice, s));
  TCUDA(cudaMemcpyAsync(d_out_scores, g->d_s, (size_t)g->total_k * 4, cudaMemcpyDeviceToDevice, s));
  return TACHIOM_OK;
}

extern "C" tachiom_status tachiom_graph_destroy(tachiom_graph *graph) {
  graph_free(reinterpret_cast<Graph *>(graph));
  return TACHIOM_OK;
}

// ---- autotuner ------------------------------------------------------------------------------
extern "C" tachiom_status tachiom_autotune(tachiom_index *index, const tachiom_search_params *params,
                                           const float *d_queries, const int32_t *h_ntok, const int32_t *h_k,
                                           int32_t nq, int32_t *best_plan, float *best_ms, void *stream) {
  Index *ix = as_index(index);
  if (!ix || !params || !best_plan) return fail(TACHIOM_ERR_INVALID, "NULL argument");
  tachiom_status st;
  if ((st = check_params(params))) return st;
  Batch b;
  if ((st = check_batch(h_ntok, h_k, nq, 0, &b))) return st;
  if (nq < 1 || !d_queries || !h_k) return fail(TACHIOM_ERR_INVALID, "autotuning needs a batch");
  DeviceGuard dg(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  int32_t *d_ids = nullptr;
  float *d_s = nullptr;
  if (cudaMalloc(&d_ids, (size_t)b.total_k * 4) != cudaSuccess || cudaMalloc(&d_s, (size_t)b.total_k * 4) != cudaSuccess) {
    cudaGetLastError();
    if (d_ids) cudaFree(d_ids);
    return fail(TACHIOM_ERR_OOM, "autotune buffers");
  }
  // candidate plans: step (a) kernel x step (c) kernel (x FP32 scan slices on the FP32 path)
  std::vector<int32_t> plans;
  const int tc = use_tc(params) ? 1 : 0;
  if (tc) {
    for (int sk : {SCAN_TC1, SCAN_TC2})
      for (int rk : {REFINE_DEC, REFINE_TC, REFINE_F32}) {
        if (sk == SCAN_TC1 && params->kappa_c > topc_tc1_max_kc()) continue;
        plans.push_back(sk | (rk << 2));
      }
    // the default kernels with other gather group counts (4, 8, 12 per query)
    for (int g : {2, 4, 6}) plans.push_back(SCAN_TC2 | (REFINE_DEC << 2) | (g << 26));
  } else {
    const int sms = sm_count(ix->device);
    const int row_tiles = (b.rows + 31) / 32;
    const int base = std::max(1, (2 * sms + row_tiles - 1) / row_tiles);
    for (int m : {1, 2, 4}) plans.push_back(SCAN_F32 | (REFINE_F32 << 2) | ((base * m / 2 > 0 ? base * m / 2 : 1) << 4));
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int32_t bestp = -1;
  for (int32_t pl : plans) {
    tachiom_search_params p = *params;
    p.plan_id = pl;
    // one untimed run (scratch, attributes), then the median of three timed runs
    if ((st = search_device(ix, &p, d_queries, h_ntok, h_k, nq, d_ids, d_s, s, nullptr))) break;
    float t[3];
    for (int r = 0; r < 3; r++) {
      cudaEventRecord(e0, s);
      if ((st = search_device(ix, &p, d_queries, h_ntok, h_k, nq, d_ids, d_s, s, nullptr))) break;
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&t[r], e0, e1);
    }
    if (st) break;
    std::sort(t, t + 3);
    if (t[1] < best) {
      best = t[1];
      bestp = pl;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(d_ids);
  cudaFree(d_s);
  if (st) return st;
  *best_plan = bestp;
  if (best_ms) *best_ms = best;
  return TACHIOM_OK;
}

extern "C" tachiom_status tachiom_debug_topc_groups(tachiom_index *index, const tachiom_search_params *params,
                                                   const float *d_rows, int32_t nrows, int32_t *h_groups) {
  Index *ix = as_index(index);
  if (!ix || !params || !h_groups) return fail(TACHIOM_ERR_INVALID, "NULL argument");
  tachiom_status st;
  if ((st = check_params(params))) return st;
  if (scan_kind(params) != SCAN_TC2) return fail(TACHIOM_ERR_INVALID, "not the candidate-emission path");
  if (nrows <= 0) return TACHIOM_OK;
  DeviceGuard g(ix->device);
  int32_t *ids = nullptr;
  float *sc = nullptr;
  if (cudaMalloc(&ids, (size_t)nrows * params->kappa_c * 4) != cudaSuccess ||
      cudaMalloc(&sc, (size_t)nrows * params->kappa_c * 4) != cudaSuccess) {
    cudaGetLastError();
    if (ids) cudaFree(ids);
    return fail(TACHIOM_ERR_OOM, "debug buffers");
  }
  st = tachiom_top_centroids(index, params, d_rows, nrows, ids, sc, nullptr);
  Workspace *w = nullptr;
  if (!st) st = ws_get(ix, nullptr, &w);
  if (!st && cudaMemcpy(h_groups, w->d_gcount, (size_t)nrows * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    st = fail(TACHIOM_ERR_CUDA, "copy failed");
  cudaFree(ids);
  cudaFree(sc);
  return st;
}
