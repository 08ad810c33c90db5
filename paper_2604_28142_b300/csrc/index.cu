// Index residency: validation, inverted-list construction, device copies.
//
// The inverted list L_j holds the ids of the documents that have a token
// assigned to centroid c_j (Sec. 2.2, "Index Structure"); each list is kept
// deduplicated and in ascending doc order so that a gather range [r0, r0+R)
// of documents is one contiguous slice of every list.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "tachiom_internal.cuh"

namespace tachiom {

static thread_local std::string g_err;

void set_error(const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}

tachiom_status fail(tachiom_status st, const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

// Gather ranges: a range is a block of consecutive document ids; the offset
// table gives the slice of every list that starts at a range boundary, and the
// gather finds finer cuts by binary search inside a slice. The ranges are sized
// so that a 32-token query with kappa_c = 40 has about kRangeEntries of its list
// entries in one range when its tokens hit lists of the token-weighted length
// Lw = sum_j n_j |L_j| / T (the gather merges consecutive ranges into one piece
// of work when a query's entries are sparser than that), and the table is kept
// below the size of the lists themselves. Document offsets inside a range must
// fit 20 bits.
constexpr int64_t kRangeEntries = 2048;
constexpr int64_t kRangeDocsMax = 1 << 20;

__global__ void k_widen_bf16(const uint16_t *__restrict__ in, float *__restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __uint_as_float(((uint32_t)in[i]) << 16);
}

__global__ void k_round_bf16(const float *__restrict__ in, __nv_bfloat16 *__restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16_rn(in[i]);
}

// max_j ||c_j|| and max_j ||bf16(c_j) - c_j|| (slightly rounded up)
__global__ void k_row_norm_max(const float *__restrict__ c, const __nv_bfloat16 *__restrict__ cb, int64_t C,
                               unsigned *__restrict__ out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < C;
       j += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f, e = 0.f;
    for (int k = 0; k < DIM; k++) {
      const float x = c[j * DIM + k], d = __bfloat162float(cb[j * DIM + k]) - x;
      s = fmaf(x, x, s);
      e = fmaf(d, d, e);
    }
    // non-negative floats order as uints
    atomicMax(out, __float_as_uint(sqrtf(s) * (1.f + ldexpf(1.f, -12))));
    atomicMax(out + 1, __float_as_uint(sqrtf(e) * (1.f + ldexpf(1.f, -12))));
  }
}

static void free_index(Index *ix) {
  if (!ix) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ix->device);
  for (auto &kv : ix->ws) ws_destroy(kv.second);
  ix->ws.clear();
  void *ptrs[] = {ix->cent_f32, ix->cent_bf16, ix->cent_e4m3, ix->cent_inv_sc, ix->cent_type, ix->doc_off, ix->tok_cid, ix->codes,
                  ix->rnorm, ix->codebooks, ix->doc_xe, ix->cbk_h16, ix->cbk_err2, ix->list_off,
                  ix->list_doc, ix->list_roff};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  cudaSetDevice(prev);
  delete ix;
}

template <typename T>
static tachiom_status dalloc(Index *ix, T **p, size_t n) {
  size_t bytes = n * sizeof(T);
  if (bytes == 0) bytes = sizeof(T);
  cudaError_t e = cudaMalloc((void **)p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(TACHIOM_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  ix->device_bytes += bytes;
  return TACHIOM_OK;
}

template <typename T>
static tachiom_status upload(Index *ix, T **p, const T *h, size_t n) {
  tachiom_status st = dalloc(ix, p, n);
  if (st) return st;
  if (n) TCUDA(cudaMemcpy(*p, h, n * sizeof(T), cudaMemcpyHostToDevice));
  return TACHIOM_OK;
}

static tachiom_status validate(const tachiom_index_desc *d) {
  if (!d) return fail(TACHIOM_ERR_INVALID, "desc is NULL");
  if (d->dim != DIM) return fail(TACHIOM_ERR_INVALID, "dim must be 128 (got %d)", d->dim);
  if (d->n_centroids < 1 || d->n_centroids >= (1LL << 31))
    return fail(TACHIOM_ERR_INVALID, "n_centroids out of range");
  if (d->n_docs < 1 || d->n_docs >= (1LL << 31)) return fail(TACHIOM_ERR_INVALID, "n_docs out of range");
  if (d->n_tokens < 0) return fail(TACHIOM_ERR_INVALID, "n_tokens < 0");
  if (d->pq_m != 8 && d->pq_m != 16 && d->pq_m != 32)
    return fail(TACHIOM_ERR_INVALID, "pq_m must be 8, 16 or 32 (got %d)", d->pq_m);
  if (d->pq_nbits != 8) return fail(TACHIOM_ERR_INVALID, "pq_nbits must be 8");
  if (d->centroid_dtype != TACHIOM_DTYPE_F32 && d->centroid_dtype != TACHIOM_DTYPE_BF16)
    return fail(TACHIOM_ERR_INVALID, "unknown centroid_dtype %d", d->centroid_dtype);
  if (!d->centroids || !d->doc_offsets || !d->pq_codebooks)
    return fail(TACHIOM_ERR_INVALID, "NULL centroids, doc_offsets or pq_codebooks");
  if (d->n_tokens > 0 && (!d->token_centroid || !d->pq_codes))
    return fail(TACHIOM_ERR_INVALID, "NULL token_centroid or pq_codes");
  const int64_t *off = d->doc_offsets;
  if (off[0] != 0) return fail(TACHIOM_ERR_INVALID, "doc_offsets[0] != 0");
  for (int64_t i = 0; i < d->n_docs; i++)
    if (off[i + 1] < off[i]) return fail(TACHIOM_ERR_INVALID, "doc_offsets not monotone at doc %lld", (long long)i);
  if (off[d->n_docs] != d->n_tokens)
    return fail(TACHIOM_ERR_INVALID, "doc_offsets[n_docs] (%lld) != n_tokens (%lld)",
                (long long)off[d->n_docs], (long long)d->n_tokens);
  for (int64_t t = 0; t < d->n_tokens; t++) {
    int32_t j = d->token_centroid[t];
    if (j < 0 || j >= d->n_centroids)
      return fail(TACHIOM_ERR_INVALID, "token_centroid[%lld] = %d out of [0, C)", (long long)t, j);
  }
  return TACHIOM_OK;
}

}  // namespace tachiom

using namespace tachiom;

extern "C" tachiom_status tachiom_index_load(const tachiom_index_desc *desc, int cuda_device,
                                             tachiom_index **out) {
  if (!out) return fail(TACHIOM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  tachiom_status st = validate(desc);
  if (st) return st;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cuda_device < 0 || cuda_device >= ndev) {
    cudaGetLastError();
    return fail(TACHIOM_ERR_CUDA, "CUDA device %d not available", cuda_device);
  }
  int prev = 0;
  cudaGetDevice(&prev);
  TCUDA(cudaSetDevice(cuda_device));

  Index *ix = new (std::nothrow) Index();
  if (!ix) return fail(TACHIOM_ERR_OOM, "host allocation failed");
  ix->device = cuda_device;
  ix->C = desc->n_centroids;
  ix->D = desc->n_docs;
  ix->T = desc->n_tokens;
  ix->M = desc->pq_m;
  ix->ds = DIM / desc->pq_m;
  ix->cdtype = desc->centroid_dtype;

  // ---- inverted lists on the host: count (centroid, doc) pairs once per doc,
  //      then fill in doc order, which leaves every list sorted ascending.
  const int64_t C = ix->C, D = ix->D, T = ix->T;
  std::vector<int64_t> loff(C + 1, 0);
  std::vector<int32_t> last(C, -1);
  const int64_t *doff = desc->doc_offsets;
  const int32_t *cid = desc->token_centroid;
  for (int64_t d = 0; d < D; d++)
    for (int64_t t = doff[d]; t < doff[d + 1]; t++) {
      int32_t j = cid[t];
      if (last[j] != (int32_t)d) { last[j] = (int32_t)d; loff[j + 1]++; }
    }
  for (int64_t j = 0; j < C; j++) loff[j + 1] += loff[j];
  ix->n_list = loff[C];
  if (ix->n_list >= (1LL << 31)) {
    delete ix;
    cudaSetDevice(prev);
    return fail(TACHIOM_ERR_CAPACITY, "more than 2^31 (doc, centroid) list entries");
  }
  std::vector<int32_t> ldoc((size_t)ix->n_list);
  {
    std::vector<int64_t> fill(loff.begin(), loff.end() - 1);
    std::fill(last.begin(), last.end(), -1);
    for (int64_t d = 0; d < D; d++)
      for (int64_t t = doff[d]; t < doff[d + 1]; t++) {
        int32_t j = cid[t];
        if (last[j] != (int32_t)d) { last[j] = (int32_t)d; ldoc[fill[j]++] = (int32_t)d; }
      }
  }
  // range size from the token-weighted list length
  {
    std::vector<int64_t> ntokj(C, 0);
    for (int64_t t = 0; t < T; t++) ntokj[cid[t]]++;
    double lw = 0.0;
    for (int64_t j = 0; j < C; j++) lw += (double)ntokj[j] * (double)(loff[j + 1] - loff[j]);
    lw = T > 0 ? lw / (double)T : 0.0;
    const double entries = (double)MAX_NTOK * 40.0 * lw;
    int64_t nr = (int64_t)std::ceil(entries / (double)kRangeEntries);
    nr = std::max<int64_t>(nr, (D + kRangeDocsMax - 1) / kRangeDocsMax);
    const int64_t nr_cap = std::max<int64_t>(1, std::max<int64_t>(ix->n_list, 16LL << 20) / std::max<int64_t>(1, C)) - 1;
    nr = std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(nr, nr_cap), D));
    int64_t rd = (D + nr - 1) / nr;
    if (rd > kRangeDocsMax) rd = kRangeDocsMax;
    ix->range_docs = (int)rd;
    ix->n_ranges = (int)((D + rd - 1) / rd);
  }
  // range offsets: roff[j][r] = position in L_j of the first doc >= r * R
  const int64_t RD = ix->range_docs;
  const int nr1 = ix->n_ranges + 1;
  std::vector<int32_t> roff((size_t)C * nr1);
  for (int64_t j = 0; j < C; j++) {
    int64_t p = loff[j], e = loff[j + 1];
    int32_t *row = &roff[(size_t)j * nr1];
    for (int r = 0; r < nr1; r++) {
      int64_t bound = (int64_t)r * RD;
      while (p < e && ldoc[p] < bound) p++;
      row[r] = (int32_t)(p - loff[j]);
    }
  }

  // ---- device copies
  const size_t cn = (size_t)C * DIM;
#define TRY(x)                 \
  do {                         \
    st = (x);                  \
    if (st) goto fail_;        \
  } while (0)
  TRY(dalloc(ix, &ix->cent_f32, cn));
  TRY(dalloc(ix, &ix->cent_bf16, cn));
  if (desc->centroid_dtype == TACHIOM_DTYPE_BF16) {
    // the BF16 values are stored as given and widened exactly for FP32 use
    st = TACHIOM_OK;
    if (cudaMemcpy(ix->cent_bf16, desc->centroids, cn * 2, cudaMemcpyHostToDevice) != cudaSuccess) {
      st = fail(TACHIOM_ERR_CUDA, "centroid upload failed");
      goto fail_;
    }
    k_widen_bf16<<<1024, 256>>>((const uint16_t *)ix->cent_bf16, ix->cent_f32, (int64_t)cn);
  } else {
    if (cudaMemcpy(ix->cent_f32, desc->centroids, cn * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
      st = fail(TACHIOM_ERR_CUDA, "centroid upload failed");
      goto fail_;
    }
    k_round_bf16<<<1024, 256>>>(ix->cent_f32, ix->cent_bf16, (int64_t)cn);
  }
  {
    unsigned *dmax = nullptr;
    TRY(dalloc(ix, &dmax, 2));
    cudaMemset(dmax, 0, 8);
    k_row_norm_max<<<(unsigned)((C + 255) / 256 < 4096 ? (C + 255) / 256 : 4096), 256>>>(ix->cent_f32, ix->cent_bf16,
                                                                                          C, dmax);
    unsigned hm[2] = {0, 0};
    cudaError_t e = cudaMemcpy(hm, dmax, 8, cudaMemcpyDeviceToHost);
    const unsigned hmax = hm[0];
    cudaFree(dmax);
    ix->device_bytes -= 8;
    if (e != cudaSuccess) {
      st = fail(TACHIOM_ERR_CUDA, "centroid norm pass failed: %s", cudaGetErrorString(e));
      goto fail_;
    }
    float f, g;
    memcpy(&f, &hmax, 4);
    memcpy(&g, &hm[1], 4);
    ix->cnorm_max = f;
    ix->cerr_max = g;
  }
  // the E4M3 operand of the FP8 step (a): a power-of-two scale per centroid
  TRY(dalloc(ix, &ix->cent_e4m3, cn));
  TRY(dalloc(ix, &ix->cent_inv_sc, (size_t)C));
  TRY(launch_cent_e4m3(*ix, 0));
  if (desc->centroid_type) TRY(upload(ix, &ix->cent_type, desc->centroid_type, (size_t)C));
  TRY(upload(ix, &ix->doc_off, desc->doc_offsets, (size_t)D + 1));
  TRY(upload(ix, &ix->tok_cid, desc->token_centroid, (size_t)T));
  TRY(upload(ix, &ix->codes, desc->pq_codes, (size_t)T * ix->M));
  {
    size_t nb = (size_t)ix->M * 256 * ix->ds;
    TRY(upload(ix, &ix->codebooks, desc->pq_codebooks, nb));
  }
  if (desc->residual_norms) {
    TRY(upload(ix, &ix->rnorm, desc->residual_norms, (size_t)T));
  } else {
    std::vector<uint16_t> ones((size_t)T, (uint16_t)0x3C00u);  // fp16 1.0
    TRY(upload(ix, &ix->rnorm, ones.data(), (size_t)T));
  }
  TRY(dalloc(ix, &ix->doc_xe, (size_t)D));
  TRY(dalloc(ix, &ix->cbk_h16, (size_t)ix->M * 256 * ix->ds));
  TRY(dalloc(ix, &ix->cbk_err2, (size_t)ix->M * 256));
  TRY(launch_decode_tables(*ix, 0));
  TRY(upload(ix, &ix->list_off, loff.data(), (size_t)C + 1));
  TRY(upload(ix, &ix->list_doc, ldoc.data(), (size_t)ix->n_list));
  TRY(upload(ix, &ix->list_roff, roff.data(), roff.size()));
#undef TRY
  if (cudaDeviceSynchronize() != cudaSuccess) {
    st = fail(TACHIOM_ERR_CUDA, "index load: %s", cudaGetErrorString(cudaGetLastError()));
    goto fail_;
  }
  cudaSetDevice(prev);
  *out = reinterpret_cast<tachiom_index *>(ix);
  return TACHIOM_OK;
fail_:
  free_index(ix);
  cudaSetDevice(prev);
  return st;
}

extern "C" tachiom_status tachiom_index_free(tachiom_index *index) {
  free_index(reinterpret_cast<Index *>(index));
  return TACHIOM_OK;
}

extern "C" tachiom_status tachiom_index_info(const tachiom_index *index, int64_t *n_centroids,
                                             int64_t *n_docs, int64_t *n_tokens,
                                             int64_t *n_list_entries, int32_t *pq_m,
                                             int64_t *device_bytes) {
  const Index *ix = reinterpret_cast<const Index *>(index);
  if (!ix) return fail(TACHIOM_ERR_INVALID, "index is NULL");
  if (n_centroids) *n_centroids = ix->C;
  if (n_docs) *n_docs = ix->D;
  if (n_tokens) *n_tokens = ix->T;
  if (n_list_entries) *n_list_entries = ix->n_list;
  if (pq_m) *pq_m = ix->M;
  if (device_bytes) *device_bytes = (int64_t)ix->device_bytes;
  return TACHIOM_OK;
}

extern "C" tachiom_status tachiom_index_lists(const tachiom_index *index, int64_t *h_off,
                                              int32_t *h_docs) {
  const Index *ix = reinterpret_cast<const Index *>(index);
  if (!ix || !h_off || !h_docs) return fail(TACHIOM_ERR_INVALID, "NULL argument");
  int prev = 0;
  cudaGetDevice(&prev);
  TCUDA(cudaSetDevice(ix->device));
  TCUDA(cudaMemcpy(h_off, ix->list_off, (ix->C + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
  if (ix->n_list)
    TCUDA(cudaMemcpy(h_docs, ix->list_doc, ix->n_list * sizeof(int32_t), cudaMemcpyDeviceToHost));
  cudaSetDevice(prev);
  return TACHIOM_OK;
}

extern "C" const char *tachiom_last_error(void) { return g_err.c_str(); }
extern "C" const char *tachiom_version(void) { return "tachiom-b300 0.1 (sm_103a)"; }
