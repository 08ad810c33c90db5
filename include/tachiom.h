/*
 * tachiom.h: C ABI of the B300 gather-and-refine scoring library.
 *
 * The library scores multivector (late-interaction) queries against an index
 * built the way TACHIOM (arXiv 2604.28142) builds one: per-token-type
 * centroids, the centroid id of every document token, PQ-coded normalised
 * residuals and their norms (Sec. 2.1, "Residuals Compression"; Sec. 2.2,
 * "Index Structure"). A search runs the four steps of Sec. 2.2 on one GPU:
 *
 *   (a) every query token against every centroid, keeping each token's
 *       kappa_c best (Sec. 2.2, Gather step 1; exact, not a graph search);
 *   (b) inverted-list gather and centroid-only late interaction,
 *       S~(q,d) = sum_i max_{j in Top_i : d in L_j} <q_i, c_j> (Gather steps
 *       2-4), truncated to the kappa_d best documents;
 *   (c) refinement of those candidates with the full MaxSim on centroid plus
 *       PQ-coded residual, S(q,d) = sum_i max_{t in d} (<q_i, c_a(t)> +
 *       rho_t <q_i, r^_t>), the residual term read from per-query lookup
 *       tables in the query-token-major layout (Sec. 2.2, Refine);
 *   (d) the k best documents by S.
 *
 * Conventions shared by every call:
 *   - Plain pointers and sizes only. "Host" pointers are read during the call
 *     and may be freed when it returns. "Device" pointers are CUDA device
 *     memory of the index's device, owned by the caller.
 *   - A `stream` argument is a cudaStream_t (NULL = the legacy default stream).
 *     Calls taking a stream are asynchronous on it: argument errors return
 *     synchronously; conditions found on the device (a capacity overflow
 *     that took the slow path, a row whose reduced-precision top-kappa_c was
 *     recomputed in FP32) are reported later by tachiom_stream_status.
 *   - Ties at every cut (kappa_c, kappa_d, k) are broken by the lower id.
 *   - A row of results that has fewer than k documents is padded with doc id
 *     -1 and score -inf.
 *   - Every call returns a tachiom_status; on failure tachiom_last_error()
 *     returns a message for the calling thread.
 *   - One index may be searched concurrently from several host threads on
 *     different streams; each stream gets its own scratch memory.
 */
#ifndef TACHIOM_H
#define TACHIOM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TACHIOM_OK = 0,
  TACHIOM_ERR_INVALID = 1,  /* bad argument or malformed index */
  TACHIOM_ERR_OOM = 2,      /* device or host allocation failed */
  TACHIOM_ERR_CUDA = 3,     /* a CUDA runtime call failed */
  TACHIOM_ERR_CAPACITY = 4, /* a size is beyond a compiled-in maximum */
  TACHIOM_ERR_TIMEOUT = 5,  /* a bounded device wait gave up */
  TACHIOM_ERR_BUSY = 6      /* the index is being freed */
} tachiom_status;

/* storage type of the centroid table */
enum { TACHIOM_DTYPE_F32 = 0, TACHIOM_DTYPE_BF16 = 1 };

/* arithmetic of step (a); steps (b)-(d) always accumulate in FP32 */
enum {
  TACHIOM_PREC_FP32 = 0, /* FP32 CUDA-core products: the plain comparator path */
  TACHIOM_PREC_BF16 = 1, /* BF16 tensor-core products with FP32 accumulation, then the
                            candidates near each row's kappa_c boundary rescored in FP32;
                            the window is the rigorous error bound, so the result is the
                            FP32 path's, bit for bit */
  TACHIOM_PREC_FP8 = 2   /* FP8-E4M3 tensor-core products (a power-of-two scale per query row
                            and per centroid) with FP32 accumulation, then the candidates in a
                            window of rescore_margin times the rigorous error bound rescored
                            in FP32 (rescore_margin >= 1: the FP32 path's result; below 1:
                            a narrower window, accuracy measured against the FP64 oracle) */
};

/* device status flags, OR-ed per stream since the last tachiom_stream_status */
enum {
  TACHIOM_FLAG_TOPC_RESCUED = 1u << 0,   /* a row's candidate buffer overflowed in step (a);
                                            that row was recomputed exactly */
  TACHIOM_FLAG_SELECT_TIES = 1u << 1,    /* reserved (no longer raised: the kappa_d selection
                                            orders equal scores by doc id in every case) */
  TACHIOM_FLAG_CAPACITY = 1u << 2,       /* a buffer overflow that could not be rescued: the
                                            affected query's result may be incomplete */
  TACHIOM_FLAG_BAD_INPUT = 1u << 3,      /* a device-side range check failed */
  TACHIOM_FLAG_TIMEOUT = 1u << 4         /* a bounded wait inside a kernel gave up; the
                                            results of that call are not valid */
};

typedef struct tachiom_index tachiom_index; /* opaque, owned by the library */

/* Index description. Every pointer is a HOST pointer read during
 * tachiom_index_load only; the library keeps its own device copies.
 * Layouts are row-major and packed.                                         */
typedef struct {
  int32_t dim;                 /* embedding dimension; must be 128 */
  int64_t n_centroids;         /* C >= 1 */
  int64_t n_docs;              /* D >= 1, D < 2^31 */
  int64_t n_tokens;            /* T = doc_offsets[D] */
  int32_t pq_m;                /* PQ subspaces M: 8, 16 or 32 (d/M dims each) */
  int32_t pq_nbits;            /* bits per code; must be 8 (256 codewords) */
  int32_t centroid_dtype;      /* TACHIOM_DTYPE_F32 or TACHIOM_DTYPE_BF16 */
  const void *centroids;       /* [C x dim] fp32, or bf16 bit patterns (uint16) */
  const int32_t *centroid_type;/* [C] token-type id of each centroid; may be NULL */
  const int64_t *doc_offsets;  /* [D+1] CSR over tokens: doc d owns [off[d], off[d+1]) */
  const int32_t *token_centroid;/* [T] centroid id a(t) of every token, in [0, C) */
  const float *pq_codebooks;   /* [M x 256 x dim/M] codewords of the normalised residual */
  const uint8_t *pq_codes;     /* [T x M] one byte per token and subspace */
  const uint16_t *residual_norms;/* [T] fp16 bit patterns of rho_t; NULL means rho_t = 1
                                    (the codes then encode the raw residual) */
} tachiom_index_desc;

/* Copy an index to `cuda_device` and build its inverted lists L_j (document
 * ids of the tokens assigned to c_j, Sec. 2.2 "Index Structure";
 * deduplicated, ascending). Validates the CSR and every id; on any failure
 * nothing is leaked and *out is left NULL. Blocking.                        */
tachiom_status tachiom_index_load(const tachiom_index_desc *desc, int cuda_device,
                                  tachiom_index **out);

/* Release an index and all scratch memory it allocated. The caller must have
 * synchronised every stream that used it. NULL is accepted.                */
tachiom_status tachiom_index_free(tachiom_index *index);

/* Read-only facts about a loaded index (any pointer may be NULL).          */
tachiom_status tachiom_index_info(const tachiom_index *index, int64_t *n_centroids,
                                  int64_t *n_docs, int64_t *n_tokens, int64_t *n_list_entries,
                                  int32_t *pq_m, int64_t *device_bytes);

/* Copy the inverted lists back to the host: off [C+1] int64, docs
 * [n_list_entries] int32 (host buffers owned by the caller). Blocking.     */
tachiom_status tachiom_index_lists(const tachiom_index *index, int64_t *h_off, int32_t *h_docs);

typedef struct {
  int32_t kappa_c;    /* centroids kept per query token, 1..128 */
  int32_t kappa_d;    /* candidates refined per query, 1..4096; 0 means max(1000, 4 max_k) capped
                         at 4096 */
  int32_t precision;  /* TACHIOM_PREC_* for step (a) */
  int32_t plan_id;    /* -1: the library's choice of kernels; >= 0: a plan from tachiom_autotune
                         (bits 0-1 step (a) kernel, 2-3 step (c) kernel, 4-23 FP32 scan slices,
                         24 small gather pieces, 25 FP32 window over every pair, 26-28 g: 2 g
                         gather range groups per query); every plan gives the same results */
  float rescore_margin; /* TACHIOM_PREC_FP8 only: the FP32 repair window of step (a) as a multiple
                           of the rigorous E4M3 error bound; <= 0 means 0.1 (about 4 standard
                           deviations of the typical error of unit-norm rows). Ignored otherwise. */
} tachiom_search_params;

/* The whole path, steps (a)-(d), for a batch of nq queries.
 *   d_queries  device fp32 [sum(ntok) x 128], query q's tokens at rows
 *              [sum_{p<q} ntok_p, +ntok_q); unit norm expected, not checked
 *   h_ntok     host int32 [nq], each 1..32
 *   h_k        host int32 [nq], each 1..kappa_d
 *   d_out_ids / d_out_scores  device int32 / fp32 [sum(k)], row q at
 *              [sum_{p<q} k_p, +k_q), sorted by (score desc, doc asc)
 * nq may be 0 (nothing is launched). Asynchronous on `stream`.             */
tachiom_status tachiom_search(tachiom_index *index, const tachiom_search_params *params,
                              const float *d_queries, const int32_t *h_ntok, const int32_t *h_k,
                              int32_t nq, int32_t *d_out_ids, float *d_out_scores, void *stream);

/* Same as tachiom_search with HOST queries and HOST outputs: the library copies
 * the queries in and the results out on `stream` (through pinned staging it
 * owns) and returns after the stream has finished the batch. Blocking.     */
tachiom_status tachiom_search_host(tachiom_index *index, const tachiom_search_params *params,
                                   const float *h_queries, const int32_t *h_ntok,
                                   const int32_t *h_k, int32_t nq, int32_t *h_out_ids,
                                   float *h_out_scores, void *stream);

/* ---- single steps, for replaying one step on given inputs ---- */

/* Step (a) alone (Sec. 2.2, Gather step 1, exhaustive): for each of nrows
 * device fp32 rows [nrows x 128], the kappa_c best centroids by (FP32 score
 * desc, id asc): d_top_ids int32 / d_top_scores fp32 [nrows x kappa_c].
 * With TACHIOM_PREC_BF16 the products run in BF16 and the result is rescored
 * in FP32, so the output is the FP32 path's. Asynchronous.                 */
tachiom_status tachiom_top_centroids(tachiom_index *index, const tachiom_search_params *params,
                                     const float *d_rows, int32_t nrows, int32_t *d_top_ids,
                                     float *d_top_scores, void *stream);

/* Step (b) alone (Sec. 2.2, Gather steps 2-4 and the kappa_d truncation) on
 * given top centroids. d_top_ids int32 [sum(ntok) x kappa_c] (entries < 0
 * are skipped; the FP32 scores are recomputed from the ids). Writes, per
 * query, the kappa_d best documents by (S~ desc, doc asc) to d_cand_ids
 * int32 / d_cand_scores fp32 [nq x kappa_d] (padded with -1 / -inf) and their
 * count to d_ncand int32 [nq]. Asynchronous.                                */
tachiom_status tachiom_gather(tachiom_index *index, const tachiom_search_params *params,
                              const float *d_queries, const int32_t *h_ntok, int32_t nq,
                              const int32_t *d_top_ids, int32_t *d_cand_ids,
                              float *d_cand_scores, int32_t *d_ncand, void *stream);

/* Steps (c)-(d) alone (Sec. 2.2, Refine; then top-k) on given candidates:
 * d_cand_ids int32 [nq x kappa_d] (entries < 0 are skipped), outputs as in
 * tachiom_search. Asynchronous.                                             */
tachiom_status tachiom_refine(tachiom_index *index, const tachiom_search_params *params,
                              const float *d_queries, const int32_t *h_ntok, const int32_t *h_k,
                              int32_t nq, const int32_t *d_cand_ids, int32_t *d_out_ids,
                              float *d_out_scores, void *stream);

/* Full centroid interaction (the variant of step (b)'s scoring that Sec. 2.2
 * contrasts with the Top_i-restricted one: every document token replaced by
 * its assigned centroid, the max over all of the document's tokens):
 *   S_ci(q, d) = sum_i max_{t in d} <q_i, c_a(t)>
 * for the documents of given candidate lists (for example step (b)'s
 * kappa_d candidates), then the k best by (S_ci desc, doc asc). Arguments,
 * layouts and padding as tachiom_refine; always FP32 (the refine kernel with
 * every residual norm taken as 0), whatever params->precision says; kappa_c
 * is not used. An empty document scores 0; an id outside [0, n_docs) raises
 * TACHIOM_FLAG_BAD_INPUT and scores 0. Asynchronous. */
tachiom_status tachiom_centroid_interaction(tachiom_index *index, const tachiom_search_params *params,
                                            const float *d_queries, const int32_t *h_ntok, const int32_t *h_k,
                                            int32_t nq, const int32_t *d_cand_ids, int32_t *d_out_ids,
                                            float *d_out_scores, void *stream);

/* tachiom_refine without allocating. The paper has no counterpart: this is an
 * interface for callers that cannot allocate device memory during a call, for
 * example a process whose device memory is handed out in advance by a
 * fixed-budget allocator, a plug-in living inside another framework's memory
 * pool, or a latency-critical thread that must not block in cudaMalloc (which
 * can synchronise the whole device). tachiom_refine takes its scratch from a
 * per-stream workspace that grows with cudaMalloc; this call instead uses one
 * static device array compiled into the library (2 MiB + 4 KiB, held on every
 * device that loads the library until the process exits) and one file-scope
 * host array for its per-query metadata, and calls no cudaMalloc, cudaFree,
 * pinned-host or heap allocation.
 *   Same arguments as tachiom_refine. It always scores in FP32 (step (c) of
 *   Sec. 2.2 with the lookup tables), whatever params->precision says, so its
 *   results equal tachiom_refine's FP32 results; with TACHIOM_PREC_BF16 they
 *   can differ from tachiom_refine's within the reduced-precision tolerance.
 *   Limits: nq <= 64 and params->kappa_d given explicitly in 1..1024; larger
 *   sizes return TACHIOM_ERR_CAPACITY with a message, and nothing is launched.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current. Every call shares the
 *   two arrays: calls whose work overlaps on the GPU (other streams, other
 *   host threads) race on them, so serialise them. Device-side range-check
 *   flags raised by this call go to a status word in the static array, read
 *   and cleared by tachiom_refine_noalloc_status (not by
 *   tachiom_stream_status). Asynchronous on `stream`.                        */
tachiom_status tachiom_refine_noalloc(tachiom_index *index, const tachiom_search_params *params,
                                      const float *d_queries, const int32_t *h_ntok,
                                      const int32_t *h_k, int32_t nq, const int32_t *d_cand_ids,
                                      int32_t *d_out_ids, float *d_out_scores, void *stream);

/* Synchronise `stream`, then return and clear the TACHIOM_FLAG_* bits that
 * tachiom_refine_noalloc calls raised on the index's device (a candidate id
 * out of [0, n_docs) gives TACHIOM_FLAG_BAD_INPUT and is scored 0). Copies
 * into the caller's variable and clears the word with cudaMemcpyAsync and
 * cudaMemsetAsync; allocates nothing. Blocking.                              */
tachiom_status tachiom_refine_noalloc_status(tachiom_index *index, void *stream, uint32_t *h_flags);

/* ---- continuous-batching request loop ----
 * A server owns n_slots CUDA streams. Requests (one query each: host fp32
 * [ntok x 128], its own k) are submitted from any host thread; a scheduler
 * thread forms batches from the queue in arrival order whenever a slot is
 * free and launches them, so requests that arrive while other batches run are
 * admitted as slots free up and their work overlaps on the device. A batch is
 * launched when it is full, when its oldest request has waited max_wait_us,
 * or at once when nothing else runs; it is held back while the scratch that
 * in-flight batches may use would exceed scratch_budget_bytes (0: no limit).
 * A request's result is the same bits alone and in any mix.              */
typedef struct {
  int32_t n_slots;              /* batches in flight at once, 1..64 */
  int32_t max_batch_queries;    /* queries per batch */
  int32_t max_batch_rows;       /* query tokens per batch, >= 32 */
  int32_t max_wait_us;          /* longest a queued request waits for a fuller batch */
  int64_t scratch_budget_bytes; /* device scratch all in-flight batches may use; 0 = unlimited */
} tachiom_server_config;

typedef struct {
  int64_t completed;   /* requests finished */
  int64_t batches;     /* batches launched and finished */
  double mean_batch;   /* queries per batch */
  double p50_ms, p95_ms, p99_ms; /* latency: submission to results on the host */
  double qps;          /* completed / (last completion - first submission) */
} tachiom_server_stats;

typedef struct tachiom_server tachiom_server;

tachiom_status tachiom_server_create(tachiom_index *index, const tachiom_search_params *params,
                                     const tachiom_server_config *cfg, tachiom_server **out);
/* Queue one query; *id receives its request id. The query is copied. */
tachiom_status tachiom_server_submit(tachiom_server *server, const float *h_query, int32_t ntok,
                                     int32_t k, uint64_t *id);
/* Wait up to timeout_ms (< 0: forever) for a request; copy its k ids and
 * scores to host buffers (may be NULL) and its latency in ms, then forget it.
 * TACHIOM_ERR_TIMEOUT if it has not finished in time (it stays queued). */
tachiom_status tachiom_server_wait(tachiom_server *server, uint64_t id, int32_t timeout_ms,
                                   int32_t *h_ids, float *h_scores, double *latency_ms);
tachiom_status tachiom_server_read_stats(tachiom_server *server, tachiom_server_stats *out);
/* Finish every queued and running request, then release the server. */
tachiom_status tachiom_server_destroy(tachiom_server *server);

/* ---- CUDA graphs and the autotuner ----
 * tachiom_graph_create captures the whole search for one batch shape (nq
 * queries with these token counts and k) into a CUDA graph, after one
 * uncaptured run that sizes its scratch; tachiom_graph_launch copies the
 * device queries in, replays the graph on `stream` and copies the results out
 * (same layouts as tachiom_search). Launches of one graph must not overlap.
 * Blocking create; asynchronous launch.                                     */
typedef struct tachiom_graph tachiom_graph;
tachiom_status tachiom_graph_create(tachiom_index *index, const tachiom_search_params *params,
                                    const int32_t *h_ntok, const int32_t *h_k, int32_t nq,
                                    tachiom_graph **out);
tachiom_status tachiom_graph_launch(tachiom_graph *graph, const float *d_queries, int32_t *d_out_ids,
                                    float *d_out_scores, void *stream);
tachiom_status tachiom_graph_destroy(tachiom_graph *graph);

/* Time every kernel choice for this batch (step (a): single-pass or two-pass
 * tensor-core scan, or FP32 scan slices; step (c): tensor-core refine with the
 * FP32 window, or FP32 refine; every choice returns the same results) and
 * return the fastest as a plan id for tachiom_search_params.plan_id, with its
 * median time in ms. Blocking.                                              */
tachiom_status tachiom_autotune(tachiom_index *index, const tachiom_search_params *params,
                                const float *d_queries, const int32_t *h_ntok, const int32_t *h_k,
                                int32_t nq, int32_t *best_plan, float *best_ms, void *stream);

/* The k best documents of the whole collection by the refined score of step
 * (c), S(q, d) = sum_i max_t (<q_i, c_a(t)> + rho_t <q_i, r^_t>) (Sec. 2.2,
 * Refine): the cascade with kappa_c = C and kappa_d = D. Every document is
 * scored by the refine (precision as in tachiom_refine; its top-k is exact in
 * both) in chunks of 4,096 per query; the running top-k per query is merged
 * on the host by (score desc, doc asc). d_queries: device fp32 [sum(ntok) x
 * 128]; h_ntok host [nq] (1..32), nq <= 4096, k in 1..1000; h_ids / h_scores:
 * host [nq x k] outputs, padded with (-1, -inf). Blocking.                  */
tachiom_status tachiom_exhaustive_topk(tachiom_index *index, int32_t precision, const float *d_queries,
                                       const int32_t *h_ntok, int32_t nq, int32_t k, int32_t *h_ids,
                                       float *h_scores, void *stream);

/* The candidate budgets by measurement (the paper tunes kappa_c and kappa_d on
 * a grid, Sec. 3): on the tuning queries, every (kappa_c, kappa_d) of the
 * grid (n_kc x n_kd <= 256 points, kappa_d >= k) is timed (CUDA events on
 * `stream`, median of 3 searches) and its recall@k against
 * tachiom_exhaustive_topk is measured; *best_kc / *best_kd receive the fastest
 * point with recall >= min_recall (none: the point of highest recall, the
 * faster on a tie), *best_recall and *best_ms its recall and time (may be
 * NULL). h_table (host [n_kc x n_kd x 4] floats, may be NULL) receives
 * (kappa_c, kappa_d, recall, ms) of every point, kappa_c-major. Blocking.   */
tachiom_status tachiom_autotune_budgets(tachiom_index *index, int32_t precision, const float *d_queries,
                                        const int32_t *h_ntok, int32_t nq, int32_t k, const int32_t *h_grid_kc,
                                        int32_t n_kc, const int32_t *h_grid_kd, int32_t n_kd, float min_recall,
                                        int32_t *best_kc, int32_t *best_kd, float *best_recall, float *best_ms,
                                        float *h_table, void *stream);

/* Synchronise `stream`, then return and clear the TACHIOM_FLAG_* bits raised
 * by work on that stream. Blocking.                                         */
tachiom_status tachiom_stream_status(tachiom_index *index, void *stream, uint32_t *h_flags);

/* ---- timing of the library's own launches ----
 * When enabled, every launcher records a CUDA event pair around its kernels on
 * the launching stream (not while the stream is being captured into a graph).
 * tachiom_profile_read synchronises `stream`, then returns, per launcher name in
 * first-launch order, the number of launches and their summed device time
 * since the previous read, and forgets them. `out` is a host array of `cap`
 * entries; *n_out receives the number written.                              */
typedef struct {
  char name[32];
  int32_t launches;
  double total_ms;
} tachiom_profile_entry;

tachiom_status tachiom_profile_enable(int on);
tachiom_status tachiom_profile_read(void *stream, tachiom_profile_entry *out, int32_t cap,
                                    int32_t *n_out);

/* Message of the last failed call on this thread ("" if none).             */
const char *tachiom_last_error(void);

/* 1 when the current device runs the tensor-core step (a) (compute capability
 * 10.3, the library's only target), else 0; TACHIOM_PREC_BF16 then uses the
 * FP32 CUDA-core path.                                                      */
int tachiom_tc_available(void);

/* Diagnostics of the tensor-core step (a): the BF16 x BF16 -> FP32 score of
 * each of nrows device fp32 rows (rounded to BF16 on the way) against every
 * centroid, written to d_out [nrows x C] fp32 (device, caller-owned). Used by
 * the tests to check the error bound the FP32 repair relies on.
 * TACHIOM_ERR_INVALID when the device has no tensor-core path.              */
tachiom_status tachiom_debug_tc_scores(tachiom_index *index, const float *d_rows, int32_t nrows,
                                       float *d_out, void *stream);

/* Diagnostics of step (c): the refined score S of every candidate slot,
 * d_cand_ids int32 [nq x kappa_d] (slots < 0 are left untouched), to d_scores
 * fp32 [nq x kappa_d], before any top-k. With TACHIOM_PREC_BF16 on a
 * tensor-core device these are the approximate scores of the decode-and-MMA
 * pass, and d_bounds (fp32 [nq x kappa_d], may be NULL) receives each
 * document's rigorous bound on |approximate - FP32 score| that the FP32
 * repair relies on; the tests check both against the oracle. Asynchronous. */
tachiom_status tachiom_debug_refine_scores(tachiom_index *index, const tachiom_search_params *params,
                                           const float *d_queries, const int32_t *h_ntok, int32_t nq,
                                           const int32_t *d_cand_ids, float *d_scores, float *d_bounds,
                                           void *stream);

/* Same with FP8-E4M3 products (each row and each centroid scaled by a power of
 * two; the scales undone): d_out [nrows x C] fp32. d_margins (fp32 [nrows], may
 * be NULL) receives twice the rigorous bound on |E4M3 score - FP32 score| of
 * each row. TACHIOM_ERR_INVALID when the device has no tensor-core path.     */
tachiom_status tachiom_debug_tc_scores_fp8(tachiom_index *index, const float *d_rows, int32_t nrows,
                                           float *d_out, float *d_margins, void *stream);

/* Diagnostics of the bounded waits of the tensor-core kernels: launches one CTA
 * of the step (a) tensor-core pass whose TMA producer issues no copy and whose
 * mbarrier waits give up after timeout_us (1..2e6) microseconds instead of the
 * usual 2 s. The MMA issuer's first wait runs out, so the kernel raises
 * TACHIOM_FLAG_TIMEOUT on `stream`, every role leaves its loop, TMEM is freed
 * and the kernel returns; read the flag with tachiom_stream_status. The
 * device stays usable. Asynchronous.                                         */
tachiom_status tachiom_debug_wait_timeout(tachiom_index *index, int32_t timeout_us, void *stream);

/* Diagnostics of the tensor-core step (a): runs it on nrows device rows on the
 * legacy default stream and copies, per row, the number of candidate centroids
 * emitted for exact FP32 rescoring to h_groups int32 [nrows] (host). Blocking. */
tachiom_status tachiom_debug_topc_groups(tachiom_index *index, const tachiom_search_params *params,
                                         const float *d_rows, int32_t nrows, int32_t *h_groups);

/* ---- Token-Aware Clustering: centroid allotment (Sec. 2.1, Phases 1-4) ----
 * Shares a centroid budget over token types before each type is clustered on
 * its own. Phase 1: a type with 0 < n_j < mu occurrences gets 1 centroid, one
 * with mu <= n_j < tau gets 2. Phase 2: every other type ("active", n_j >= tau)
 * gets floor(w_j / sum(w) * B), w_j = sqrt(n_j) * s_j, B = the budget left after
 * Phase 1, sum(w) over the active types. Phase 3: clamped to
 * [min(eps, cap_j), cap_j], cap_j = min(n_j, max(1, floor(n_j / theta))).
 * Phase 4: one centroid at a time to the active type below its cap with the
 * largest share_j - kappa_j (ties: lower id), or from the active type above its
 * floor with the smallest (ties: higher id), until the total is the budget.
 * The paper gives no values for mu, tau, eps, theta and no reconciliation
 * rule: these are the library's readings. Host-only, synchronous, no GPU. */
typedef struct {
  int64_t mu;    /* types with fewer occurrences get 1 centroid */
  int64_t tau;   /* types with fewer occurrences (and >= mu) get 2 */
  int32_t eps;   /* floor of an active type's allotment */
  double theta;  /* an active type keeps at least theta vectors per centroid (> 0) */
  int32_t gemm_min_kappa; /* tachiom_tac_cluster only: a type with at least this many centroids is
                             assigned through a BF16 GEMM on the tensor cores and an exact FP32
                             rescoring within a rigorous margin (the same labels); 0: 64; < 0: never */
} tachiom_tac_params;

/* n: host int64 [n_types] occurrences per type (<= 0: absent, 0 centroids);
 * s: host float64 [n_types] spread s_j = mean squared distance of the type's
 * vectors to their mean (read for active types; must be finite and >= 0);
 * kappa: host int32 [n_types] output, summing to `budget`. Returns
 * TACHIOM_ERR_INVALID (kappa unspecified) on a bad argument or when the bounds
 * cannot meet the budget. */
tachiom_status tachiom_tac_allot(const int64_t *n, const double *s, int32_t n_types, int64_t budget,
                                 const tachiom_tac_params *p, int32_t *kappa);

/* Token-Aware Clustering of a collection on the GPU (Sec. 2.1): groups the
 * vectors by token type, measures each type's spread s_j, shares `budget`
 * centroids out with tachiom_tac_allot (same parameters), then runs Lloyd's
 * kappa_j-means on every type on its own for `iters` rounds from its points at
 * positions floor((r + 1/2) n_j / kappa_j), r < kappa_j, and assigns every
 * vector once more. Squared L2 in FP32, ties to the lower centroid; means and
 * spreads in compensated FP32 (fixed summation order, so runs repeat bit for
 * bit); a centroid left without members keeps its place. Types with at least
 * p->gemm_min_kappa centroids are assigned through a cuBLAS BF16 GEMM on the
 * tensor cores with an exact FP32 rescoring of every centroid within a
 * rigorous margin of the approximate best (the same labels as the CUDA-core
 * kernel); the library links cuBLAS for this call only.
 *   d_vectors: device fp32 [n_vectors x 128], 16-byte aligned;
 *   d_types: device int32 [n_vectors], each in [0, n_types);
 *   h_kappa: host int32 [n_types] output; h_spread: host float64 [n_types]
 *   output or NULL; d_centroids: device fp32 [budget x 128] output, centroids
 *   numbered type by type; d_centroid_type: device int32 [budget] output;
 *   d_labels: device int32 [n_vectors] output, the centroid of each vector (-1
 *   when its type received none).
 * Allocates its own scratch (about 28 bytes per vector) and blocks until done
 * on `stream`. TACHIOM_ERR_INVALID on a bad argument, a type out of range or
 * a budget the allotment cannot meet; TACHIOM_ERR_OOM when scratch fails. */
tachiom_status tachiom_tac_cluster(const float *d_vectors, const int32_t *d_types, int64_t n_vectors,
                                   int32_t n_types, int64_t budget, const tachiom_tac_params *p,
                                   int32_t iters, int32_t *h_kappa, double *h_spread, float *d_centroids,
                                   int32_t *d_centroid_type, int32_t *d_labels, void *stream);

/* Residual compression (Sec. 2.1): for vector i with centroid row
 * d_centroids[d_labels[i]], r = x - c, rho = ||r||, r / rho split into pq_m
 * contiguous subspaces of 128 / pq_m dims, each coded by its nearest codeword
 * of d_codebooks (device fp32 [pq_m x 256 x 128 / pq_m]; squared L2 in FP32,
 * ties to the lower code). Outputs d_codes (device uint8 [n_vectors x pq_m])
 * and d_rnorm (device fp16 bits [n_vectors], rho rounded to nearest) - the
 * index's codes and residual norms. A zero residual or a label < 0 gives
 * rho = 0 and code 0. d_vectors (fp32 [n_vectors x 128]) and d_centroids must
 * be 16-byte aligned; labels must index rows of d_centroids. pq_m in {8, 16,
 * 32}. Asynchronous on `stream`; TACHIOM_ERR_INVALID on a bad argument. */
tachiom_status tachiom_pq_encode(const float *d_vectors, const float *d_centroids, const int32_t *d_labels,
                                 int64_t n_vectors, const float *d_codebooks, int32_t pq_m, uint8_t *d_codes,
                                 uint16_t *d_rnorm, void *stream);

/* Codebooks of the residual compression (Sec. 2.1), trained on the GPU: the
 * normalised residuals r / ||r|| (r = x - d_centroids[label]; the zero vector
 * for a zero residual or a label < 0) of `sample` vectors at positions
 * floor((s + 1/2) n_vectors / sample), split into pq_m subspaces, each
 * clustered into 256 codewords by `iters` Lloyd rounds from the sample points
 * at positions floor((j + 1/2) sample / 256) (squared L2 in FP32, ties to the
 * lower codeword, compensated FP32 means in a fixed order, an empty codeword
 * keeps its place). d_codebooks: device fp32 [pq_m x 256 x
 * 128 / pq_m] output, the layout tachiom_pq_encode and the index take.
 * 256 <= sample <= n_vectors. Allocates its scratch and blocks until done on
 * `stream`; TACHIOM_ERR_INVALID on a bad argument, TACHIOM_ERR_OOM. */
tachiom_status tachiom_pq_train(const float *d_vectors, const float *d_centroids, const int32_t *d_labels,
                                int64_t n_vectors, int32_t pq_m, int32_t sample, int32_t iters,
                                float *d_codebooks, void *stream);

/* Library version string. */
const char *tachiom_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TACHIOM_H */
