/*
 * FP64 CPU oracle for the gather-and-refine scoring path of TACHIOM
 * (arXiv 2604.28142, Sec. 2.2). TEST INFRASTRUCTURE ONLY: the tests, the
 * smoke check and the benchmark's CPU-baseline leg call it; the library never
 * does. It shares no code with the CUDA path.
 *
 * Plain and slow on purpose: every score is an FP64 dot product of the stored
 * values widened exactly (fp32 / bf16 centroids, fp32 queries and codebooks,
 * uint8 codes, fp16 residual norms); every selection is a full sort by
 * (score desc, id asc).
 *
 * Steps (the paper's order):
 *   1. top centroids   Sec. 2.2 Gather step 1. The paper finds them with a graph
 *                      search; here they are the exact kappa_c best by an
 *                      exhaustive scan, the set that search approximates.
 *   2./3. gather       Sec. 2.2 Gather steps 2-3: walk L_j for j in Top_i and keep
 *                      s~_i(d) = max_{j in Top_i : d in L_j} <q_i, c_j>.
 *   4. accumulate      Sec. 2.2 Gather step 4: S~(q,d) = sum_i s~_i(d), a query
 *                      token that reaches no list of d adds nothing.
 *   5. truncate        Sec. 2.2 (after the gather steps): the kappa_d docs with
 *                      the highest S~ (candidate pruning with alpha is off).
 *   6. refine          Sec. 2.2 Refine: S(q,d) = sum_i max_{t in d} v_it with
 *                      v_it = <q_i, c_a(t)> + rho_t <q_i, r^_t>, r^_t the PQ
 *                      decoded normalised residual (Sec. 2.1, Residuals
 *                      Compression: the norm is stored apart). Computed as a dot
 *                      with the decoded residual, not through lookup tables.
 *   7. top-k           rank the refined candidates by S.
 *
 * Inverted lists: L_j holds the ids of the documents with a token assigned to
 * c_j (Sec. 2.2, Index Structure), deduplicated and sorted ascending (max is
 * idempotent, so duplicates cannot change a result).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int dim;
  int64_t C, D, T;
  int M, ds;
  int cdtype; /* 0 = fp32, 1 = bf16 bit patterns */
  const void *cents;
  const int64_t *doc_off;
  const int32_t *tok_cid;
  const float *codebooks; /* [M][256][ds] */
  const uint8_t *codes;   /* [T][M] */
  const uint16_t *rnorm;  /* [T] fp16 bits, or NULL (rho = 1) */
  int64_t *list_off;      /* [C+1] */
  int32_t *list_doc;
} oracle_index;

/* ---- exact widening of the stored formats ---- */
static double bf16_to_double(uint16_t h) {
  uint32_t u = ((uint32_t)h) << 16;
  float f;
  memcpy(&f, &u, 4);
  return (double)f;
}

/* IEEE binary16 -> double, decoded field by field. */
static double half_to_double(uint16_t h) {
  int sign = (h >> 15) & 1, e = (h >> 10) & 31, m = h & 1023;
  double v;
  if (e == 0) v = ldexp((double)m, -24);               /* subnormal / zero */
  else if (e == 31) v = m ? NAN : INFINITY;
  else v = ldexp((double)(m + 1024), e - 25);          /* (1 + m/1024) 2^(e-15) */
  return sign ? -v : v;
}

static double cent_at(const oracle_index *ix, int64_t j, int k) {
  if (ix->cdtype == 1) return bf16_to_double(((const uint16_t *)ix->cents)[j * ix->dim + k]);
  return (double)((const float *)ix->cents)[j * ix->dim + k];
}

static double rho_at(const oracle_index *ix, int64_t t) {
  return ix->rnorm ? half_to_double(ix->rnorm[t]) : 1.0;
}

/* <q, c_j> in FP64 */
static double dot_qc(const oracle_index *ix, const float *q, int64_t j) {
  double s = 0.0;
  for (int k = 0; k < ix->dim; k++) s += (double)q[k] * cent_at(ix, j, k);
  return s;
}

/* decoded normalised residual component k of token t: codeword of subspace k/ds */
static double rhat_at(const oracle_index *ix, int64_t t, int k) {
  int m = k / ix->ds, r = k % ix->ds;
  int code = ix->codes[t * ix->M + m];
  return (double)ix->codebooks[((int64_t)m * 256 + code) * ix->ds + r];
}

/* ---- sorting helpers: (score desc, id asc) ---- */
typedef struct { double s; int64_t id; } scored;

static int cmp_scored(const void *a, const void *b) {
  const scored *x = (const scored *)a, *y = (const scored *)b;
  if (x->s > y->s) return -1;
  if (x->s < y->s) return 1;
  return (x->id > y->id) - (x->id < y->id);
}

/* ---- index ---- */
oracle_index *oracle_index_new(int dim, int64_t C, int64_t D, int64_t T, int M, int cdtype,
                               const void *cents, const int64_t *doc_off, const int32_t *tok_cid,
                               const float *codebooks, const uint8_t *codes, const uint16_t *rnorm) {
  if (dim <= 0 || M <= 0 || dim % M != 0 || C <= 0 || D < 0 || T < 0) return NULL;
  oracle_index *ix = (oracle_index *)calloc(1, sizeof(oracle_index));
  ix->dim = dim; ix->C = C; ix->D = D; ix->T = T; ix->M = M; ix->ds = dim / M;
  ix->cdtype = cdtype; ix->cents = cents; ix->doc_off = doc_off; ix->tok_cid = tok_cid;
  ix->codebooks = codebooks; ix->codes = codes; ix->rnorm = rnorm;
  /* inverted lists: count (doc, centroid) pairs once per doc, then fill in doc order */
  ix->list_off = (int64_t *)calloc((size_t)C + 1, sizeof(int64_t));
  int64_t *last = (int64_t *)malloc((size_t)C * sizeof(int64_t));
  for (int64_t j = 0; j < C; j++) last[j] = -1;
  for (int64_t d = 0; d < D; d++)
    for (int64_t t = doc_off[d]; t < doc_off[d + 1]; t++) {
      int32_t j = tok_cid[t];
      if (j < 0 || j >= C) { free(last); free(ix->list_off); free(ix); return NULL; }
      if (last[j] != d) { last[j] = d; ix->list_off[j + 1]++; }
    }
  for (int64_t j = 0; j < C; j++) ix->list_off[j + 1] += ix->list_off[j];
  ix->list_doc = (int32_t *)malloc((size_t)(ix->list_off[C] > 0 ? ix->list_off[C] : 1) * sizeof(int32_t));
  int64_t *fill = (int64_t *)malloc((size_t)C * sizeof(int64_t));
  for (int64_t j = 0; j < C; j++) { fill[j] = ix->list_off[j]; last[j] = -1; }
  for (int64_t d = 0; d < D; d++)
    for (int64_t t = doc_off[d]; t < doc_off[d + 1]; t++) {
      int32_t j = tok_cid[t];
      if (last[j] != d) { last[j] = d; ix->list_doc[fill[j]++] = (int32_t)d; }
    }
  free(fill);
  free(last);
  return ix;
}

void oracle_index_free(oracle_index *ix) {
  if (!ix) return;
  free(ix->list_off);
  free(ix->list_doc);
  free(ix);
}

int64_t oracle_list_total(const oracle_index *ix) { return ix->list_off[ix->C]; }
void oracle_lists(const oracle_index *ix, int64_t *off, int32_t *docs) {
  memcpy(off, ix->list_off, (size_t)(ix->C + 1) * sizeof(int64_t));
  memcpy(docs, ix->list_doc, (size_t)ix->list_off[ix->C] * sizeof(int32_t));
}

/* ---- step 1: exact top-kappa_c centroids of each query token (Sec. 2.2 Gather 1) ---- */
static void topc_row(const oracle_index *ix, const float *q, int kc, scored *work,
                     int32_t *out_id, double *out_s) {
  for (int64_t j = 0; j < ix->C; j++) { work[j].s = dot_qc(ix, q, j); work[j].id = j; }
  qsort(work, (size_t)ix->C, sizeof(scored), cmp_scored);
  for (int r = 0; r < kc; r++) {
    if (r < ix->C) { out_id[r] = (int32_t)work[r].id; out_s[r] = work[r].s; }
    else { out_id[r] = -1; out_s[r] = -INFINITY; }
  }
}

int oracle_top_centroids(const oracle_index *ix, const float *q, int64_t nrows, int kc,
                         int32_t *out_id, double *out_s) {
  if (kc <= 0) return 1;
#pragma omp parallel
  {
    scored *work = (scored *)malloc((size_t)ix->C * sizeof(scored));
#pragma omp for schedule(dynamic, 1)
    for (int64_t r = 0; r < nrows; r++)
      topc_row(ix, q + r * ix->dim, kc, work, out_id + r * kc, out_s + r * kc);
    free(work);
  }
  return 0;
}

/* ---- steps 2-4, list route (Sec. 2.2 Gather 2-4) ----
 * top_id [ntok][kc] (entries < 0 ignored). The scores <q_i, c_j> are recomputed
 * here in FP64 from the ids, so a replay of another implementation's choice
 * of Top_i is scored exactly. Output: every document reached by at least one
 * list, ascending doc id, with S~. Returns the number written (<= D).      */
typedef struct { double *best, *acc; char *hit, *seen_i; int32_t *touched, *touched_i; } gather_ws;

static void ws_alloc(gather_ws *w, int64_t D) {
  w->best = (double *)malloc((size_t)(D > 0 ? D : 1) * sizeof(double));
  w->acc = (double *)malloc((size_t)(D > 0 ? D : 1) * sizeof(double));
  w->hit = (char *)calloc((size_t)(D > 0 ? D : 1), 1);
  w->seen_i = (char *)calloc((size_t)(D > 0 ? D : 1), 1);
  w->touched = (int32_t *)malloc((size_t)(D > 0 ? D : 1) * sizeof(int32_t));
  w->touched_i = (int32_t *)malloc((size_t)(D > 0 ? D : 1) * sizeof(int32_t));
}
static void ws_free(gather_ws *w) {
  free(w->best); free(w->acc); free(w->hit); free(w->seen_i); free(w->touched); free(w->touched_i);
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

static int64_t gather_list_route(const oracle_index *ix, const float *q, int ntok, const int32_t *top_id,
                                 int kc, gather_ws *w, int32_t *out_doc, double *out_s) {
  int64_t ntouched = 0;
  for (int i = 0; i < ntok; i++) {
    const float *qi = q + (int64_t)i * ix->dim;
    int64_t nti = 0;
    for (int r = 0; r < kc; r++) {          /* step 2: each retrieved centroid's list */
      int32_t j = top_id[(int64_t)i * kc + r];
      if (j < 0) continue;
      double s = dot_qc(ix, qi, j);
      for (int64_t p = ix->list_off[j]; p < ix->list_off[j + 1]; p++) {
        int32_t d = ix->list_doc[p];
        if (!w->seen_i[d]) { w->seen_i[d] = 1; w->best[d] = s; w->touched_i[nti++] = d; }
        else if (s > w->best[d]) w->best[d] = s; /* step 3: keep the max */
      }
    }
    for (int64_t u = 0; u < nti; u++) {    /* step 4: accumulate over query tokens */
      int32_t d = w->touched_i[u];
      w->seen_i[d] = 0;
      if (!w->hit[d]) { w->hit[d] = 1; w->acc[d] = 0.0; w->touched[ntouched++] = d; }
      w->acc[d] += w->best[d];
    }
  }
  qsort(w->touched, (size_t)ntouched, sizeof(int32_t), cmp_i32);
  for (int64_t u = 0; u < ntouched; u++) {
    int32_t d = w->touched[u];
    out_doc[u] = d;
    out_s[u] = w->acc[d];
    w->hit[d] = 0;
  }
  return ntouched;
}

int64_t oracle_gather(const oracle_index *ix, const float *q, int ntok, const int32_t *top_id, int kc,
                      int32_t *out_doc, double *out_s) {
  gather_ws w;
  ws_alloc(&w, ix->D);
  int64_t n = gather_list_route(ix, q, ntok, top_id, kc, &w, out_doc, out_s);
  ws_free(&w);
  return n;
}

/* ---- the same S~ by the document route ----
 * s~_i(d) = max over the tokens t of d whose centroid a(t) is in Top_i of
 * <q_i, c_a(t)>: each document token is replaced by its centroid and the
 * per-query-token max runs over the document's tokens. Written independently
 * of the list route so that the two can check each other.                 */
int64_t oracle_gather_docroute(const oracle_index *ix, const float *q, int ntok, const int32_t *top_id,
                               int kc, int32_t *out_doc, double *out_s) {
  int64_t n = 0;
  for (int64_t d = 0; d < ix->D; d++) {
    double sum = 0.0;
    int any = 0;
    for (int i = 0; i < ntok; i++) {
      double m = -INFINITY;
      int found = 0;
      for (int64_t t = ix->doc_off[d]; t < ix->doc_off[d + 1]; t++) {
        int32_t j = ix->tok_cid[t];
        int in_top = 0;
        for (int r = 0; r < kc; r++)
          if (top_id[(int64_t)i * kc + r] == j) { in_top = 1; break; }
        if (!in_top) continue;
        double s = dot_qc(ix, q + (int64_t)i * ix->dim, j);
        if (!found || s > m) m = s;
        found = 1;
      }
      if (found) { sum += m; any = 1; }
    }
    if (any) { out_doc[n] = (int32_t)d; out_s[n] = sum; n++; }
  }
  return n;
}

/* ---- step 5 / step 7: first k by (score desc, doc asc) ---- */
int64_t oracle_select(const int32_t *doc, const double *s, int64_t n, int64_t k, int32_t *out_doc,
                      double *out_s) {
  scored *w = (scored *)malloc((size_t)(n > 0 ? n : 1) * sizeof(scored));
  for (int64_t u = 0; u < n; u++) { w[u].s = s[u]; w[u].id = doc[u]; }
  qsort(w, (size_t)n, sizeof(scored), cmp_scored);
  int64_t m = n < k ? n : k;
  for (int64_t u = 0; u < m; u++) { out_doc[u] = (int32_t)w[u].id; out_s[u] = w[u].s; }
  free(w);
  return m;
}

/* ---- step 6: refined MaxSim of one document (Sec. 2.2 Refine) ---- */
static double refine_doc(const oracle_index *ix, const float *q, int ntok, int32_t d) {
  double total = 0.0;
  for (int i = 0; i < ntok; i++) {
    const float *qi = q + (int64_t)i * ix->dim;
    double m = -INFINITY;
    for (int64_t t = ix->doc_off[d]; t < ix->doc_off[d + 1]; t++) {
      double cterm = dot_qc(ix, qi, ix->tok_cid[t]);   /* centroid contribution */
      double rterm = 0.0;                               /* residual contribution */
      for (int k = 0; k < ix->dim; k++) rterm += (double)qi[k] * rhat_at(ix, t, k);
      double v = cterm + rho_at(ix, t) * rterm;
      if (v > m) m = v;
    }
    if (ix->doc_off[d + 1] > ix->doc_off[d]) total += m;
  }
  return total;
}

int oracle_refine(const oracle_index *ix, const float *q, int ntok, const int32_t *docs, int64_t n,
                  double *out_s) {
  for (int64_t u = 0; u < n; u++)
    if (docs[u] < 0 || docs[u] >= ix->D) return 1;
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t u = 0; u < n; u++) out_s[u] = refine_doc(ix, q, ntok, docs[u]);
  return 0;
}

/* ---- the whole cascade for a batch of queries ----
 * queries packed [sum ntok][dim]; per-query ntok, k. Output row qi holds k_qi
 * entries at offset sum_{p<qi} k_p, padded with (-1, -inf) when fewer than k
 * documents survive. Optional stage outputs (may be NULL):
 *   top_id/top_s  [sum ntok][kc]
 *   cand_doc/cand_s [nq][kd]  (S~ of the kappa_d candidates, padded)        */
int oracle_search(const oracle_index *ix, const float *queries, const int32_t *ntok, const int32_t *kk,
                  int32_t nq, int kc, int kd, int32_t *out_doc, double *out_s, int32_t *top_id_out,
                  double *top_s_out, int32_t *cand_doc_out, double *cand_s_out) {
  if (kc <= 0 || kd <= 0 || nq < 0) return 1;
  int64_t *qoff = (int64_t *)malloc(((size_t)nq + 1) * sizeof(int64_t));
  int64_t *koff = (int64_t *)malloc(((size_t)nq + 1) * sizeof(int64_t));
  qoff[0] = 0; koff[0] = 0;
  for (int32_t u = 0; u < nq; u++) {
    if (ntok[u] <= 0 || kk[u] <= 0) { free(qoff); free(koff); return 1; }
    qoff[u + 1] = qoff[u] + ntok[u];
    koff[u + 1] = koff[u] + kk[u];
  }
  int err = 0;
#pragma omp parallel
  {
    scored *work = (scored *)malloc((size_t)ix->C * sizeof(scored));
    gather_ws w;
    ws_alloc(&w, ix->D);
    int32_t *gdoc = (int32_t *)malloc((size_t)(ix->D > 0 ? ix->D : 1) * sizeof(int32_t));
    double *gs = (double *)malloc((size_t)(ix->D > 0 ? ix->D : 1) * sizeof(double));
#pragma omp for schedule(dynamic, 1)
    for (int32_t u = 0; u < nq; u++) {
      const float *q = queries + qoff[u] * ix->dim;
      int nt = ntok[u];
      int32_t *top_id = (int32_t *)malloc((size_t)nt * kc * sizeof(int32_t));
      double *top_s = (double *)malloc((size_t)nt * kc * sizeof(double));
      for (int i = 0; i < nt; i++)
        topc_row(ix, q + (int64_t)i * ix->dim, kc, work, top_id + (int64_t)i * kc, top_s + (int64_t)i * kc);
      if (top_id_out) {
        memcpy(top_id_out + qoff[u] * kc, top_id, (size_t)nt * kc * sizeof(int32_t));
        memcpy(top_s_out + qoff[u] * kc, top_s, (size_t)nt * kc * sizeof(double));
      }
      int64_t ng = gather_list_route(ix, q, nt, top_id, kc, &w, gdoc, gs);
      int32_t *cdoc = (int32_t *)malloc((size_t)kd * sizeof(int32_t));
      double *cs = (double *)malloc((size_t)kd * sizeof(double));
      int64_t nc = oracle_select(gdoc, gs, ng, kd, cdoc, cs);
      if (cand_doc_out) {
        for (int64_t r = 0; r < kd; r++) {
          cand_doc_out[(int64_t)u * kd + r] = r < nc ? cdoc[r] : -1;
          cand_s_out[(int64_t)u * kd + r] = r < nc ? cs[r] : -INFINITY;
        }
      }
      double *rs = (double *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(double));
      if (oracle_refine(ix, q, nt, cdoc, nc, rs)) err = 1;
      int32_t *fdoc = (int32_t *)malloc((size_t)kk[u] * sizeof(int32_t));
      double *fs = (double *)malloc((size_t)kk[u] * sizeof(double));
      int64_t nf = oracle_select(cdoc, rs, nc, kk[u], fdoc, fs);
      for (int64_t r = 0; r < kk[u]; r++) {
        out_doc[koff[u] + r] = r < nf ? fdoc[r] : -1;
        out_s[koff[u] + r] = r < nf ? fs[r] : -INFINITY;
      }
      free(fdoc); free(fs); free(rs); free(cdoc); free(cs); free(top_id); free(top_s);
    }
    free(gdoc); free(gs);
    ws_free(&w);
    free(work);
  }
  free(qoff);
  free(koff);
  return err;
}
