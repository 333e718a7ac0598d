/*
 * CPU ORACLE for filtered top-K retrieval -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may load
 * this file's library.  The product path never calls it.  It shares no code with
 * the CUDA path.
 *
 * What it computes, plainly and slowly, in FP64:
 *
 *   1. Term predicate (F-TBR; Sec. 5.3 "System Implementation" and the
 *      appendix paragraph "TBR").  A filter is in conjunctive normal form: an AND
 *      of clauses, each clause an OR over term ids.  Job j passes filter q iff
 *      every clause of q shares at least one term with T_j, the job's sorted set
 *      of terms.  Each clause test is the sorted two-pointer intersection the
 *      appendix describes.  A filter with zero clauses passes every job.
 *
 *   2. Score (F-EBR; Sec. 5.3 and appendix paragraph "EBR"): the inner product
 *      s = sum_k q_k x_jk accumulated in FP64 from the FP32 inputs, or the cosine
 *      s = dot / (|q| |x_j|) with FP64 norms (a zero norm gives s = 0).
 *
 *   3. Top-K (appendix "Fast Top K Selection" defines the goal; the oracle does
 *      not use the bucket trick): all passing jobs are sorted FULLY by the key
 *      (score descending, job id ascending) and the first min(K, #passing) kept.
 *
 *   4. Messenger (appendix "Message Passing between Layers" and "Batch
 *      Inference"): the list of (rowId, batchId) pairs that pass the filter,
 *      ordered by rowId, then batchId.
 *
 * No blocking, fusion or reordering beyond these definitions.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int cmp_u32(const void *a, const void *b) {
  uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
  return (x > y) - (x < y);
}

/* sort ascending and drop duplicates in place; returns the new length */
static int64_t sort_unique(uint32_t *v, int64_t n) {
  if (n <= 1) return n;
  qsort(v, (size_t)n, sizeof(uint32_t), cmp_u32);
  int64_t w = 1;
  for (int64_t i = 1; i < n; ++i)
    if (v[i] != v[w - 1]) v[w++] = v[i];
  return w;
}

/* Two sorted vectors intersect?  Classic two-pointer walk. */
static int sorted_intersect(const uint32_t *a, int64_t na, const uint32_t *b, int64_t nb) {
  int64_t i = 0, k = 0;
  while (i < na && k < nb) {
    if (a[i] == b[k]) return 1;
    if (a[i] < b[k]) ++i; else ++k;
  }
  return 0;
}

/* A corpus of job term sets, each sorted and de-duplicated (T_j). */
typedef struct {
  int64_t n;
  int64_t *off;   /* [n+1] */
  uint32_t *t;    /* sorted unique terms */
} termsets_t;

static int termsets_build(termsets_t *S, int64_t n, const int64_t *job_off, const int32_t *job_terms) {
  S->n = n;
  S->off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  S->t = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(job_off[n] > 0 ? job_off[n] : 1));
  if (!S->off || !S->t) return 1;
  S->off[0] = 0;
  for (int64_t j = 0; j < n; ++j) {
    int64_t len = job_off[j + 1] - job_off[j];
    uint32_t *dst = S->t + S->off[j];
    for (int64_t p = 0; p < len; ++p) dst[p] = (uint32_t)job_terms[job_off[j] + p];
    S->off[j + 1] = S->off[j] + sort_unique(dst, len);
  }
  return 0;
}

static void termsets_free(termsets_t *S) { free(S->off); free(S->t); }

/* One query's CNF with each clause sorted and de-duplicated. */
typedef struct {
  int32_t nc;
  int64_t *coff;  /* [nc+1] */
  uint32_t *t;
} cnf_t;

static int cnf_build(cnf_t *C, int32_t b, const int32_t *q_off, const int32_t *c_off, const uint32_t *terms) {
  int32_t c0 = q_off[b], c1 = q_off[b + 1];
  C->nc = c1 - c0;
  C->coff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(C->nc + 1));
  int64_t tot = (C->nc > 0) ? (int64_t)(c_off[c1] - c_off[c0]) : 0;
  C->t = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(tot > 0 ? tot : 1));
  if (!C->coff || !C->t) return 1;
  C->coff[0] = 0;
  for (int32_t c = 0; c < C->nc; ++c) {
    int64_t len = c_off[c0 + c + 1] - c_off[c0 + c];
    uint32_t *dst = C->t + C->coff[c];
    for (int64_t p = 0; p < len; ++p) dst[p] = terms[c_off[c0 + c] + p];
    C->coff[c + 1] = C->coff[c] + sort_unique(dst, len);
  }
  return 0;
}

static void cnf_free(cnf_t *C) { free(C->coff); free(C->t); }

/* pass(q, j) = AND over clauses of (clause ∩ T_j ≠ ∅); zero clauses -> 1 */
static int cnf_pass(const cnf_t *C, const termsets_t *S, int64_t j) {
  const uint32_t *tj = S->t + S->off[j];
  int64_t nj = S->off[j + 1] - S->off[j];
  for (int32_t c = 0; c < C->nc; ++c)
    if (!sorted_intersect(C->t + C->coff[c], C->coff[c + 1] - C->coff[c], tj, nj)) return 0;
  return 1;
}

static double dot64(const float *a, const float *b, int32_t d) {
  double s = 0.0;
  for (int32_t k = 0; k < d; ++k) s += (double)a[k] * (double)b[k];
  return s;
}

typedef struct { double s; int64_t id; } scored_t;

/* strict order: higher score first; equal scores -> lower id first */
static int cmp_scored(const void *a, const void *b) {
  const scored_t *x = (const scored_t *)a, *y = (const scored_t *)b;
  if (x->s > y->s) return -1;
  if (x->s < y->s) return 1;
  return (x->id > y->id) - (x->id < y->id);
}

/* ------------------------------------------------------------------ API -- */

/* pass counts (and optionally the pass matrix as bytes [B][n]) */
int oracle_filter(int64_t n, const int64_t *job_off, const int32_t *job_terms, int32_t B,
                  const int32_t *q_off, const int32_t *c_off, const uint32_t *terms,
                  int64_t *out_pass_count, uint8_t *out_pass /* nullable [B][n] */) {
  termsets_t S;
  if (termsets_build(&S, n, job_off, job_terms)) return 1;
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t b = 0; b < B; ++b) {
    cnf_t C;
    if (cnf_build(&C, b, q_off, c_off, terms)) { err = 1; continue; }
    int64_t cnt = 0;
    for (int64_t j = 0; j < n; ++j) {
      int p = cnf_pass(&C, &S, j);
      cnt += p;
      if (out_pass) out_pass[(size_t)b * (size_t)n + (size_t)j] = (uint8_t)p;
    }
    out_pass_count[b] = cnt;
    cnf_free(&C);
  }
  termsets_free(&S);
  return err;
}

/* Messenger list of the batch: all passing (rowId, batchId) ordered by rowId
 * then batchId.  With rows == NULL only the count is returned. */
int64_t oracle_messenger(int64_t n, const int64_t *job_off, const int32_t *job_terms, int32_t B,
                         const int32_t *q_off, const int32_t *c_off, const uint32_t *terms,
                         int64_t *rows, int32_t *batch) {
  termsets_t S;
  if (termsets_build(&S, n, job_off, job_terms)) return -1;
  cnf_t *C = (cnf_t *)malloc(sizeof(cnf_t) * (size_t)(B > 0 ? B : 1));
  for (int32_t b = 0; b < B; ++b) cnf_build(&C[b], b, q_off, c_off, terms);
  int64_t m = 0;
  for (int64_t j = 0; j < n; ++j)
    for (int32_t b = 0; b < B; ++b)
      if (cnf_pass(&C[b], &S, j)) {
        if (rows) { rows[m] = j; batch[m] = b; }
        ++m;
      }
  for (int32_t b = 0; b < B; ++b) cnf_free(&C[b]);
  free(C);
  termsets_free(&S);
  return m;
}

/* Filtered top-K.  metric: 0 = dot, 1 = cosine.  k: per-query K (k[b] >= 0).
 * Outputs (row b, stride kmax): ids (-1 padded), FP64 scores (-inf padded),
 * count[b] = min(k[b], passing), pass_count[b] = passing. */
int oracle_search(int64_t n, int32_t d, const float *X, const int64_t *job_off, const int32_t *job_terms,
                  int32_t B, const float *Q, const int32_t *q_off, const int32_t *c_off,
                  const uint32_t *terms, const int32_t *k, int32_t kmax, int32_t metric,
                  int64_t *out_ids, double *out_scores, int64_t *out_count, int64_t *out_pass_count) {
  termsets_t S;
  if (termsets_build(&S, n, job_off, job_terms)) return 1;
  double *xnorm = NULL;
  if (metric == 1) {
    xnorm = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t j = 0; j < n; ++j) {
      const float *x = X + (size_t)j * (size_t)d;
      xnorm[j] = sqrt(dot64(x, x, d));
    }
  }
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t b = 0; b < B; ++b) {
    cnf_t C;
    scored_t *all = (scored_t *)malloc(sizeof(scored_t) * (size_t)(n > 0 ? n : 1));
    if (!all || cnf_build(&C, b, q_off, c_off, terms)) { err = 1; free(all); continue; }
    const float *q = Q + (size_t)b * (size_t)d;
    double qn = (metric == 1) ? sqrt(dot64(q, q, d)) : 1.0;
    int64_t m = 0;
    for (int64_t j = 0; j < n; ++j) {
      if (!cnf_pass(&C, &S, j)) continue;
      double s = dot64(q, X + (size_t)j * (size_t)d, d);
      if (metric == 1) s = (qn > 0.0 && xnorm[j] > 0.0) ? s / (qn * xnorm[j]) : 0.0;
      all[m].s = s;
      all[m].id = j;
      ++m;
    }
    qsort(all, (size_t)m, sizeof(scored_t), cmp_scored);
    int64_t kk = k[b] < m ? k[b] : m;
    for (int64_t i = 0; i < kmax; ++i) {
      out_ids[(size_t)b * (size_t)kmax + (size_t)i] = (i < kk) ? all[i].id : -1;
      out_scores[(size_t)b * (size_t)kmax + (size_t)i] = (i < kk) ? all[i].s : -INFINITY;
    }
    out_count[b] = kk;
    out_pass_count[b] = m;
    cnf_free(&C);
    free(all);
  }
  free(xnorm);
  termsets_free(&S);
  return err;
}

/* FP64 scores of given (query, job) pairs: s = dot or cosine as above. */
int oracle_pair_scores(int32_t d, const float *X, const float *Q, int64_t npairs, const int64_t *qi,
                       const int64_t *ji, int32_t metric, double *out) {
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < npairs; ++p) {
    const float *q = Q + (size_t)qi[p] * (size_t)d, *x = X + (size_t)ji[p] * (size_t)d;
    double s = dot64(q, x, d);
    if (metric == 1) {
      double qn = sqrt(dot64(q, q, d)), xn = sqrt(dot64(x, x, d));
      s = (qn > 0.0 && xn > 0.0) ? s / (qn * xn) : 0.0;
    }
    out[p] = s;
  }
  return 0;
}

/* pass(q, j) of given (query, job) pairs, same definition as above. */
int oracle_pair_pass(int64_t n, const int64_t *job_off, const int32_t *job_terms, int32_t B, const int32_t *q_off,
                     const int32_t *c_off, const uint32_t *terms, int64_t npairs, const int64_t *qi,
                     const int64_t *ji, uint8_t *out) {
  cnf_t *C = (cnf_t *)malloc(sizeof(cnf_t) * (size_t)(B > 0 ? B : 1));
  if (!C) return 1;
  for (int32_t b = 0; b < B; ++b) cnf_build(&C[b], b, q_off, c_off, terms);
  int err = 0;
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < npairs; ++p) {
    const int64_t j = ji[p];
    if (j < 0 || j >= n || qi[p] < 0 || qi[p] >= B) { err = 1; out[p] = 0; continue; }
    /* T_j for this one job, sorted and de-duplicated */
    int64_t len = job_off[j + 1] - job_off[j];
    uint32_t *tj = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(len > 0 ? len : 1));
    for (int64_t i = 0; i < len; ++i) tj[i] = (uint32_t)job_terms[job_off[j] + i];
    len = sort_unique(tj, len);
    const cnf_t *c = &C[qi[p]];
    int pass = 1;
    for (int32_t k = 0; k < c->nc && pass; ++k)
      pass = sorted_intersect(c->t + c->coff[k], c->coff[k + 1] - c->coff[k], tj, len);
    out[p] = (uint8_t)pass;
    free(tj);
  }
  for (int32_t b = 0; b < B; ++b) cnf_free(&C[b]);
  free(C);
  return err;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------ sign-bit pre-selection -- */
/*
 * Sign codes (appendix "Quantization", Sec. 5.3: a quantisation akin to
 * OP+ORP).  The caller gives the random projection: sample b of a row is
 *     s_b = sum_{m < bin} sgn[b * bin + m] * x[idx[b * bin + m]],
 * added in FP32 in the order m = 0, 1, ..., and bit b of the code is 1 iff
 * s_b > 0 (bit b % 64 of word b / 64).  The projection is the appendix's:
 * coordinates permuted, cut into bins, each entry multiplied by a random sign
 * and the bin summed (several permutations when the row has fewer coordinates
 * than bits).
 */
int oracle_sign_codes(int64_t n, int32_t d, const float *X, int32_t nbits, int32_t bin, const int32_t *idx,
                      const int8_t *sgn, uint64_t *codes) {
  const int32_t W = nbits / 64;
  for (int64_t i = 0; i < (int64_t)nbits * bin; ++i)
    if (idx[i] < 0 || idx[i] >= d) return 1;
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) {
    const float *x = X + (size_t)j * (size_t)d;
    uint64_t *c = codes + (size_t)j * (size_t)W;
    for (int32_t w = 0; w < W; ++w) c[w] = 0;
    for (int32_t b = 0; b < nbits; ++b) {
      float s = 0.0f;
      for (int32_t m = 0; m < bin; ++m) {
        const float v = x[idx[(size_t)b * bin + m]];
        const float t = sgn[(size_t)b * bin + m] > 0 ? v : -v;
        s = s + t;
      }
      if (s > 0.0f) c[b / 64] |= (uint64_t)1 << (b % 64);
    }
  }
  return 0;
}

/* Eq. 4: the number of positions at which two codes hold the same bit. */
static int32_t sign_agree(const uint64_t *a, const uint64_t *b, int32_t W) {
  int32_t s = 0;
  for (int32_t w = 0; w < W; ++w) s += __builtin_popcountll(~(a[w] ^ b[w]));
  return s;
}

/*
 * Filtered search with sign-bit pre-selection: for each query the passing jobs
 * are scored by Eq. 4 against the query's code; the pre-selection keeps whole
 * score levels from the top, down to the highest level t at which at least
 * Q = min(quant_k[b], #passing) jobs are kept (one level higher when that set
 * would exceed `cap` jobs); the kept jobs are scored exactly (FP64 dot or
 * cosine, as oracle_search) and the top k[b] by (score desc, id asc) returned.
 * out_ncand[b] = the number of jobs kept by the pre-selection.
 */
int oracle_sign_search(int64_t n, int32_t d, const float *X, const int64_t *job_off, const int32_t *job_terms,
                       int32_t B, const float *Q, const int32_t *q_off, const int32_t *c_off, const uint32_t *terms,
                       const int32_t *k, int32_t kmax, int32_t metric, const uint64_t *codes,
                       const uint64_t *qcodes, int32_t nbits, const int64_t *quant_k, int64_t cap,
                       int64_t *out_ids, double *out_scores, int64_t *out_count, int64_t *out_ncand) {
  termsets_t S;
  if (termsets_build(&S, n, job_off, job_terms)) return 1;
  const int32_t W = nbits / 64;
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t b = 0; b < B; ++b) {
    cnf_t C;
    int32_t *level = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t *hist = (int64_t *)calloc((size_t)nbits + 2, sizeof(int64_t));
    scored_t *all = (scored_t *)malloc(sizeof(scored_t) * (size_t)(n > 0 ? n : 1));
    if (!level || !hist || !all || cnf_build(&C, b, q_off, c_off, terms)) {
      err = 1;
      free(level); free(hist); free(all);
      continue;
    }
    int64_t P = 0;
    for (int64_t j = 0; j < n; ++j) {
      level[j] = -1;
      if (!cnf_pass(&C, &S, j)) continue;
      level[j] = sign_agree(codes + (size_t)j * W, qcodes + (size_t)b * W, W);
      hist[level[j]] += 1;
      ++P;
    }
    const int64_t want = quant_k[b] < P ? quant_k[b] : P;
    int32_t t = nbits + 1;  /* keep nothing when want == 0 */
    int64_t kept = 0;
    if (want > 0) {
      int64_t cum = 0;
      for (t = nbits; t >= 0; --t) {
        cum += hist[t];
        if (cum >= want) break;
      }
      kept = cum;
      if (kept > cap) { kept -= hist[t]; t += 1; }
    }
    const float *q = Q + (size_t)b * (size_t)d;
    const double qn = (metric == 1) ? sqrt(dot64(q, q, d)) : 1.0;
    int64_t m = 0;
    for (int64_t j = 0; j < n; ++j) {
      if (level[j] < t) continue;
      const float *x = X + (size_t)j * (size_t)d;
      double s = dot64(q, x, d);
      if (metric == 1) {
        const double xn = sqrt(dot64(x, x, d));
        s = (qn > 0.0 && xn > 0.0) ? s / (qn * xn) : 0.0;
      }
      all[m].s = s;
      all[m].id = j;
      ++m;
    }
    qsort(all, (size_t)m, sizeof(scored_t), cmp_scored);
    const int64_t kk = k[b] < m ? k[b] : m;
    for (int64_t i = 0; i < kmax; ++i) {
      out_ids[(size_t)b * (size_t)kmax + (size_t)i] = (i < kk) ? all[i].id : -1;
      out_scores[(size_t)b * (size_t)kmax + (size_t)i] = (i < kk) ? all[i].s : -INFINITY;
    }
    out_count[b] = kk;
    out_ncand[b] = m;
    cnf_free(&C);
    free(level); free(hist); free(all);
  }
  termsets_free(&S);
  return err;
}
