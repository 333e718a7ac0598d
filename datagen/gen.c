/*
 * Seeded synthetic workload generator for filtered top-K retrieval.
 *
 * This file produces INPUTS only (embeddings, per-job term sets, CNF filters and
 * the input-format conversions between term layouts).  It holds none of the
 * retrieval arithmetic: no predicate evaluation, no scoring, no selection.
 * Both the CPU oracle tests and the CUDA path consume what it writes.
 *
 * Random numbers: every logical stream (one job's embedding, one job's term
 * set, one query, one filter) owns an independent xoshiro256** generator
 * (Blackman & Vigna, 2018) whose 256-bit state is filled by SplitMix64
 * (Steele, Lea & Flood, 2014) from (seed, stream id).  Output therefore does
 * not depend on the OpenMP thread count or schedule.
 *
 * Distributions:
 *   - Gaussian: Box-Muller transform on two 53-bit uniforms.
 *   - Truncated Zipf(s) on ranks 1..V (rank r -> term id r-1), p_r ∝ r^-s,
 *     sampled with Walker's alias method (Vose's construction).
 *   - Poisson(lambda): inversion by sequential search of the CDF.
 *   - "n distinct terms": sequential rejection of repeats from the Zipf stream.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- RNG -- */
static inline uint64_t sm64_next(uint64_t *x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } xo_t;

static inline uint64_t rotl64(uint64_t v, int k) { return (v << k) | (v >> (64 - k)); }

static void xo_seed(xo_t *g, uint64_t seed, uint64_t stream) {
  uint64_t x = seed * 0xD1B54A32D192ED03ULL ^ stream;
  /* two SplitMix rounds of the combined key so nearby streams decorrelate */
  x = sm64_next(&x) ^ stream;
  for (int i = 0; i < 4; ++i) g->s[i] = sm64_next(&x);
}

static inline uint64_t xo_next(xo_t *g) {
  uint64_t *s = g->s;
  uint64_t r = rotl64(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl64(s[3], 45);
  return r;
}

/* uniform in [0, 1) with 53 random bits */
static inline double xo_unif(xo_t *g) { return (double)(xo_next(g) >> 11) * 0x1.0p-53; }

/* standard normal by Box-Muller; draws a fresh pair each call and keeps the spare */
typedef struct { xo_t g; int has; double spare; } gauss_t;

static inline double gauss_next(gauss_t *G) {
  if (G->has) { G->has = 0; return G->spare; }
  double u1, u2;
  do { u1 = xo_unif(&G->g); } while (u1 <= 0.0);
  u2 = xo_unif(&G->g);
  double r = sqrt(-2.0 * log(u1));
  double th = 6.283185307179586476925286766559 * u2;
  G->spare = r * sin(th);
  G->has = 1;
  return r * cos(th);
}

/* stream-id namespaces: high bits name the purpose, low bits the item */
#define STREAM_JOB_EMB   (1ULL << 56)
#define STREAM_JOB_TERMS (2ULL << 56)
#define STREAM_QUERY_EMB (3ULL << 56)
#define STREAM_FILTER    (4ULL << 56)

/* ----------------------------------------------------------- embeddings -- */
/* out[i][k], i in [0,n): Gaussian, normalised in FP64, rounded to FP32 (RNE).
 * stream_kind: 0 = job embeddings, 1 = query embeddings.  first_item offsets
 * the item index so a caller can generate a range of a larger set. */
int gen_embeddings(uint64_t seed, int stream_kind, int64_t first_item, int64_t n, int32_t d,
                   int normalise, float *out) {
  if (n < 0 || d <= 0 || !out) return 1;
  const uint64_t base = stream_kind ? STREAM_QUERY_EMB : STREAM_JOB_EMB;
#pragma omp parallel
  {
    double *tmp = (double *)malloc(sizeof(double) * (size_t)d);
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      gauss_t G;
      xo_seed(&G.g, seed, base | (uint64_t)(first_item + i));
      G.has = 0;
      double ss = 0.0;
      for (int32_t k = 0; k < d; ++k) { tmp[k] = gauss_next(&G); ss += tmp[k] * tmp[k]; }
      double inv = (normalise && ss > 0.0) ? 1.0 / sqrt(ss) : 1.0;
      float *row = out + (size_t)i * (size_t)d;
      for (int32_t k = 0; k < d; ++k) row[k] = (float)(tmp[k] * inv);
    }
    free(tmp);
  }
  return 0;
}

/* --------------------------------------------------------- Zipf (alias) -- */
typedef struct { int32_t V; double *prob; int32_t *alias; } alias_t;

static int alias_build(alias_t *A, int32_t V, double s) {
  A->V = V;
  A->prob = (double *)malloc(sizeof(double) * (size_t)V);
  A->alias = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
  double *p = (double *)malloc(sizeof(double) * (size_t)V);
  int32_t *small = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
  int32_t *large = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
  if (!A->prob || !A->alias || !p || !small || !large) return 1;
  double tot = 0.0;
  for (int32_t r = 0; r < V; ++r) { p[r] = pow((double)(r + 1), -s); tot += p[r]; }
  int32_t ns = 0, nl = 0;
  for (int32_t r = 0; r < V; ++r) {
    p[r] = p[r] / tot * (double)V;
    if (p[r] < 1.0) small[ns++] = r; else large[nl++] = r;
  }
  while (ns > 0 && nl > 0) {
    int32_t l = small[--ns], g = large[--nl];
    A->prob[l] = p[l];
    A->alias[l] = g;
    p[g] = (p[g] + p[l]) - 1.0;
    if (p[g] < 1.0) small[ns++] = g; else large[nl++] = g;
  }
  while (nl > 0) { int32_t g = large[--nl]; A->prob[g] = 1.0; A->alias[g] = g; }
  while (ns > 0) { int32_t l = small[--ns]; A->prob[l] = 1.0; A->alias[l] = l; }
  free(p); free(small); free(large);
  return 0;
}

static void alias_free(alias_t *A) { free(A->prob); free(A->alias); }

static inline int32_t alias_draw(const alias_t *A, xo_t *g) {
  double u = xo_unif(g) * (double)A->V;
  int32_t i = (int32_t)u;
  if (i >= A->V) i = A->V - 1;
  double f = u - (double)i;
  return (f < A->prob[i]) ? i : A->alias[i];
}

static inline int32_t poisson_draw(double lam, xo_t *g) {
  double u = xo_unif(g);
  double p = exp(-lam), F = p;
  int32_t k = 0;
  while (u > F && k < 100000) { ++k; p *= lam / (double)k; F += p; if (p == 0.0 && F < u) break; }
  return k;
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* draw n distinct Zipf terms (sequential rejection of repeats); seen is a V-bit
 * scratch bitmap that is returned all-zero */
static void distinct_terms(const alias_t *A, xo_t *g, int32_t n, int32_t *dst, uint64_t *seen) {
  int32_t V = A->V;
  if (n >= V) { for (int32_t t = 0; t < V; ++t) dst[t] = t; return; }
  int32_t got = 0;
  while (got < n) {
    int32_t t = alias_draw(A, g);
    uint64_t bit = 1ULL << (t & 63);
    if (seen[t >> 6] & bit) continue;
    seen[t >> 6] |= bit;
    dst[got++] = t;
  }
  for (int32_t i = 0; i < n; ++i) seen[dst[i] >> 6] &= ~(1ULL << (dst[i] & 63));
  qsort(dst, (size_t)n, sizeof(int32_t), cmp_i32);
}

/* ------------------------------------------------------------ job terms -- */
/* Pass 1: counts[i] = min(Poisson(lam), V) for jobs [first, first+n). */
int gen_job_term_counts(uint64_t seed, int64_t first, int64_t n, int32_t V, double lam,
                        int32_t *counts) {
  if (n < 0 || V <= 0 || !counts) return 1;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    xo_t g;
    xo_seed(&g, seed, STREAM_JOB_TERMS | (uint64_t)(first + i));
    int32_t c = poisson_draw(lam, &g);
    counts[i] = c > V ? V : c;
  }
  return 0;
}

/* Pass 2: job_terms[job_off[i] .. job_off[i+1]) = sorted distinct term ids of
 * job first+i.  job_off is the exclusive prefix sum of the pass-1 counts. */
int gen_job_terms(uint64_t seed, int64_t first, int64_t n, int32_t V, double lam, double zipf_s,
                  const int64_t *job_off, int32_t *job_terms) {
  if (n < 0 || V <= 0 || !job_off || !job_terms) return 1;
  alias_t A;
  if (alias_build(&A, V, zipf_s)) return 2;
  int err = 0;
#pragma omp parallel
  {
    uint64_t *seen = (uint64_t *)calloc((size_t)(V + 63) / 64, sizeof(uint64_t));
    if (!seen) err = 3;
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      if (!seen) continue;
      xo_t g;
      xo_seed(&g, seed, STREAM_JOB_TERMS | (uint64_t)(first + i));
      int32_t c = poisson_draw(lam, &g);
      if (c > V) c = V;
      if ((int64_t)c != job_off[i + 1] - job_off[i]) { err = 4; continue; }
      distinct_terms(&A, &g, c, job_terms + job_off[i], seen);
    }
    free(seen);
  }
  alias_free(&A);
  return err;
}

/* -------------------------------------------------------------- filters -- */
/* A filter is a CNF: clauses AND-ed, each an OR over distinct terms.
 * Clause count ~ U{cmin..cmax}, terms per clause ~ U{tmin..tmax} (capped at V),
 * terms drawn from the same truncated Zipf, distinct within a clause and
 * sorted.  Pass 1 returns the clause count and the total term count of
 * filters [first, first+n) so the caller can size the CSR arrays. */
static inline int32_t unif_int(xo_t *g, int32_t lo, int32_t hi) {
  if (hi <= lo) return lo;
  int32_t v = lo + (int32_t)(xo_unif(g) * (double)(hi - lo + 1));
  return v > hi ? hi : v;
}

int gen_filter_sizes(uint64_t seed, int64_t first, int64_t n, int32_t V, int32_t cmin, int32_t cmax,
                     int32_t tmin, int32_t tmax, int32_t *n_clauses, int32_t *n_terms) {
  if (n < 0 || !n_clauses || !n_terms) return 1;
  for (int64_t i = 0; i < n; ++i) {
    xo_t g;
    xo_seed(&g, seed, STREAM_FILTER | (uint64_t)(first + i));
    int32_t nc = unif_int(&g, cmin, cmax), tt = 0;
    if (nc > 64) nc = 64;
    for (int32_t c = 0; c < nc; ++c) {
      int32_t nt = unif_int(&g, tmin, tmax);
      if (nt > V) nt = V;
      tt += nt;
      /* skip the term draws: the sizes are fixed before any term is drawn */
    }
    n_clauses[i] = nc;
    n_terms[i] = tt;
  }
  return 0;
}

/* Pass 2: q_off[n+1] (clause ranges per filter), c_off[total_clauses+1]
 * (term ranges per clause), terms[total_terms].  q_off/c_off are written here. */
int gen_filters(uint64_t seed, int64_t first, int64_t n, int32_t V, double zipf_s, int32_t cmin,
                int32_t cmax, int32_t tmin, int32_t tmax, int32_t *q_off, int32_t *c_off,
                uint32_t *terms) {
  if (n < 0 || !q_off || !c_off || !terms) return 1;
  alias_t A;
  if (alias_build(&A, V, zipf_s)) return 2;
  uint64_t *seen = (uint64_t *)calloc((size_t)(V + 63) / 64, sizeof(uint64_t));
  int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(tmax > 0 ? (tmax < V ? tmax : V) : 1));
  if (!seen || !tmp) { alias_free(&A); free(seen); free(tmp); return 3; }
  int32_t nq_c = 0, nq_t = 0;
  q_off[0] = 0;
  c_off[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    xo_t g;
    xo_seed(&g, seed, STREAM_FILTER | (uint64_t)(first + i));
    int32_t nc = unif_int(&g, cmin, cmax);
    int32_t sizes[64];
    if (nc > 64) nc = 64;
    for (int32_t c = 0; c < nc; ++c) {
      int32_t nt = unif_int(&g, tmin, tmax);
      sizes[c] = nt > V ? V : nt;
    }
    for (int32_t c = 0; c < nc; ++c) {
      distinct_terms(&A, &g, sizes[c], tmp, seen);
      for (int32_t t = 0; t < sizes[c]; ++t) terms[nq_t + t] = (uint32_t)tmp[t];
      nq_t += sizes[c];
      c_off[++nq_c] = nq_t;
    }
    q_off[i + 1] = nq_c;
  }
  alias_free(&A);
  free(seen);
  free(tmp);
  return 0;
}

/* ------------------------------------------------- layout conversions -- */
/* Term-major CSR (posting lists) from job-major term lists: post_off[V+1],
 * post_ids[nnz] with ids ascending within each term. */
int invert_to_postings(int64_t n, int32_t V, const int64_t *job_off, const int32_t *job_terms,
                       int64_t *post_off, uint32_t *post_ids) {
  if (n < 0 || V <= 0) return 1;
  memset(post_off, 0, sizeof(int64_t) * (size_t)(V + 1));
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = job_off[i]; p < job_off[i + 1]; ++p) {
      int32_t t = job_terms[p];
      if (t < 0 || t >= V) return 2;
      post_off[t + 1]++;
    }
  for (int32_t t = 0; t < V; ++t) post_off[t + 1] += post_off[t];
  int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)V);
  if (!cur) return 3;
  memcpy(cur, post_off, sizeof(int64_t) * (size_t)V);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = job_off[i]; p < job_off[i + 1]; ++p) post_ids[cur[job_terms[p]]++] = (uint32_t)i;
  free(cur);
  return 0;
}

/* Job-major bitsets: bitsets[i][w] bit b set iff job i holds term 64*w + b. */
int terms_to_bitsets(int64_t n, int32_t V, const int64_t *job_off, const int32_t *job_terms,
                     uint64_t *bitsets) {
  if (n < 0 || V <= 0) return 1;
  const int64_t W = (V + 63) / 64;
  int err = 0;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    uint64_t *row = bitsets + (size_t)i * (size_t)W;
    memset(row, 0, sizeof(uint64_t) * (size_t)W);
    for (int64_t p = job_off[i]; p < job_off[i + 1]; ++p) {
      int32_t t = job_terms[p];
      if (t < 0 || t >= V) { err = 2; continue; }
      row[t >> 6] |= 1ULL << (t & 63);
    }
  }
  return err;
}

/* document frequency of every term (a histogram of the inputs) */
int term_df(int64_t n, int32_t V, const int64_t *job_off, const int32_t *job_terms, int64_t *df) {
  memset(df, 0, sizeof(int64_t) * (size_t)V);
  for (int64_t p = 0; p < job_off[n]; ++p) {
    int32_t t = job_terms[p];
    if (t < 0 || t >= V) return 2;
    df[t]++;
  }
  return 0;
}
