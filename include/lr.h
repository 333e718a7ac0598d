/*
 * lr.h -- C ABI of a single-GPU (B300, sm_103a) filtered top-K retrieval library.
 *
 * The operation is the on-GPU hybrid retrieval of "Learning to Retrieve for Job
 * Matching" (Sec. 5.3, "System Implementation"; appendix "Optimizing System on
 * GPU"): a term-based filter in conjunctive normal form (F-TBR) fused with a
 * full scan of job embeddings (F-EBR) and a per-query top-K selection, with
 * several queries served by one scan ("Batch Inference").
 *
 * Conventions shared by every entry point:
 *   - Status: every call returns lr_status; LR_OK is 0.  No C++ exception and
 *     no abort crosses the ABI.  lr_last_error_message() describes the last
 *     failure of the calling thread.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are stream-ordered and return before the GPU finishes
 *     unless a pointer argument is host memory, in which case the call copies
 *     through it and synchronises the stream before returning.
 *   - Pointer kinds: arguments documented "host or device" are classified with
 *     cudaPointerGetAttributes (pinned or pageable host memory, device memory,
 *     managed memory).  Arguments documented "host" must be host memory.
 *   - Ownership: the index copies everything it needs into device memory it
 *     owns; the caller keeps ownership of every pointer it passes.
 *   - Scores are FP32 and higher is better.  Ties are broken by ascending job
 *     id, so every result is a deterministic total order.
 *   - Job ids are 0-based row indices below 2^32 - 1.
 */
#ifndef LR_H_
#define LR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lr_status {
  LR_OK = 0,
  LR_ERR_INVALID = 1,     /* argument or input data violates the contract          */
  LR_ERR_NOMEM = 2,       /* device or pinned host allocation failed (create only)  */
  LR_ERR_WORKSPACE = 3,   /* request exceeds what the index's workspace was sized for */
  LR_ERR_CUDA = 4,        /* a CUDA runtime call failed                             */
  LR_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up                     */
  LR_ERR_UNSUPPORTED = 6  /* valid request this build does not implement            */
} lr_status;

typedef enum lr_dtype { LR_F32 = 0, LR_BF16 = 1, LR_FP8_E4M3 = 2 } lr_dtype;

/* LR_DOT: s = <q, x_j>.  LR_COSINE: s = <q, x_j> / (|q| |x_j|), evaluated as the
 * dot product of vectors normalised in FP32 (job rows at create, queries at
 * search); a zero vector scores 0.  (Sec. 5.2 uses cosine similarity.) */
typedef enum lr_metric { LR_DOT = 0, LR_COSINE = 1 } lr_metric;

/* Scoring plan (Sec. 5.3, "EBR first or TBR first").  AUTO picks the plan with
 * the smallest estimated cost from the batch size and the terms' document
 * frequencies. */
typedef enum lr_plan {
  LR_PLAN_AUTO = 0,
  LR_PLAN_GEMV = 1,  /* F-TBR + F-EBR fused: SIMT FP32 matrix-vector scan that
                        tests the CNF per 256-row group and scores passing rows */
  LR_PLAN_TC = 2,    /* F-TBR + F-EBR: tile filter, then tcgen05 tensor-core
                        scoring (3xTF32 split) of the tiles some query passes  */
  LR_PLAN_TBR = 3    /* TBR first (H-TBR): per query the clause with the
                        shortest posting lists gives the candidate rows, the
                        whole CNF is tested on them, only the passing rows are
                        scored (FP32).  Needs an index built from posting lists
                        (each list naming a job at most once), at least one
                        clause per query and at most the query's share of the
                        candidate buffer (max_batch x 65,536 keys from 65,536
                        rows up, split evenly over the batch) postings in the
                        chosen clause; LR_ERR_UNSUPPORTED otherwise.           */
} lr_plan;

typedef struct lr_index lr_index;

/*
 * Index description (appendix "TBR", "Storing Dense Matrix", "Memory
 * Pre-Allocation").
 *
 *   n_jobs, dim      rows and columns of the embedding matrix (dim <= 512).
 *   dtype            LR_F32: the plain method, FP32 rows.
 *                    LR_BF16 / LR_FP8_E4M3: the precision form.  The index keeps
 *                    the FP32 rows and a low-precision copy (BF16 rounded to
 *                    nearest even; or e4m3 with a per-row FP32 scale
 *                    max|x|/448) that the scan reads.  A search then gathers the
 *                    top oversample*K candidates per query by the low-precision
 *                    score, rescores them in FP32 from the FP32 rows, keeps the
 *                    top K, and re-ranks the candidates within the FP32 error
 *                    band of the K-th score by an FP64 dot product.  The
 *                    returned scores are FP32 dot products (FP64 ones rounded to
 *                    FP32 inside the band).  (Appendix "Quantization": a coarse
 *                    low-precision pass followed by exact rescoring.)
 *   metric           lr_metric.
 *   emb              [n_jobs][dim] row-major FP32, host or device.  Must be finite
 *                    (checked; LR_ERR_INVALID otherwise).
 *   vocab            term ids are in [0, vocab).
 *   bitsets          optional [n_jobs][ceil(vocab/64)] uint64 job-major term sets
 *                    (bit t%64 of word t/64 set iff the job holds term t), host or
 *                    device.  Every term becomes a dense term-major bitmap.
 *   post_off,        optional term-major CSR posting lists, host memory:
 *   post_ids         post_ids[post_off[t] .. post_off[t+1]) are the jobs holding
 *                    term t.  Exactly one of bitsets / postings must be given.
 *   n_dense_terms    with postings: the n most frequent terms are kept as dense
 *                    bitmaps (n_jobs bits each); the others stay posting lists and
 *                    are expanded into per-batch bitmaps at search time.  -1 = all.
 *   max_batch        largest batch lr_search accepts (workspace sizing).
 *   max_k            largest K lr_search accepts (<= 4096; precision form:
 *                    oversample * max_k <= 4096).
 *   max_batch_terms  total term occurrences over all filters of one batch that
 *                    the workspace holds (0: 16 per query).
 *   max_sparse_terms distinct posting-list terms one batch may use (0: 256).
 *   oversample       precision form: candidates per query = oversample * K
 *                    (0: 4).  Ignored for LR_F32.
 *   id_base          global id of row 0 (0 for a whole index).  An index over
 *                    rows [id_base, id_base + n_jobs) of a larger job set -- one
 *                    contiguous row shard -- returns global ids; ties still
 *                    break by ascending id, so per-shard results merge exactly
 *                    with lr_merge_topk.  id_base + n_jobs <= 2^31 - 1.
 *   sign_bits,       optional sign-bit codes for the pre-selection of the
 *   sign_bin,        appendix "Quantization" (Sec. 5.3: akin to OP+ORP):
 *   sign_idx,        sign_bits in {128, 256, 512, 1024} (0: none; the paper
 *   sign_sgn         uses 512).  Bit b of a row's code is 1 iff
 *                        sum_{m < sign_bin} sign_sgn[b*sign_bin+m] * x[sign_idx[b*sign_bin+m]] > 0,
 *                    summed in FP32 in m order over the row as given in emb
 *                    (before any normalisation).  sign_idx (int32, in [0, dim))
 *                    and sign_sgn (int8, +1 / -1), host, [sign_bits * sign_bin]
 *                    (sign_bits * sign_bin <= 32768), hold the random draws:
 *                    coordinates permuted and cut into bins, a random sign per
 *                    entry, several permutations when dim < sign_bits.
 *   max_quant_k      largest pre-selection size quant_mult * K a search may ask
 *                    for (0: 200 * max_k); sizes the candidate lists (twice this).
 */
typedef struct lr_index_desc {
  int64_t n_jobs;
  int32_t dim;
  int32_t dtype;
  int32_t metric;
  int32_t vocab;
  const float *emb;
  const uint64_t *bitsets;
  const int64_t *post_off;
  const uint32_t *post_ids;
  int32_t n_dense_terms;
  int32_t max_batch;
  int32_t max_k;
  int32_t max_batch_terms;
  int32_t max_sparse_terms;
  int32_t oversample;
  int64_t id_base;
  int32_t sign_bits;
  int32_t sign_bin;
  const int32_t *sign_idx;
  const int8_t *sign_sgn;
  int64_t max_quant_k;
} lr_index_desc;

/*
 * A batch of B filters in conjunctive normal form (Sec. 5.3: "Each TBR query is
 * transformed into Conjunctive Normal Form"), host memory:
 *   clauses of query b: q_off[b] .. q_off[b+1]   (q_off[0] = 0, non-decreasing)
 *   terms of clause c:  c_off[c] .. c_off[c+1]   (c_off[0] = 0, increasing)
 *   term ids:           terms[i] < vocab
 * A query with zero clauses is unfiltered.  A clause with zero terms is
 * LR_ERR_INVALID (it could never be satisfied).  Terms may repeat or appear in
 * any order.
 */
typedef struct lr_filters {
  const int32_t *q_off;
  const int32_t *c_off;
  const uint32_t *terms;
} lr_filters;

/* Search options; a zero-initialised struct (or NULL) means defaults. */
/* lr_search_opts.flags */
#define LR_SEARCH_ASYNC_HOST 1

typedef struct lr_search_opts {
  int32_t plan;           /* lr_plan                                                  */
  int32_t sample_stride;  /* threshold sample: every n-th 256-row group (0 = auto,
                             -1 = no sample: every passing job is a candidate)        */
  int32_t cand_cap;       /* candidate slots per query (0 = auto; capped by workspace) */
  int32_t force_exact_fallback; /* 1: also run the exact radix fallback for every query */
  int32_t quant_mult;     /* > 0 (index with sign codes): sign-bit pre-selection of
                             about quant_mult * K jobs per query (the paper: 200),
                             then exact FP32 scoring of those only; 0: off.  The
                             pre-selection keeps whole Eq. 4 agreement levels from
                             the top down to the highest level with at least
                             min(quant_mult * K, #passing) jobs at or above it (one
                             level higher if that would exceed 2 * max_quant_k);
                             the result is the exact top K of the kept jobs.  F32
                             indexes only.                                        */
  int32_t flags;          /* 0, or LR_SEARCH_ASYNC_HOST: outputs in page-locked host
                             memory (cudaHostAlloc / cudaHostRegister) are copied in
                             stream order and the call does not synchronise
                             `stream`; the caller synchronises it before reading them.
                             Pageable host outputs and host statistics arrays still
                             make the call synchronise.  A page-locked host query
                             array is then read in stream order too: keep it
                             unchanged until `stream` has been synchronised.      */
  int64_t row_begin;      /* search only job rows [row_begin, row_end) (both 0: every */
  int64_t row_end;        /* row); row_begin a multiple of 256, row_end a multiple of
                             256 or n; ids stay the index's row ids (+ id_base).  The
                             exact top K of the range: its rows are a chunk of the
                             index for a scan that covers the index in steps (the
                             rotating scan of the serving loop).  Not with
                             quant_mult or the TBR-first plan (LR_PLAN_AUTO then
                             chooses a scan).  Invalid ranges: LR_ERR_INVALID.      */
} lr_search_opts;

/* Per-call statistics and instrumentation (every field optional).  Arrays may be
 * device or host memory; a host array makes the call synchronise the stream. */
typedef struct lr_search_stats {
  int64_t *pass_count;   /* [B] jobs passing each filter                            */
  int32_t *cand_count;   /* [B] candidates gathered by the threshold pass           */
  int32_t *fallback;     /* [B] 1 if the exact radix fallback produced the result   */
  int32_t *n_launches;   /* host, 1 value: kernels this call launched               */
  void *scan_start;      /* cudaEvent_t recorded on the stream right before the     */
  void *scan_stop;       /* main scan launches, and right after them                */
  int32_t *n_scan_launches; /* host, 1 value: launches between scan_start/stop     */
  int32_t *rescore_ties; /* [B] precision form: candidates re-ranked in FP64         */
  int32_t *plan_used;    /* host, 1 value: the scan plan the call ran (LR_PLAN_GEMV  */
                         /* or LR_PLAN_TC; LR_PLAN_AUTO picks by the estimated bytes) */
} lr_search_stats;

/* Build an index (allocates every device buffer it will ever use: appendix
 * "Memory Pre-Allocation").  *out receives the handle.  Errors: LR_ERR_INVALID
 * (bad description, non-finite embeddings, term id >= vocab, job id >= n_jobs),
 * LR_ERR_NOMEM, LR_ERR_CUDA.  Synchronises `stream` before returning. */
lr_status lr_index_create(const lr_index_desc *desc, void *stream, lr_index **out);

/* Free an index and its workspace.  NULL is accepted.  The caller must make
 * sure no search on it is still running. */
lr_status lr_index_destroy(lr_index *index);

/* Bytes of device memory held by the index (embeddings, term bitmaps, posting
 * lists, workspace).  Returns 0 for NULL. */
size_t lr_index_device_bytes(const lr_index *index);

/*
 * Filtered top-K search: for each query b the K[b] passing jobs with the
 * highest score, ordered by (score desc, job id asc).
 *
 *   q           [B][dim] FP32 query embeddings, host or device.
 *   B           1 <= B <= max_batch.
 *   f           B CNF filters (host).
 *   k           [B] per-query K (host) or NULL to use k_all for every query;
 *               1 <= K <= max_k.
 *   k_all       K when k is NULL; also the row stride of the outputs, which
 *               must be >= every K.
 *   out_ids     [B][k_all] int32, host or device: job ids, -1 past out_count.
 *   out_scores  [B][k_all] FP32, host or device: scores, -inf past out_count.
 *   out_count   [B] int32, host or device (nullable): min(K[b], #passing).
 *   opts        NULL for defaults.
 *   stats       NULL or per-query statistics.
 *
 * The result is exact: candidates are gathered above a threshold estimated from
 * a sample of the index, and a query whose candidate set cannot prove it holds
 * the top K is finished by an exact radix selection over the whole index.
 * Errors: LR_ERR_INVALID, LR_ERR_WORKSPACE (batch larger than the workspace),
 * LR_ERR_CUDA.
 *
 * Debugging aids (read once per process from the environment; the paper has
 * no counterpart):
 *   LR_PLAN=gemv|simt|tc|tbr  the plan of every search whose options leave it
 *                             to the library (LR_PLAN_AUTO); a forced TBR-first
 *                             plan fails on filters it cannot serve, and is not
 *                             applied to row-range searches.
 *   LR_TIMERS=1               each lr_search / lr_search_ex records CUDA events
 *                             between its stages on `stream`, synchronises the
 *                             stream before returning and prints one line of
 *                             stage times (ms) to stderr.
 * Each stage is also an NVTX range (free when no profiling tool is attached).
 */
lr_status lr_search(lr_index *index, const float *q, int32_t B, const lr_filters *f, const int32_t *k,
                    int32_t k_all, int32_t *out_ids, float *out_scores, int32_t *out_count, void *stream);

lr_status lr_search_ex(lr_index *index, const float *q, int32_t B, const lr_filters *f, const int32_t *k,
                       int32_t k_all, int32_t *out_ids, float *out_scores, int32_t *out_count,
                       const lr_search_opts *opts, const lr_search_stats *stats, void *stream);

/*
 * Allocation-free variant of lr_search.  The paper has no counterpart: it exists
 * for callers that may not call cudaMalloc (a plugin whose host framework owns
 * all device memory through its own pool, or a serving thread where an
 * allocation could block or fail mid-request).  Such callers cannot build an
 * lr_index, so the embeddings, queries, filters (as pass bitmaps) and outputs
 * all come from the caller, and every intermediate lives in one fixed
 * file-scope device array of about 10 MiB that each GPU loading the library
 * keeps until the process exits.  No cudaMalloc, cudaFree or allocating library
 * routine is called.
 *
 *   X            device [n_jobs][dim] FP32, contiguous rows, dim in {32, 64, 128,
 *                256}, base 16-byte aligned (rows are copied in 16-byte pieces);
 *                the score is the plain inner product (normalise beforehand for
 *                cosine).
 *   n_jobs       1 .. 16,777,216.
 *   q            device [B][dim] FP32, contiguous, 1 <= B <= 8.
 *   pass_bitmap  device, nullable (NULL = every job passes).  Row b starts at
 *                pass_bitmap + b * bitmap_stride_words; bit j%32 of word j/32 is
 *                set iff job j may be returned for query b.  The row stride must
 *                be a multiple of 8 words and at least ceil(n_jobs/256)*8 words,
 *                and the base 32-byte aligned (whole 256-job groups are read;
 *                bits past n_jobs are ignored).
 *   k            1 .. 1024; outputs are [B][k] (ids -1 / scores -inf past
 *                out_count) and out_count [B] (nullable), device memory.
 * Results equal lr_search's for the same data and the LR_DOT metric.
 * Sizes beyond these limits return LR_ERR_WORKSPACE (LR_ERR_UNSUPPORTED for
 * dim).  A pointer that is not device (or managed) memory, or that breaks the
 * alignment above (outputs and q: 4 bytes), returns LR_ERR_INVALID before any
 * work is enqueued.  Every call looks up the array's device address with the
 * current device; the first call on a device also loads the library's device
 * code there, so make that first call before any stream capture.  All calls
 * share the array and keep the last call's contents (each call clears what must
 * start at zero, the device error word included), so calls that overlap on the
 * GPU race: serialise them.  Returns after enqueueing the work on `stream`.
 */
lr_status lr_search_noalloc(const float *X, int64_t n_jobs, int32_t dim, const float *q, int32_t B,
                            const uint32_t *pass_bitmap, int64_t bitmap_stride_words, int32_t k, int32_t *out_ids,
                            float *out_scores, int32_t *out_count, void *stream);
/* Wait for `stream` and report the device error word of the last
 * lr_search_noalloc call on the current device (LR_ERR_TIMEOUT: a bounded
 * device wait gave up; LR_ERR_CUDA: inconsistent selection state), then clear
 * it.  Call it after the search and before the next one, whose start clears
 * the word.  Allocates nothing. */
lr_status lr_search_noalloc_status(void *stream);

/*
 * Exact term filter only (F-TBR, Sec. 5.3 and appendix "TBR"): for each query the
 * number of passing jobs and, optionally, the pass bitmap.
 *   out_pass    [B] int64, host or device: number of jobs passing each filter.
 *   out_bitmap  nullable [B][ceil(n_jobs/32)] uint32, host or device: bit j%32 of
 *               word j/32 of row b set iff job j passes filter b.
 */
lr_status lr_filter_count(lr_index *index, const lr_filters *f, int32_t B, int64_t *out_pass,
                          uint32_t *out_bitmap, void *stream);

/* Wait for `stream` and report any error the library's kernels recorded on the
 * device for this index (LR_ERR_TIMEOUT for a bounded wait that gave up). */
lr_status lr_index_sync(lr_index *index, void *stream);

/*
 * Exact merge of per-part top-K lists (Sec. 5.3, "Communication cost": the
 * search splits by job rows; each part -- a row shard, on this GPU or another --
 * returns its own top K' and one exchange brings the lists together).  The top
 * K of a union of disjoint job sets is the top K of the union of each set's top
 * K (K <= K'), so merging the lists under the same order (score desc, id asc)
 * reproduces the unsharded result.
 *
 *   ids, scores  device [G][B][k_in] int32 / FP32: list g of query b, sorted by
 *                (score desc, id asc), ids distinct across lists (global ids).
 *   counts       device [G][B] int32: valid entries of each list (0 .. k_in).
 *   k            1 .. 4096, k <= G * k_in; outputs device [B][k] int32 / FP32
 *                (-1 / -inf past out_count) and out_count [B] (nullable):
 *                min(k, sum_g counts).
 * 1 <= G <= 64.  Lists that break the sort precondition give unspecified (but
 * in-bounds) rows.  Stream-ordered; allocates nothing.
 */
lr_status lr_merge_topk(const int32_t *ids, const float *scores, const int32_t *counts, int32_t G, int32_t B,
                        int32_t k_in, int32_t k, int32_t *out_ids, float *out_scores, int32_t *out_count,
                        void *stream);

/*
 * Sign codes of rows (appendix "Quantization"), the encoding an index with
 * sign_bits builds for its rows and every search for its queries: bit b of row
 * j is 1 iff sum_{m < bin} sgn[b*bin+m] * x[j][idx[b*bin+m]] > 0, summed in FP32
 * in m order; bit b is bit b % 64 of word b / 64 of the row's code.
 *   x      device [n][dim] FP32 (dim <= 256); idx device int32 [nbits * bin] in
 *          [0, dim) (an entry outside reads coordinate 0: wrong codes, never an
 *          out-of-bounds read); sgn device int8 [nbits * bin] (+1 / -1; entries
 *          > 0 count as +1); codes device [n][nbits / 64] uint64, 16-byte aligned.
 *   nbits  128, 256, 512 or 1024; nbits * bin <= 32768.
 * Stream-ordered; allocates nothing.
 */
lr_status lr_sign_encode(const float *x, int64_t n, int32_t dim, int32_t nbits, int32_t bin, const int32_t *idx,
                         const int8_t *sgn, uint64_t *codes, void *stream);

/*
 * Top K of dense score rows (appendix "Fast Top K Selection").  For each row b
 * of scores the k largest (score desc, index asc), written as (index, score).
 *
 *   LR_TOPK_BUCKET  the appendix's selection: bucketised score = (int)(t * G) + G
 *                   with t the score mapped from [lo, hi] onto [-1, 1] (scores
 *                   outside go to the end buckets), buckets counted, the first
 *                   bucket l from the top at which k scores are gathered, and
 *                   only the scores in buckets >= l selected and sorted.
 *   LR_TOPK_RADIX   no bounds: the library's radix select over every score.
 * Both return the exact top k (the bucket pass only narrows the candidates).
 *
 *   scores      device [B][row_stride] FP32, finite; the first n of each row.
 *   k           1 .. 4096; out_ids [B][k] int32 (index in the row, -1 past n)
 *               and out_scores [B][k] FP32 (-inf past n), device.
 *   lo, hi, granularity   bucket method: score bounds and G (1 .. 2048; the
 *               paper uses 100 on cosine scores, lo = -1, hi = 1).
 *   out_threshold_bucket  nullable device [B]: the bucket l of each row.
 *   workspace   device, lr_topk_workspace_size(B, n) bytes, caller-owned.
 * Stream-ordered; allocates nothing.
 */
typedef enum lr_topk_method { LR_TOPK_BUCKET = 0, LR_TOPK_RADIX = 1 } lr_topk_method;
size_t lr_topk_workspace_size(int32_t B, int64_t n);
lr_status lr_topk(const float *scores, int32_t B, int64_t n, int64_t row_stride, int32_t k, int32_t method, float lo,
                  float hi, int32_t granularity, int32_t *out_ids, float *out_scores, int32_t *out_threshold_bucket,
                  void *workspace, size_t workspace_bytes, void *stream);

/*
 * Masked in-batch / sampled softmax loss of the two towers (Sec. 5.1, Eq. 1
 * and Eq. 2) and its gradients, on the tensor cores (BF16 operands, FP32
 * accumulation), recomputing the B x M logits instead of storing them.
 *
 *   z_ij  = inv_tau <Q_i, J_j> for j allowed for query i: bit j of row i of
 *           mask_bits is set (the job meets the query's term constraint), or
 *           j = pos[i] (the positive is always allowed); other columns are
 *           excluded from the softmax (logit -inf).
 *   loss  = (1/B) sum_i ( log sum_{j allowed} exp z_ij  -  z_i,pos[i] )
 *   lse   = [B] the log-sum-exp of each row, saved for the backward pass.
 *   dQ    = d loss / dQ [B][d] FP32,  dJ = d loss / dJ [M][d] FP32, scaled by
 *           *dloss (NULL: 1).
 *
 *   Q [B][d], J [M][d] row-major, dtype LR_BF16 (used as is) or LR_F32 (rounded
 *   to BF16 first); 1 <= d <= 128.  pos [B] int32 in [0, M).  mask_bits
 *   [B][ceil(M/32)] uint32, or NULL (every column allowed).  All pointers are
 *   device memory; workspace holds lr_score_workspace_size(B, M, d) bytes and
 *   is owned by the caller (nothing is allocated).  Stream-ordered and
 *   asynchronous; a positive outside [0, M) makes the loss NaN; a timed-out
 *   device wait is reported by lr_score_status.
 */
size_t lr_score_workspace_size(int32_t B, int32_t M, int32_t d);
lr_status lr_score_forward(const void *Q, const void *J, int32_t B, int32_t M, int32_t d, int32_t dtype,
                           const int32_t *pos, const uint32_t *mask_bits, float inv_tau, float *loss, float *lse,
                           void *workspace, size_t workspace_bytes, void *stream);
lr_status lr_score_backward(const void *Q, const void *J, int32_t B, int32_t M, int32_t d, int32_t dtype,
                            const int32_t *pos, const uint32_t *mask_bits, float inv_tau, const float *lse,
                            const float *dloss, float *dQ, float *dJ, void *workspace, size_t workspace_bytes,
                            void *stream);
/*
 * Online hard-negative mining (Sec. 5.1, "Online Hard Negative Sampling"; Sec.
 * 5.2, the second curriculum stage): for every query i the n_neg allowed
 * columns j != pos[i] with the highest score <Q_i, J_j> (BF16 operands, FP32
 * accumulation, the loss kernels' tensor-core product), ordered by (score desc,
 * column asc).  "Allowed" is the loss's mask (bit j of row i of mask_bits, or
 * every column when NULL).  out_ids / out_scores [B][n_neg] device (-1 / -inf
 * past out_count), out_count [B] (nullable unless out_mask is given):
 * min(n_neg, allowed negatives).  out_mask (nullable) [B][ceil(M/32)] device:
 * the mined columns as a loss mask, so lr_score_forward / lr_score_backward with
 * it compute the loss over each query's positive and its hard negatives only
 * (the m x k training matrix of Sec. 5.1).  1 <= n_neg <= min(4096, M); other
 * arguments as lr_score_forward; workspace: lr_hard_negatives_workspace_size.
 */
size_t lr_hard_negatives_workspace_size(int32_t B, int32_t M, int32_t d);
lr_status lr_hard_negatives(const void *Q, const void *J, int32_t B, int32_t M, int32_t d, int32_t dtype,
                            const int32_t *pos, const uint32_t *mask_bits, int32_t n_neg, int32_t *out_ids,
                            float *out_scores, int32_t *out_count, uint32_t *out_mask, void *workspace,
                            size_t workspace_bytes, void *stream);
/* Synchronise `stream` and report (then clear) a device wait timeout of the last loss call on `workspace`. */
lr_status lr_score_status(void *workspace, int32_t B, int32_t M, int32_t d, void *stream);

/*
 * Serving (appendix "Batch Inference", "Memory Pre-Allocation"): continuous
 * batching of independent requests over a resident index.  The server owns
 * `slots` search contexts that share the index's rows and term storage, each
 * with its own workspace for up to `max_queries` queries and its own CUDA
 * stream, so batches of different slots run on the GPU at the same time.
 * arena_bytes (0: no limit) caps the device memory of the slots: fewer slots
 * than asked are created when they would not fit (memory-based admission).
 * A scheduler thread forms each batch from the pending requests, first come
 * first served, while it fits the slot; requests that arrive while every slot
 * is busy join the next batch a slot forms.  Each request's result is the same
 * as an lr_search of that request alone with the same plan.
 *
 * lr_server_submit copies the request (host q [B][dim] FP32, host filters,
 * host k [B] or NULL with k_all) and returns at once with a ticket; a request
 * with more queries or term occurrences than a slot holds is rejected with
 * LR_ERR_WORKSPACE.  lr_server_wait blocks until the request is done (or
 * timeout_ms passes: LR_ERR_TIMEOUT; negative = no limit), copies its rows into
 * host outputs with row stride k_stride (-1 / -inf padded) and the latency from
 * submit to completion, and releases the ticket.  lr_server_get_stats reports
 * counts and latency percentiles since creation or the last reset.
 * lr_server_destroy finishes pending work and frees the slots (the index stays).
 */
typedef struct lr_server lr_server;
typedef struct lr_server_opts {
  int32_t slots;        /* concurrent batches                          */
  int32_t max_queries;  /* queries per batch (a slot's capacity)       */
  int32_t plan;         /* lr_plan used for every batch                */
  int32_t chunks;       /* <= 1: slots, each batch one whole search;   */
                        /* C >= 2: the rotating scan -- the index in C */
                        /* row chunks, each step scans one chunk for   */
                        /* every active query (one slot of max_queries */
                        /* lanes); a request joins at the next chunk   */
                        /* boundary and is done after C steps, its     */
                        /* chunks' top K merged exactly on the device  */
} lr_server_opts;
typedef struct lr_server_stats {
  int64_t submitted, completed, batches, queries;
  int32_t slots;
  size_t slot_bytes;
  double p50_ms, p99_ms, mean_ms, max_ms, elapsed_s;
} lr_server_stats;
lr_status lr_server_create(lr_index *index, const lr_server_opts *opts, size_t arena_bytes, lr_server **out);
lr_status lr_server_submit(lr_server *server, const float *q, int32_t B, const lr_filters *f, const int32_t *k,
                           int32_t k_all, uint64_t *ticket);
lr_status lr_server_wait(lr_server *server, uint64_t ticket, int32_t timeout_ms, int32_t *out_ids, float *out_scores,
                         int32_t *out_count, int32_t k_stride, double *latency_ms);
lr_status lr_server_get_stats(lr_server *server, lr_server_stats *stats, int32_t reset);
lr_status lr_server_destroy(lr_server *server);

/* Human-readable description of the calling thread's last failure. */
const char *lr_last_error_message(void);

/* ABI version: major * 10000 + minor * 100 + patch. */
int32_t lr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LR_H_ */
