// Internal declarations of the filtered top-K library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "lr.h"

namespace lr {

// ---------------------------------------------------------------- constants
constexpr int kGroupRows = 256;     // rows per predicate group: 8 bitmap words of 32 jobs
constexpr int kGroupWords = 8;
constexpr int kMaxK = 4096;         // largest K (bitonic sort of the survivors in shared memory)
constexpr int kMaxDim = 512;
constexpr int kGemvMaxQ = 8;        // queries per GEMV launch (held in registers)
constexpr int kGemvMaxSlots = 256;  // distinct terms per scan launch (shared-memory word table)
constexpr int kTcMaxQ = 64;         // queries per tensor-core launch (MMA N <= 64)
constexpr int kTc2BlockQ = 48;      // FP32 rows, batches above kTc2MinBatch: queries per block of a two-block launch
constexpr int kTc2MinBatch = 128;   // up to it (and above 64) the two blocks hold 64 queries each
constexpr int kBf16Blocks = 4;      // BF16 / e4m3 rows above 64 queries: 64-query blocks per launch (one N = 256 MMA)
constexpr int kTcMinBatch = 16;     // batches from this size use the tensor-core plan by default
constexpr int kFbBits = 11;         // radix digit of the exact fallback selection
constexpr int kFbBins = 1 << kFbBits;
constexpr int kFbPasses = 6;        // 5 x 11 + 9 = 64 key bits
constexpr int kScanThreads = 256;

// ------------------------------------------------------------- score keys
// A candidate is one 64-bit key: the high word orders FP32 scores (larger key =
// larger score; -0.0 is folded onto +0.0), the low word is ~job_id so that at
// equal scores the smaller id has the larger key.  All keys of one query are
// distinct, so "top K by key" is the (score desc, id asc) order.
__host__ __device__ __forceinline__ uint32_t score_key(float s) {
  s = s + 0.0f;  // -0.0 -> +0.0 (round-to-nearest)
  uint32_t u;
#ifdef __CUDA_ARCH__
  u = __float_as_uint(s);
#else
  __builtin_memcpy(&u, &s, 4);
#endif
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__host__ __device__ __forceinline__ float key_score(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
  float s;
#ifdef __CUDA_ARCH__
  s = __uint_as_float(u);
#else
  __builtin_memcpy(&s, &u, 4);
#endif
  return s;
}

__host__ __device__ __forceinline__ uint64_t make_key(float s, uint32_t id) {
  return ((uint64_t)score_key(s) << 32) | (uint64_t)(0xFFFFFFFFu - id);
}

__host__ __device__ __forceinline__ uint32_t key_id(uint64_t k) { return 0xFFFFFFFFu - (uint32_t)k; }

// ------------------------------------------------------------ row storage
enum ElemType : int { kElemF32 = 0, kElemBF16 = 1, kElemFP8 = 2 };
constexpr float kFp8Max = 448.0f;  // largest finite e4m3 magnitude

// ------------------------------------------------------------ scan launch
enum ScanMode : int {
  kCollect = 0,  // append keys >= tau[q] to the query's buffer
  kHist = 1,     // histogram one radix digit of the keys that match prefix[q]
};

// Device view of one compiled sub-batch of filters and the per-query state.
struct ScanArgs {
  const float *X;        // [n][d_pad] FP32
  const void *Xq;        // [n][d_pad] BF16 or FP8 e4m3 rows when elem != kElemF32
  const float *xscale;   // [n] per-row scale of FP8 rows (score = scale * <q, x8>)
  int32_t elem;          // kElemF32 / kElemBF16 / kElemFP8
  int64_t n;
  int32_t d_pad;
  const float *Q;        // [B][d_pad] FP32 (the whole batch)
  int32_t q_base, nq;    // this launch serves queries q_base .. q_base+nq-1
  // compiled filters of this launch (query and slot ids are launch-local)
  const uint32_t *const *slot_bm;  // [n_slots] term-major bitmap per distinct term
  int32_t n_slots;
  const int32_t *qc_off;  // [nq+1] clause ranges
  const int32_t *cl_off;  // [n_clauses+1] slot ranges
  const int32_t *cl_slot; // slot ids
  int32_t n_cl, n_tm;     // clauses and slot ids of the launch (sizes of cl_off - 1 and cl_slot)
  // 256-row groups visited: g = g_begin + i * g_step, g < n_groups
  int64_t g_begin, g_step, n_groups;
  int32_t mode;
  // per-query state, indexed by the batch-global query id
  const uint64_t *tau;
  uint64_t *buf;
  int64_t buf_cap;
  uint32_t *buf_cnt;
  uint32_t *overflow;
  unsigned long long *pass_cnt;  // nullable
  const uint32_t *active;        // nullable: per-query participation
  const uint32_t *any_active;    // nullable: the launch returns at once when *any_active == 0
  // kHist mode
  uint64_t *prefix;              // [B] key bits fixed so far
  int32_t *krem;                 // [B] rank still to find below the prefix
  uint32_t *hist;                // [B][kFbBins]
  uint64_t *tau_out;             // nullable: the last pass writes the selected key (the new tau)
  uint32_t *done_ctr;            // grid-completion counter (last CTA applies the digit step)
  uint32_t *work_ctr;            // dynamic work distribution (reset by the last CTA)
  int32_t hist_pass;             // 0 .. kFbPasses-1
  int32_t batch;                 // B (for the last-CTA step)
  uint32_t *err;                 // device error word
  // tile list of the tensor-core plan: written by the tile filter, read by the
  // scan, whose last CTA resets the count
  int32_t *tile_row;             // [tile_cap] ids e of the listed 128-row tiles: tile e & 1 of the
                                 // (e >> 1)-th visited group (rows 128 e .. for a full pass)
  void *tile_msg;                // [tile_cap][128] row masks by tile id: bit q = query q passes the row
                                 // (32-bit words if nq <= 32, else 64-bit)
  uint32_t *tile_cnt;            // tiles listed
  int64_t tile_cap;
  int32_t keep_list;             // 1: the scan leaves the list for later launches (else its last CTA empties it)
  // two-block scans (128 queries per tensor-core launch): the tile filter of
  // each 64-query block writes the masks of EVERY visited tile (zero when no
  // query passes) and no list; the scan visits every tile in order and reads
  // block 1's masks from tile_msg2
  int32_t dense_tiles;
  void *tile_msg2;
  int32_t block_q;  // queries per block of a several-block launch (48 or 64)
  int64_t msg_block_stride;  // row-mask words between blocks 1, 2, .. in tile_msg2
};

struct SelectArgs {
  int32_t mode;                  // 0: threshold from a sample, 1: final top-K
  const uint64_t *buf;
  int64_t cap;
  uint32_t *cnt;                 // reset with overflow for the queries a final launch flags
  uint32_t *overflow;
  // threshold mode
  const int32_t *rank;           // [B] r: tau = r-th largest sample key (0 if fewer)
  uint64_t *tau;                 // [B]
  // final mode
  const int32_t *k;              // [B]
  const unsigned long long *pass_cnt;  // [B]
  int32_t k_stride;
  int32_t *out_ids;
  float *out_scores;
  int32_t *out_count;            // nullable
  uint32_t *flag;                // [B] set when the candidate set cannot prove exactness
  uint32_t *n_flagged;
  uint64_t *fb_prefix;           // [B] exact-fallback state, initialised for the queries flagged here
  int32_t *fb_krem;              // [B]
  const uint32_t *only;          // nullable: process only queries with only[q] != 0
  const uint32_t *any;           // nullable: early exit when *any == 0
  int32_t *cand_count_out;       // nullable stats
  int32_t *fallback_out;         // nullable stats
  int32_t fallback_round;        // 1 when this launch finishes fallback queries
  int32_t force_flag;            // 1: flag every query (exercise the exact fallback)
  int32_t unsorted;              // 1: final mode writes the top K in any order (the caller re-ranks them)
  uint32_t *err;                 // device error word
  int64_t id_base;               // added to every written job id (row shards of a larger index)
};

// Programmatic dependent launch: a kernel launched by launch_pdl may be set
// up on the SMs while the kernel before it in the stream is still finishing,
// which hides the launch latency between the search's dependent kernels.
// Such a kernel calls pdl_wait() before it touches global memory; the call
// returns once the previous kernel has completed and its writes are visible
// (launched without the attribute, it returns at once).  The kernels never
// signal early completion, so the next kernel is not placed before every CTA
// of the previous one has exited.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#endif

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Raise a kernel's dynamic shared-memory cap to at least `bytes` on the
// current device.  The cap is a per-function attribute and setting it is a
// costly driver call, so each (function, device) is raised only when a launch
// needs more than it already allows; caps only grow, under a lock, so a
// concurrent caller never lowers the cap another launch relies on.
inline cudaError_t allow_dynamic_smem(const void *fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void *, int>, size_t> allowed;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t &cur = allowed[{fn, dev}];
  if (cur >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_scan_gemv(const ScanArgs &a, int nq_tmpl, int vec, int grid, cudaStream_t s);
// Tile filter (term predicate of the tensor-core plan) and the scan that reads
// its list; launch them back to back on one stream.
cudaError_t launch_tile_filter(const ScanArgs &a, int num_sms, cudaStream_t s);
cudaError_t launch_scan_tc(const ScanArgs &a, const void *tmap_x, int grid, cudaStream_t s);
// The same scan for several query blocks per tile (d <= 128, dense tile masks
// in tile_msg for block 0 and tile_msg2 + (b - 1) msg_block_stride for block b):
// FP32 rows, two blocks of a.block_q (48 or 64) per converted tile; BF16 and
// e4m3 rows, four blocks of 64 in one N = 256 MMA.  The index is read once per
// launch.
cudaError_t launch_scan_tc2(const ScanArgs &a, const void *tmap_x, int grid, cudaStream_t s);
cudaError_t launch_select(const SelectArgs &a, int B, cudaStream_t s);

// Per-query threshold of the sample (the r-th largest sampled key, 0 when the
// sample holds fewer than r keys or overflowed), split over up to 32 CTAs per
// query for large samples.
struct ThrArgs {
  const uint64_t *buf;    // [B][cap] sample keys
  int64_t cap;
  const uint32_t *cnt;    // [B]
  const uint32_t *overflow;
  const int32_t *rank;    // [B] r
  uint64_t *tau;          // [B] out
  uint64_t *scratch;      // [B][8192] the slices' top keys
  uint32_t *slice_n;      // [B][32] keys each slice kept
  uint32_t *done;         // [B] slices finished (zero between launches)
};
constexpr int kThrScratchKeys = 8192;  // per query (the selection's shared-memory key capacity)
cudaError_t launch_threshold(const ThrArgs &a, int B, cudaStream_t s);

// FP32 rescore of the low-precision candidates with an FP64 re-rank of the
// near ties at the K-th score (precision form).
struct RescoreArgs {
  const float *X;          // [n][d_pad] FP32 rows (normalised for cosine)
  int32_t d_pad, dim;
  const float *Q;          // [B][d_pad] FP32 queries (normalised for cosine)
  const int32_t *cid;      // [B][c_stride] candidate ids from the low-precision selection
  const int32_t *ccnt;     // [B] candidates per query
  int32_t c_stride;
  const int32_t *k;        // [B] final K per query
  int32_t k_stride;
  int32_t *out_ids;
  float *out_scores;
  int32_t *out_count;      // nullable
  int32_t *tie_count;      // nullable [B]: candidates re-ranked in FP64
  uint32_t *err;
  uint64_t *keys;          // [B][c_stride] FP32 keys of the candidates (written by the scoring launch)
  uint32_t *gmax;          // [B] bits of max_j sum_k |q_k x_jk| (zero before the scoring launch)
  int64_t id_base;         // added to every written job id (row shards of a larger index)
};
// Two launches: the candidates' FP32 scores over several CTAs per query, then
// per query the K-th key, the FP64 re-rank of the near-tie band and the output.
cudaError_t launch_rescore(const RescoreArgs &a, int B, cudaStream_t s);
// Sign-bit pre-selection (sign.cu).
struct SignScanArgs {
  const uint64_t *codes;      // [n][nbits/64] job codes
  int64_t n;
  int32_t nbits;
  const uint64_t *qcodes;     // [B][nbits/64] query codes
  const uint32_t *pass;       // [B][pass_words] pass bitmaps (bit j of row b: job j passes filter b)
  int64_t pass_words;
  int32_t q_base, nq;         // queries of this launch (nq <= 32)
  int32_t mode;               // 0: histogram of agreement levels, 1: collect jobs at or above level[q]
  uint32_t *hist;             // [B][hist_stride]
  int32_t hist_stride;
  const int32_t *level;       // [B]
  uint64_t *buf;              // [B][cap] job ids
  int64_t cap;
  uint32_t *cnt;              // [B]
};
size_t sign_encode_smem(int nbits, int bin, int dim);
cudaError_t launch_sign_encode(const float *x, int64_t n, int dim, int64_t ld, int nbits, int bin, const int32_t *idx,
                               const int8_t *sgn, uint64_t *codes, int num_sms, cudaStream_t s);
cudaError_t launch_sign_scan(const SignScanArgs &a, int num_sms, cudaStream_t s);
cudaError_t launch_sign_levels(const uint32_t *hist, int hist_stride, int nbits, int B, const int64_t *quant_k,
                               const unsigned long long *pass_cnt, int64_t cap, int32_t *level,
                               unsigned long long *ncand, cudaStream_t s);
cudaError_t launch_sign_rescore(const float *X, int d_pad, const float *Q, uint64_t *buf, int64_t cap,
                                const uint32_t *cnt, int B, int num_sms, cudaStream_t s);
// TBR-first plan (tbr.cu): candidate rows from the postings of one clause per query.
struct TbrRange {
  int64_t begin, end;     // posting-list offsets of one term of the chosen clause
  const uint32_t *bm;     // that term's bitmap (to drop rows an earlier term already produced)
};
struct TbrArgs {
  int64_t n;
  int32_t q_base, nq;                // this launch's queries (CNF tables are launch-local)
  const uint32_t *const *slot_bm;
  const int32_t *qc_off, *cl_off, *cl_slot;
  const int32_t *r_off;              // [B+1] ranges of each (batch-global) query
  const TbrRange *ranges;
  const uint32_t *post_ids;
  uint64_t *buf;                     // [B][cap] kept row ids (the messenger list), scored in place later
  int64_t cap;
  uint32_t *cnt;                     // [B]
  unsigned long long *pass_cnt;      // [B] rows passing the CNF
  uint32_t *err;
};
cudaError_t launch_tbr_collect(const TbrArgs &a, int num_sms, int64_t max_postings, cudaStream_t s);
// Exact merge of G per-part top-K lists per query (merge.cu).
cudaError_t launch_merge_topk(const int32_t *ids, const float *scores, const int32_t *counts, int G, int B, int k_in,
                              int k, int32_t *out_ids, float *out_scores, int32_t *out_count, cudaStream_t s);
// Rotating scan of the serving loop: merge each batch row's chunk result into
// the running top-K of its lane (lane_of[b], k_of[b]); reset lanes; gather the
// rows of finished lanes into a compact block.
cudaError_t launch_lane_merge(const int32_t *c_ids, const float *c_sc, const int32_t *c_cnt, int B, int c_stride,
                              const int32_t *lane_of, const int32_t *k_of, int32_t *run_ids, float *run_sc,
                              int32_t *run_cnt, int run_stride, cudaStream_t s);
cudaError_t launch_lane_reset(const int32_t *lanes, int n, int32_t *run_cnt, cudaStream_t s);
cudaError_t launch_lane_gather(const int32_t *lanes, int n, const int32_t *run_ids, const float *run_sc,
                               const int32_t *run_cnt, int run_stride, int k_stride, int32_t *out_ids, float *out_sc,
                               int32_t *out_cnt, cudaStream_t s);
// Masked softmax loss passes (loss.cu).  Row tiles of 128 over R, streamed
// 64-row tiles of C; see loss.cu for the three modes.
struct LossArgs {
  int32_t B, M;            // queries, jobs (true sizes)
  int32_t dp;              // padded dimension (64 or 128)
  int32_t rows_p;          // padded rows of the forward partials (= padded B)
  int32_t n_ctiles;        // 64-row tiles of C
  int32_t c_per_split;     // C tiles per CTA (grid.y splits the C range)
  float inv_tau;
  float inv_b;             // 1 / B
  const float *dloss;      // device scalar dL (backward; null = 1)
  const int32_t *pos;      // [B] positive column per query
  const uint32_t *mask;    // [B][Mw] bit j of row i: job j allowed for query i (null = all allowed)
  int32_t Mw;
  const float *lse;        // [B] saved log-sum-exp (backward)
  float *part_m, *part_s;  // forward partials [splits][rows_p]
  float *zpos;             // [rows_p] z of each query's positive
  float *out;              // backward output rows (dQ partials or dJ)
  size_t out_split;        // elements between splits of out
  int32_t out_ld, out_cols;
  uint32_t *status;        // device status word (timeouts)
  uint64_t *keys;          // hard negatives: [rows_p][keys_ld] selection keys of the allowed negatives
  int64_t keys_ld;
  uint32_t *key_cnt;       // [B] keys listed per query (zero before the pass)
};
cudaError_t launch_hn_setup(int B, int n_neg, const uint32_t *key_cnt, int32_t *kq, unsigned long long *npass,
                            cudaStream_t s);
cudaError_t launch_hn_mask(const int32_t *ids, const int32_t *count, int B, int n_neg, int Mw, uint32_t *mask,
                           cudaStream_t s);
// Operand copies of two row-major matrices X0, X1 ([rows][d], BF16 or FP32) in one launch: P [rows_p][dp]
// and/or PT [dp][rows_p] BF16, zero padded (null outputs are skipped).
cudaError_t launch_loss_prep(int elem, int d, int dp, const void *X0, int rows0, int rows_p0, void *P0, void *PT0,
                             const void *X1, int rows1, int rows_p1, void *P1, void *PT1, cudaStream_t s);
cudaError_t launch_loss_pass(int mode, const LossArgs &a, int grid_x, int grid_y, const void *tm_r, const void *tm_c,
                             const void *tm_ct, cudaStream_t s);
cudaError_t launch_loss_combine(const LossArgs &a, int splits, float *lse, double *bsum, uint32_t *done, float *loss,
                                cudaStream_t s);
int loss_combine_blocks(int B);  // blocks of launch_loss_combine (one FP64 partial each)
cudaError_t launch_loss_dq_reduce(const float *part, int splits, size_t split_stride, int B, int d, int dp, float *dQ,
                                  cudaStream_t s);
// 2-D tiled TMA descriptor (innermost dimension first); false when the driver
// entry point is unavailable or the encoder rejects the description.
bool encode_tmap_2d(void *tmap, int dtype_code, const void *base, uint64_t dim0, uint64_t dim1, uint64_t stride1,
                    uint32_t box0, uint32_t box1, int swizzle_code);

// Serving slots: search contexts sharing one resident index (runtime.cu).
lr_status index_clone_slot(const lr_index *base, int max_batch, void *stream, lr_index **out);
void index_destroy_slot(lr_index *ix);
int index_max_k(const lr_index *ix);
int index_max_batch_terms(const lr_index *ix);
int index_dim(const lr_index *ix);
int index_vocab(const lr_index *ix);
int index_device(const lr_index *ix);
int64_t index_rows(const lr_index *ix);

cudaError_t launch_quantize_rows(const float *X, int64_t n, int d_pad, int elem, void *Xq, float *scale,
                                 cudaStream_t s);
cudaError_t launch_prep_queries(const float *q_in, float *q_out, int B, int dim, int d_pad, int cosine,
                                uint32_t *err, cudaStream_t s);
// Sorted posting lists -> term-major bitmaps, every word written (no clearing
// needed); spans: [vocab][n_spans + 1] posting offsets at span boundaries.
cudaError_t launch_expand_postings(const int64_t *post_off, const uint32_t *post_ids, const int32_t *spans,
                                   int n_spans, int span_log2, const int32_t *terms, int n_terms, uint32_t *bitmaps,
                                   int64_t n_words, int64_t n, cudaStream_t s);
// Jobs holding each of n_terms term-major bitmaps (popcount), int64 per term.
cudaError_t launch_term_counts(const uint32_t *bitmaps, int n_terms, int64_t n_words, int64_t *out, cudaStream_t s);
cudaError_t launch_scatter_postings(const int64_t *post_off, const uint32_t *post_ids, const int32_t *terms,
                                    int n_terms, uint32_t *bitmaps, int64_t n_words, int64_t n, uint32_t *err,
                                    cudaStream_t s);
cudaError_t launch_rows_to_index(const float *in, float *out, int64_t n, int dim, int d_pad, int cosine,
                                 uint32_t *err, cudaStream_t s);
cudaError_t launch_bitsets_to_termmajor(const uint64_t *bits, int64_t n, int vocab, uint32_t *out, int64_t n_words,
                                        cudaStream_t s);
cudaError_t launch_filter_eval(const ScanArgs &a, unsigned long long *pass_cnt, uint32_t *out_bitmap,
                               int64_t out_words, int out_row0, int grid, cudaStream_t s);

// ------------------------------------------------------------------ errors
void set_error(const std::string &msg);
lr_status fail(lr_status st, const std::string &msg);
lr_status cuda_fail(cudaError_t e, const char *what);

}  // namespace lr
