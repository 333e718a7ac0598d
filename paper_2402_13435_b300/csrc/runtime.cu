// Host runtime of the filtered top-K library: index construction with a
// workspace sized once (appendix "Memory Pre-Allocation"), the per-batch filter
// compiler, the launch plan of a search and the C ABI entry points.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "lr_internal.h"
#include "ptx.h"

namespace lr {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

lr_status fail(lr_status st, const std::string &msg) {
  set_error(msg);
  return st;
}

lr_status cuda_fail(cudaError_t e, const char *what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return LR_ERR_CUDA;
}

}  // namespace lr

using namespace lr;

#define LR_CK(call)                                     \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

// a kernel launch of the search path, counted for the caller's statistics
#define LR_LAUNCH(call) \
  do {                  \
    ++n_launch;         \
    LR_CK(call);        \
  } while (0)

namespace {

bool is_device_ptr(const void *p) {
  if (p == nullptr) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Page-locked host memory: a device-to-host copy into it is ordered on the
// stream and needs no synchronisation before the call returns.
bool is_pinned_host(const void *p) {
  if (p == nullptr) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

// Host outputs need a synchronisation unless the caller asked for stream-ordered
// copies (LR_SEARCH_ASYNC_HOST) and every output is page-locked.
bool host_out_sync(bool async_host, const void *ids, const void *scores, const void *count) {
  return !(async_host && is_pinned_host(ids) && is_pinned_host(scores) && (count == nullptr || is_pinned_host(count)));
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int64_t pow2_ceil(int64_t v) {
  int64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Bump allocator over one device allocation.
struct Carver {
  size_t off = 0;
  template <typename T>
  size_t take(size_t count) {
    off = align_up(off, 256);
    size_t at = off;
    off += count * sizeof(T);
    return at;
  }
};

// One GEMV launch worth of compiled filters (device offsets into the filter region).
struct SubBatch {
  int q_base, nq, n_slots, n_cl, n_tm;
  size_t off_slots, off_qc, off_cl, off_cs;
};

}  // namespace

struct lr_index {
  bool owns_data = true;  // false for a serving slot: rows and term storage belong to the base index
  int device = 0, num_sms = 0;
  int64_t n = 0;
  int64_t id_base = 0;  // global id of row 0 (row shards of a larger index)
  int dim = 0, d_pad = 0, metric = 0, vocab = 0;
  int64_t n_groups = 0, n_words = 0;
  float *X = nullptr;
  // precision form: low-precision copy of X that the scan reads
  int elem = kElemF32;
  void *Xq = nullptr;
  float *xscale = nullptr;
  int oversample = 1;
  int max_kq = 0;  // candidates per query of the low-precision selection (oversample * max_k)
  // term storage
  uint32_t *dense_bm = nullptr;
  int n_dense = 0;
  std::vector<int32_t> term_dense;  // [vocab] dense bitmap index or -1
  std::vector<double> term_frac;    // [vocab] fraction of the jobs holding each term (plan choice)
  bool has_postings = false;
  std::vector<int64_t> post_off_h;
  int64_t *post_off_d = nullptr;
  uint32_t *post_ids_d = nullptr;
  // span table of the posting-list terms (sorted postings only): [vocab][n_spans + 1]
  // offsets of each term's first posting at or after every span of 2^span_log2 words
  int32_t *span_d = nullptr;
  int n_spans = 0, span_log2 = 0;
  // limits
  int max_batch = 0, max_k = 0, max_batch_terms = 0, max_sparse = 0;
  int auto_stride = 0;
  int64_t samp_cap = 0, cand_cap = 0;
  // workspace
  char *ws = nullptr;
  size_t ws_bytes = 0;
  float *q_raw = nullptr, *q_ws = nullptr;
  uint32_t *sparse_bm = nullptr;
  char *state = nullptr;
  size_t state_bytes = 0;
  uint64_t *tau = nullptr, *prefix = nullptr;
  unsigned long long *pass = nullptr;
  uint32_t *cnt = nullptr, *ovf = nullptr, *scnt = nullptr, *sovf = nullptr, *flag = nullptr;
  int32_t *krem = nullptr;
  uint32_t *n_flag = nullptr, *done_ctr = nullptr, *work_ctr = nullptr, *err = nullptr;
  uint32_t *hist = nullptr;
  uint64_t *samp_buf = nullptr, *cand_buf = nullptr;
  int32_t *tile_row = nullptr;  // tile list of the tensor-core plan: main pass
  uint64_t *tile_msg = nullptr;
  uint64_t *tile_msg2 = nullptr;  // d <= 128, batches above 64: the row masks of query blocks 1, 2, ..
  uint32_t *tile_cnt = nullptr;
  int64_t tile_cap = 0;
  uint64_t *thr_scratch = nullptr;  // split threshold selection: [B][8192] keys, [B][32] counts, [B] done
  uint32_t *thr_slice_n = nullptr, *thr_done = nullptr;
  int32_t *tile_row_s = nullptr;  // and of the threshold sample (its own, so both filters can run at once)
  uint64_t *tile_msg_s = nullptr;
  uint32_t *tile_cnt_s = nullptr;
  int64_t tile_cap_s = 0;
  // second stream of the search: the main pass's tile filter runs there while
  // the threshold sample runs on the caller's stream
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int32_t *o_ids = nullptr, *o_cnt = nullptr, *o_cand = nullptr, *o_fb = nullptr;
  int32_t *c_ids = nullptr, *c_cnt = nullptr, *o_ties = nullptr;  // precision form
  uint64_t *rs_keys = nullptr;  // precision form: FP32 keys of the candidates [B][max_kq]
  uint32_t *rs_gmax = nullptr;  // and the per-query FP32 rounding bound's magnitude [B]
  float *c_sc = nullptr;
  float *o_sc = nullptr;
  char *filt_d = nullptr;
  size_t filt_bytes = 0;
  // pinned host staging (double-buffered) and its reuse events
  char *filt_h[2] = {nullptr, nullptr};
  cudaEvent_t filt_ev[2] = {nullptr, nullptr};
  bool filt_ev_live[2] = {false, false};
  int filt_turn = 0;
  // host-side scratch of the filter compiler: term -> batch sparse id and
  // term -> launch-local slot id, each valid while its stamp equals the
  // current generation
  std::vector<int32_t> sparse_stamp, sparse_id, local_stamp, local_id;
  int32_t gen = 0;
  size_t device_bytes = 0;
  // TMA descriptor of X for the tensor-core plan (128 rows x 32 floats, 128-byte swizzle)
  CUtensorMap tmap_x;
  bool have_tmap = false;
  CUtensorMap tmap_xq;  // low-precision rows (precision form)
  bool have_tmap_q = false;
  // sign-bit pre-selection: codes of the rows, the projection, candidate lists
  int sign_bits = 0, sign_bin = 0, sign_W = 0;
  uint64_t *sign_codes = nullptr;  // [n][sign_W]
  int32_t *sign_idx_d = nullptr;   // [sign_bits * sign_bin]
  int8_t *sign_sgn_d = nullptr;
  int64_t sign_max_qk = 0, sign_cap = 0;
  uint32_t *sign_pass = nullptr;   // workspace: [max_batch][n_words] pass bitmaps
  uint64_t *sign_qcodes = nullptr; // [max_batch][sign_W]
  uint64_t *sign_buf = nullptr;    // [max_batch][sign_cap] kept ids, then keys
  int32_t *sign_level = nullptr;   // state block: [max_batch]
  unsigned long long *sign_ncand = nullptr;
};

namespace {

// Debugging aids, read once from the environment:
//   LR_PLAN=gemv|simt|tc|tbr  the plan of every search that asks for LR_PLAN_AUTO
//                             (a forced TBR-first plan fails on filters it cannot
//                             serve, as when the caller forces it);
//   LR_TIMERS=1               every lr_search times its stages with CUDA events on
//                             its stream, synchronises the stream at the end and
//                             prints one line to stderr.
// NVTX ranges name the host side of each stage (no cost without a tool attached).
struct DebugEnv {
  int plan = -1;
  bool timers = false;
};

const DebugEnv &debug_env() {
  static const DebugEnv e = [] {
    DebugEnv d;
    if (const char *p = std::getenv("LR_PLAN")) {
      const std::string v(p);
      if (v == "gemv" || v == "simt") d.plan = LR_PLAN_GEMV;
      else if (v == "tc") d.plan = LR_PLAN_TC;
      else if (v == "tbr") d.plan = LR_PLAN_TBR;
      else if (v == "auto") d.plan = LR_PLAN_AUTO;
    }
    if (const char *t = std::getenv("LR_TIMERS")) d.timers = t[0] != '\0' && t[0] != '0';
    return d;
  }();
  return e;
}

// Stage marks of one call: mark(name) ends the previous stage and starts
// `name` (an NVTX range, and with LR_TIMERS an event recorded on the stream);
// report() waits for the last event and prints the stage times.
class StageTimer {
 public:
  StageTimer(cudaStream_t s, const char *call) : s_(s), call_(call), on_(debug_env().timers) {}
  StageTimer(const StageTimer &) = delete;
  StageTimer &operator=(const StageTimer &) = delete;
  ~StageTimer() {
    if (open_) nvtxRangePop();
    for (cudaEvent_t e : ev_) cudaEventDestroy(e);
  }
  void mark(const char *name) {
    if (open_) nvtxRangePop();
    nvtxRangePushA(name);
    open_ = true;
    if (!on_) return;
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    cudaEventRecord(e, s_);
    ev_.push_back(e);
    names_.push_back(name);
  }
  void report(const std::string &what) {
    if (open_) nvtxRangePop();
    open_ = false;
    if (!on_ || ev_.empty()) return;
    cudaEvent_t end = nullptr;
    if (cudaEventCreate(&end) != cudaSuccess) return;
    cudaEventRecord(end, s_);
    ev_.push_back(end);
    if (cudaEventSynchronize(end) != cudaSuccess) return;
    std::string line = std::string(call_) + " " + what + ":";
    float total = 0.f;
    for (size_t i = 0; i + 1 < ev_.size(); ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev_[i], ev_[i + 1]);
      total += ms;
      char buf[96];
      std::snprintf(buf, sizeof buf, " %s %.3f", names_[i], ms);
      line += buf;
    }
    char buf[64];
    std::snprintf(buf, sizeof buf, " | total %.3f ms\n", total);
    line += buf;
    std::fputs(line.c_str(), stderr);
  }

 private:
  cudaStream_t s_;
  const char *call_;
  bool on_;
  bool open_ = false;
  std::vector<cudaEvent_t> ev_;
  std::vector<const char *> names_;
};

void free_index(lr_index *ix) {
  if (!ix) return;
  if (ix->owns_data) {
    cudaFree(ix->X);
    cudaFree(ix->Xq);
    cudaFree(ix->xscale);
    cudaFree(ix->dense_bm);
    cudaFree(ix->post_off_d);
    cudaFree(ix->post_ids_d);
    cudaFree(ix->span_d);
    cudaFree(ix->sign_codes);
    cudaFree(ix->sign_idx_d);
    cudaFree(ix->sign_sgn_d);
  }
  cudaFree(ix->ws);
  if (ix->ev_fork) cudaEventDestroy(ix->ev_fork);
  if (ix->ev_join) cudaEventDestroy(ix->ev_join);
  if (ix->aux) cudaStreamDestroy(ix->aux);
  for (int i = 0; i < 2; ++i) {
    if (ix->filt_h[i]) cudaFreeHost(ix->filt_h[i]);
    if (ix->filt_ev[i]) cudaEventDestroy(ix->filt_ev[i]);
  }
  delete ix;
}

lr_status check_err_word(lr_index *ix, cudaStream_t s, const char *where) {
  uint32_t e = 0;
  LR_CK(cudaMemcpyAsync(&e, ix->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  LR_CK(cudaStreamSynchronize(s));
  if (e != 0u) {
    LR_CK(cudaMemsetAsync(ix->err, 0, sizeof(uint32_t), s));
    std::string m = std::string(where) + ": ";
    if (e & 1u) m += "non-finite job embedding; ";
    if (e & 4u) m += "posting id >= n_jobs; ";
    if (e & 8u) m += "non-finite query embedding; ";
    if (e & 2u) m += "inconsistent exact-selection state; ";
    if (e & 16u) m += "a bounded device wait timed out; ";
    if (e & 32u) m += "more than 1024 candidates inside the FP64 near-tie band; ";
    if (e & 64u) m += "tile list overflow (internal); ";
    const lr_status st = (e & 16u)          ? LR_ERR_TIMEOUT
                         : (e & (2u | 64u)) ? LR_ERR_CUDA
                         : (e & 32u)        ? LR_ERR_WORKSPACE
                                            : LR_ERR_INVALID;
    return fail(st, m);
  }
  return LR_OK;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to
// the driver library is needed).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// TMA descriptor of the low-precision rows: 128-row tiles of 64 values, BF16
// with the 128-byte swizzle (128-byte rows), e4m3 as bytes with the 64-byte
// swizzle (64-byte rows).  Needs d_pad >= 64.
bool make_xq_tensor_map(lr_index *ix) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || ix->elem == kElemF32 || ix->d_pad < 64 || ix->n >= (int64_t(1) << 31)) return false;
  const bool bf = ix->elem == kElemBF16;
  const cuuint64_t dims[2] = {(cuuint64_t)ix->d_pad, (cuuint64_t)ix->n};
  const cuuint64_t strides[1] = {(cuuint64_t)ix->d_pad * (bf ? 2u : 1u)};
  const cuuint32_t box[2] = {64u, 128u};
  const cuuint32_t estr[2] = {1u, 1u};
  return enc(&ix->tmap_xq, bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, ix->Xq, dims,
             strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             bf ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_x_tensor_map(lr_index *ix) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || ix->n >= (int64_t(1) << 31)) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)ix->d_pad, (cuuint64_t)ix->n};
  const cuuint64_t strides[1] = {(cuuint64_t)ix->d_pad * sizeof(float)};
  const cuuint32_t box[2] = {32u, 128u};
  const cuuint32_t estr[2] = {1u, 1u};
  return enc(&ix->tmap_x, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ix->X, dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Threshold-sample geometry for a given stride: number of sampled groups and
// the rank of the threshold in the sample for a given K.
struct SamplePlan {
  int stride = 0;          // 0: no sample
  int64_t sampled_groups = 0;
  int64_t sampled_rows = 0;
  double frac = 1.0;
};

// Groups [g0, g1) of the index (a search of a row range samples that range).
SamplePlan make_sample_plan(const lr_index *ix, int stride, int64_t g0 = 0, int64_t g1 = -1) {
  SamplePlan p;
  if (g1 < 0) g1 = ix->n_groups;
  if (stride <= 0) return p;
  p.stride = stride;
  const int64_t begin = g0 + stride / 2;
  p.sampled_groups = g1 > begin ? (g1 - begin + stride - 1) / stride : 0;
  int64_t rows = 0;
  if (p.sampled_groups > 0) {
    // every sampled group is full except possibly the last group of the index
    const int64_t last = begin + (p.sampled_groups - 1) * (int64_t)stride;
    rows = (p.sampled_groups - 1) * kGroupRows + std::min<int64_t>(kGroupRows, ix->n - last * kGroupRows);
  }
  p.sampled_rows = rows;
  const int64_t range_rows = std::min<int64_t>(ix->n, g1 * kGroupRows) - g0 * kGroupRows;
  p.frac = range_rows > 0 ? (double)rows / (double)range_rows : 1.0;
  return p;
}

// rank r of the threshold in the sample: the expected number of index keys at or
// above the r-th sample key is r / frac, kept >= 4K and r >= 64 so that fewer
// than K candidates is a > 6-sigma event on exchangeable data.
int32_t sample_rank(const SamplePlan &p, int K) {
  if (p.stride == 0 || p.frac <= 0.0) return 0;
  const double r = std::max(64.0, std::ceil(4.0 * (double)K * p.frac));
  return (int32_t)r;
}

}  // namespace

namespace lr {
bool encode_tmap_2d(void *tmap, int dtype_code, const void *base, uint64_t dim0, uint64_t dim1, uint64_t stride1,
                    uint32_t box0, uint32_t box1, int swizzle_code) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)dim0, (cuuint64_t)dim1};
  const cuuint64_t strides[1] = {(cuuint64_t)stride1};
  const cuuint32_t box[2] = {box0, box1};
  const cuuint32_t estr[2] = {1u, 1u};
  return enc(static_cast<CUtensorMap *>(tmap), (CUtensorMapDataType)dtype_code, 2, const_cast<void *>(base), dims,
             strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, (CUtensorMapSwizzle)swizzle_code,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace lr

namespace {
// Search workspace of an index (sizes from max_batch, max_k, max_kq and the
// sampling geometry), carved from one device allocation, plus the pinned
// double-buffered filter staging and its events.
lr_status alloc_search_workspace(lr_index *ix, cudaStream_t s) {
  // ---- sampling geometry and candidate capacities
  ix->auto_stride = ix->n_groups >= 256 ? (int)std::min<int64_t>(64, ix->n_groups / 16) : 0;
  const SamplePlan sp = make_sample_plan(ix, ix->auto_stride);
  int64_t samp_rows = sp.sampled_rows;
  samp_rows = std::max<int64_t>(samp_rows, std::min<int64_t>(ix->n_groups * kGroupRows / 2 + kGroupRows, 1 << 16));
  ix->samp_cap = samp_rows;
  int64_t cap = 0;
  if (sp.stride > 0) {
    const double r = std::max(64.0, std::ceil(4.0 * ix->max_kq * sp.frac));
    cap = pow2_ceil((int64_t)std::ceil(4.0 * r / sp.frac));
  }
  cap = std::max<int64_t>(cap, std::min<int64_t>(ix->n, 1 << 16));
  cap = std::max<int64_t>(cap, ix->max_kq);
  ix->cand_cap = cap;

  // ---- workspace, one allocation
  const int B = ix->max_batch;
  const int nsp = (ix->has_postings && ix->n_dense < ix->vocab) ? ix->max_sparse : 0;
  // per query: K, final K, sample rank, quantK (24 B); TBR-first: up to 16 posting ranges (24 B) and an offset
  ix->filt_bytes =
      align_up((size_t)B * (24 + 16 * 24 + 8) + (size_t)ix->max_batch_terms * 32 + (size_t)nsp * 4 + 65536, 256);
  Carver cv;
  const size_t o_qraw = cv.take<float>((size_t)B * ix->dim);
  const size_t o_qws = cv.take<float>((size_t)B * ix->d_pad);
  const size_t o_sparse = cv.take<uint32_t>((size_t)nsp * ix->n_words);
  // per-query state block (cleared by one memset per search)
  const size_t o_state = cv.take<char>(0);
  const size_t o_tau = cv.take<uint64_t>(B);
  const size_t o_pre = cv.take<uint64_t>(B);
  const size_t o_pass = cv.take<unsigned long long>(B);
  const size_t o_cnt = cv.take<uint32_t>(B);
  const size_t o_ovf = cv.take<uint32_t>(B);
  const size_t o_scnt = cv.take<uint32_t>(B);
  const size_t o_sovf = cv.take<uint32_t>(B);
  const size_t o_flag = cv.take<uint32_t>(B);
  const size_t o_krem = cv.take<int32_t>(B);
  const size_t o_nflag = cv.take<uint32_t>(1);
  const size_t o_tcnt = cv.take<uint32_t>(1);
  const size_t o_tcnt_s = cv.take<uint32_t>(1);
  const size_t o_thr_done = cv.take<uint32_t>(B);
  const size_t o_rs_gmax = cv.take<uint32_t>(ix->elem != kElemF32 ? B : 0);
  const bool sign = ix->sign_codes != nullptr;
  const size_t o_sg_level = cv.take<int32_t>(sign ? B : 0);
  const size_t o_sg_ncand = cv.take<unsigned long long>(sign ? B : 0);
  const size_t o_state_end = cv.take<char>(0);
  const size_t o_done = cv.take<uint32_t>(2);  // completion counter, work counter
  const size_t o_err = cv.take<uint32_t>(1);
  const size_t o_hist = cv.take<uint32_t>((size_t)B * kFbBins);
  const size_t o_samp = cv.take<uint64_t>((size_t)B * ix->samp_cap);
  const size_t o_cand = cv.take<uint64_t>((size_t)B * ix->cand_cap);
  ix->tile_cap = 2 * ix->n_groups;  // every 128-row tile of the index
  const size_t o_trow = cv.take<int32_t>((size_t)ix->tile_cap);
  const size_t o_tmsg = cv.take<uint64_t>((size_t)ix->tile_cap * 128);
  // two-block scans read the index once per 128 queries (FP32 rows only: the
  // low-precision scans already reach their bound with 64)
  // several-block scans: FP32 rows two blocks, BF16 rows four (one array of
  // row masks per block after the first)
  const int extra_blocks = ix->d_pad > 128 || B <= kTcMaxQ ? 0
                           : ix->elem == kElemF32    ? 1
                                                     : kBf16Blocks - 1;
  const size_t o_tmsg2 = cv.take<uint64_t>((size_t)extra_blocks * ix->tile_cap * 128);
  ix->tile_cap_s = 2 * (ix->samp_cap / kGroupRows + 2);  // the sampled groups' tiles (sample rows <= samp_cap)
  const size_t o_trow_s = cv.take<int32_t>((size_t)ix->tile_cap_s);
  const size_t o_thr_scr = cv.take<uint64_t>((size_t)B * kThrScratchKeys);
  const size_t o_thr_sn = cv.take<uint32_t>((size_t)B * 32);
  const size_t o_tmsg_s = cv.take<uint64_t>((size_t)ix->tile_cap_s * 128);
  const size_t o_oids = cv.take<int32_t>((size_t)B * ix->max_k);
  const size_t o_osc = cv.take<float>((size_t)B * ix->max_k);
  const size_t o_ocnt = cv.take<int32_t>(B);
  const size_t o_ocand = cv.take<int32_t>(B);
  const size_t o_ofb = cv.take<int32_t>(B);
  const bool lowp = ix->elem != kElemF32;
  const size_t o_cids = cv.take<int32_t>(lowp ? (size_t)B * ix->max_kq : 0);
  const size_t o_csc = cv.take<float>(lowp ? (size_t)B * ix->max_kq : 0);
  const size_t o_ccnt = cv.take<int32_t>(lowp ? B : 0);
  const size_t o_ties = cv.take<int32_t>(lowp ? B : 0);
  const size_t o_rs_keys = cv.take<uint64_t>(lowp ? (size_t)B * ix->max_kq : 0);
  const size_t o_sg_pass = cv.take<uint32_t>(sign ? (size_t)B * ix->n_words : 0);
  const size_t o_sg_qc = cv.take<uint64_t>(sign ? (size_t)B * ix->sign_W : 0);
  const size_t o_sg_buf = cv.take<uint64_t>(sign ? (size_t)B * ix->sign_cap : 0);
  const size_t o_filt = cv.take<char>(ix->filt_bytes);
  ix->ws_bytes = align_up(cv.off, 256);
  if (cudaMalloc(&ix->ws, ix->ws_bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(LR_ERR_NOMEM, "cannot allocate the search workspace (" + std::to_string(ix->ws_bytes) +
                                          " bytes); lower max_batch, max_k or max_sparse_terms");
  }
  ix->device_bytes += ix->ws_bytes;
  char *w = ix->ws;
  ix->q_raw = (float *)(w + o_qraw);
  ix->q_ws = (float *)(w + o_qws);
  ix->sparse_bm = nsp ? (uint32_t *)(w + o_sparse) : nullptr;
  ix->state = w + o_state;
  ix->state_bytes = o_state_end - o_state;
  ix->tau = (uint64_t *)(w + o_tau);
  ix->prefix = (uint64_t *)(w + o_pre);
  ix->pass = (unsigned long long *)(w + o_pass);
  ix->cnt = (uint32_t *)(w + o_cnt);
  ix->ovf = (uint32_t *)(w + o_ovf);
  ix->scnt = (uint32_t *)(w + o_scnt);
  ix->sovf = (uint32_t *)(w + o_sovf);
  ix->flag = (uint32_t *)(w + o_flag);
  ix->krem = (int32_t *)(w + o_krem);
  ix->n_flag = (uint32_t *)(w + o_nflag);
  ix->done_ctr = (uint32_t *)(w + o_done);
  ix->work_ctr = ix->done_ctr + 1;
  ix->err = (uint32_t *)(w + o_err);
  ix->hist = (uint32_t *)(w + o_hist);
  ix->samp_buf = (uint64_t *)(w + o_samp);
  ix->cand_buf = (uint64_t *)(w + o_cand);
  ix->tile_row = (int32_t *)(w + o_trow);
  ix->tile_msg = (uint64_t *)(w + o_tmsg);
  ix->tile_msg2 = extra_blocks > 0 ? (uint64_t *)(w + o_tmsg2) : nullptr;
  ix->tile_cnt = (uint32_t *)(w + o_tcnt);
  ix->tile_row_s = (int32_t *)(w + o_trow_s);
  ix->tile_msg_s = (uint64_t *)(w + o_tmsg_s);
  ix->tile_cnt_s = (uint32_t *)(w + o_tcnt_s);
  ix->thr_scratch = (uint64_t *)(w + o_thr_scr);
  ix->thr_slice_n = (uint32_t *)(w + o_thr_sn);
  ix->thr_done = (uint32_t *)(w + o_thr_done);
  ix->o_ids = (int32_t *)(w + o_oids);
  ix->o_sc = (float *)(w + o_osc);
  ix->o_cnt = (int32_t *)(w + o_ocnt);
  ix->o_cand = (int32_t *)(w + o_ocand);
  ix->o_fb = (int32_t *)(w + o_ofb);
  if (lowp) {
    ix->c_ids = (int32_t *)(w + o_cids);
    ix->c_sc = (float *)(w + o_csc);
    ix->c_cnt = (int32_t *)(w + o_ccnt);
    ix->o_ties = (int32_t *)(w + o_ties);
    ix->rs_keys = (uint64_t *)(w + o_rs_keys);
    ix->rs_gmax = (uint32_t *)(w + o_rs_gmax);
  }
  ix->filt_d = w + o_filt;
  if (sign) {
    ix->sign_level = (int32_t *)(w + o_sg_level);
    ix->sign_ncand = (unsigned long long *)(w + o_sg_ncand);
    ix->sign_pass = (uint32_t *)(w + o_sg_pass);
    ix->sign_qcodes = (uint64_t *)(w + o_sg_qc);
    ix->sign_buf = (uint64_t *)(w + o_sg_buf);
  }
  LR_CK(cudaMemsetAsync(ix->done_ctr, 0, 2 * sizeof(uint32_t), s));
  LR_CK(cudaMemsetAsync(ix->err, 0, sizeof(uint32_t), s));
  LR_CK(cudaMemsetAsync(ix->hist, 0, (size_t)B * kFbBins * sizeof(uint32_t), s));
  for (int i = 0; i < 2; ++i) {
    LR_CK(cudaHostAlloc((void **)&ix->filt_h[i], ix->filt_bytes, cudaHostAllocDefault));
    LR_CK(cudaEventCreateWithFlags(&ix->filt_ev[i], cudaEventDisableTiming));
  }
  LR_CK(cudaStreamCreateWithFlags(&ix->aux, cudaStreamNonBlocking));
  LR_CK(cudaEventCreateWithFlags(&ix->ev_fork, cudaEventDisableTiming));
  LR_CK(cudaEventCreateWithFlags(&ix->ev_join, cudaEventDisableTiming));
  ix->sparse_stamp.assign(ix->vocab, 0);
  ix->sparse_id.assign(ix->vocab, -1);
  ix->local_stamp.assign(ix->vocab, 0);
  ix->local_id.assign(ix->vocab, -1);
  return LR_OK;
}

}  // namespace

namespace lr {
// A second search context over the same resident index: it shares the rows,
// the term storage and the TMA descriptors, and owns a workspace sized for
// max_batch queries (serving slots run their batches concurrently).
lr_status index_clone_slot(const lr_index *base, int max_batch, void *stream, lr_index **out) {
  if (!base || !out || max_batch < 1) return fail(LR_ERR_INVALID, "index_clone_slot: bad arguments");
  lr_index *ix = new lr_index(*base);
  ix->owns_data = false;
  ix->device_bytes = 0;
  ix->ws = nullptr;
  ix->aux = nullptr;  // each context gets its own stream and events
  ix->ev_fork = nullptr;
  ix->ev_join = nullptr;
  for (int i = 0; i < 2; ++i) {
    ix->filt_h[i] = nullptr;
    ix->filt_ev[i] = nullptr;
    ix->filt_ev_live[i] = false;
  }
  ix->max_batch_terms = (int)((int64_t)base->max_batch_terms * max_batch / std::max(base->max_batch, 1)) + 64;
  ix->max_batch = max_batch;
  const lr_status st = alloc_search_workspace(ix, (cudaStream_t)stream);
  if (st != LR_OK) {
    free_index(ix);
    return st;
  }
  *out = ix;
  return LR_OK;
}
void index_destroy_slot(lr_index *ix) {
  if (ix) free_index(ix);
}
int index_max_k(const lr_index *ix) { return ix->max_k; }
int index_max_batch_terms(const lr_index *ix) { return ix->max_batch_terms; }
int index_dim(const lr_index *ix) { return ix->dim; }
int index_vocab(const lr_index *ix) { return ix->vocab; }
int index_device(const lr_index *ix) { return ix->device; }
int64_t index_rows(const lr_index *ix) { return ix->n; }
}  // namespace lr

extern "C" {

int32_t lr_version(void) { return 201; }

const char *lr_last_error_message(void) { return g_last_error.c_str(); }

size_t lr_index_device_bytes(const lr_index *index) { return index ? index->device_bytes : 0; }

lr_status lr_index_destroy(lr_index *index) {
  if (!index) return LR_OK;
  cudaSetDevice(index->device);
  free_index(index);
  return LR_OK;
}

lr_status lr_index_create(const lr_index_desc *d, void *stream, lr_index **out) {
  if (!d || !out) return fail(LR_ERR_INVALID, "lr_index_create: null argument");
  *out = nullptr;
  if (d->n_jobs < 1 || d->n_jobs >= 0xFFFFFFFFll) return fail(LR_ERR_INVALID, "n_jobs must be in [1, 2^32-2]");
  if (d->dim < 1 || d->dim > 256) return fail(LR_ERR_UNSUPPORTED, "dim must be in [1, 256]");
  if (d->dtype != LR_F32 && d->dtype != LR_BF16 && d->dtype != LR_FP8_E4M3) return fail(LR_ERR_INVALID, "unknown dtype");
  const int oversample = d->dtype == LR_F32 ? 1 : (d->oversample > 0 ? d->oversample : 4);
  if (d->metric != LR_DOT && d->metric != LR_COSINE) return fail(LR_ERR_INVALID, "unknown metric");
  if (d->vocab < 1) return fail(LR_ERR_INVALID, "vocab must be >= 1");
  if (!d->emb) return fail(LR_ERR_INVALID, "emb is null");
  const bool have_bits = d->bitsets != nullptr;
  const bool have_post = d->post_off != nullptr || d->post_ids != nullptr;
  if (have_bits == have_post) return fail(LR_ERR_INVALID, "give exactly one of bitsets or posting lists");
  if (have_post && (!d->post_off || !d->post_ids)) return fail(LR_ERR_INVALID, "post_off and post_ids both needed");
  if (d->max_batch < 1) return fail(LR_ERR_INVALID, "max_batch must be >= 1");
  if (d->max_k < 1 || d->max_k > kMaxK) return fail(LR_ERR_INVALID, "max_k must be in [1, 4096]");
  if ((int64_t)oversample * d->max_k > kMaxK) return fail(LR_ERR_INVALID, "oversample * max_k must be <= 4096");
  if (d->id_base < 0 || d->id_base + d->n_jobs > 0x7FFFFFFFll)
    return fail(LR_ERR_INVALID, "id_base must be >= 0 and id_base + n_jobs <= 2^31 - 1 (int32 job ids)");
  if (d->sign_bits != 0) {
    const int sb = d->sign_bits;
    if (sb != 128 && sb != 256 && sb != 512 && sb != 1024)
      return fail(LR_ERR_INVALID, "sign_bits must be 0, 128, 256, 512 or 1024");
    if (d->sign_bin < 1 || (int64_t)sb * d->sign_bin > 32768)
      return fail(LR_ERR_INVALID, "sign_bin must be >= 1 with sign_bits * sign_bin <= 32768");
    if (!d->sign_idx || !d->sign_sgn) return fail(LR_ERR_INVALID, "sign_idx and sign_sgn are required");
    if (is_device_ptr(d->sign_idx) || is_device_ptr(d->sign_sgn))
      return fail(LR_ERR_INVALID, "sign_idx and sign_sgn must be host memory");
    for (int64_t i = 0; i < (int64_t)sb * d->sign_bin; ++i) {
      if (d->sign_idx[i] < 0 || d->sign_idx[i] >= d->dim) return fail(LR_ERR_INVALID, "sign_idx entry outside [0, dim)");
      if (d->sign_sgn[i] != 1 && d->sign_sgn[i] != -1) return fail(LR_ERR_INVALID, "sign_sgn entries must be +1 or -1");
    }
    if (d->max_quant_k < 0) return fail(LR_ERR_INVALID, "max_quant_k must be >= 0");
  }

  cudaStream_t s = (cudaStream_t)stream;
  lr_index *ix = new lr_index();
  LR_CK(cudaGetDevice(&ix->device));
  LR_CK(cudaDeviceGetAttribute(&ix->num_sms, cudaDevAttrMultiProcessorCount, ix->device));
  ix->n = d->n_jobs;
  ix->id_base = d->id_base;
  ix->dim = d->dim;
  ix->d_pad = d->dim <= 32 ? 32 : d->dim <= 64 ? 64 : d->dim <= 128 ? 128 : 256;
  ix->metric = d->metric;
  ix->vocab = d->vocab;
  ix->n_groups = (ix->n + kGroupRows - 1) / kGroupRows;
  ix->n_words = ix->n_groups * kGroupWords;
  ix->max_batch = d->max_batch;
  ix->max_k = d->max_k;
  ix->elem = d->dtype == LR_BF16 ? kElemBF16 : d->dtype == LR_FP8_E4M3 ? kElemFP8 : kElemF32;
  ix->oversample = oversample;
  ix->max_kq = oversample * d->max_k;
  ix->max_batch_terms = d->max_batch_terms > 0 ? d->max_batch_terms : 16 * d->max_batch;
  ix->max_sparse = d->max_sparse_terms > 0 ? d->max_sparse_terms : 256;

  auto cleanup = [&](lr_status st) {
    free_index(ix);
    return st;
  };
#define CK2(call)                                                 \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return cleanup(cuda_fail(e_, #call)); \
  } while (0)

  // ---- embeddings
  const size_t xbytes = (size_t)ix->n * (size_t)ix->d_pad * sizeof(float);
  if (cudaMalloc(&ix->X, xbytes) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(fail(LR_ERR_NOMEM, "cannot allocate the embedding matrix"));
  }
  ix->device_bytes += xbytes;
  uint32_t *err_tmp = nullptr;
  CK2(cudaMalloc(&err_tmp, sizeof(uint32_t)));
  CK2(cudaMemsetAsync(err_tmp, 0, sizeof(uint32_t), s));
  const bool cos = d->metric == LR_COSINE;
  if (is_device_ptr(d->emb)) {
    CK2(launch_rows_to_index(d->emb, ix->X, ix->n, ix->dim, ix->d_pad, cos, err_tmp, s));
  } else {
    const int64_t chunk = std::max<int64_t>(1, (64ll << 20) / ((int64_t)ix->dim * 4));
    float *tmp = nullptr;
    CK2(cudaMalloc(&tmp, (size_t)std::min<int64_t>(chunk, ix->n) * ix->dim * sizeof(float)));
    for (int64_t r = 0; r < ix->n; r += chunk) {
      const int64_t m = std::min<int64_t>(chunk, ix->n - r);
      CK2(cudaMemcpyAsync(tmp, d->emb + (size_t)r * ix->dim, (size_t)m * ix->dim * sizeof(float),
                          cudaMemcpyHostToDevice, s));
      CK2(launch_rows_to_index(tmp, ix->X + (size_t)r * ix->d_pad, m, ix->dim, ix->d_pad, cos, err_tmp, s));
      CK2(cudaStreamSynchronize(s));
    }
    cudaFree(tmp);
  }
  if (d->sign_bits != 0) {  // sign codes of the rows as given (before normalisation)
    ix->sign_bits = d->sign_bits;
    ix->sign_bin = d->sign_bin;
    ix->sign_W = d->sign_bits / 64;
    ix->sign_max_qk = d->max_quant_k > 0 ? d->max_quant_k : 200ll * d->max_k;
    ix->sign_cap = 2 * ix->sign_max_qk;
    const size_t np = (size_t)d->sign_bits * d->sign_bin;
    const size_t cbytes = (size_t)ix->n * ix->sign_W * sizeof(uint64_t);
    if (cudaMalloc(&ix->sign_codes, cbytes) != cudaSuccess) {
      cudaGetLastError();
      return cleanup(fail(LR_ERR_NOMEM, "cannot allocate the sign codes"));
    }
    ix->device_bytes += cbytes;
    CK2(cudaMalloc(&ix->sign_idx_d, np * sizeof(int32_t)));
    CK2(cudaMalloc(&ix->sign_sgn_d, np));
    ix->device_bytes += np * 5;
    CK2(cudaMemcpyAsync(ix->sign_idx_d, d->sign_idx, np * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CK2(cudaMemcpyAsync(ix->sign_sgn_d, d->sign_sgn, np, cudaMemcpyHostToDevice, s));
    if (is_device_ptr(d->emb)) {
      CK2(launch_sign_encode(d->emb, ix->n, ix->dim, ix->dim, ix->sign_bits, ix->sign_bin, ix->sign_idx_d,
                             ix->sign_sgn_d, ix->sign_codes, ix->num_sms, s));
    } else {
      const int64_t chunk = std::max<int64_t>(1, (64ll << 20) / ((int64_t)ix->dim * 4));
      float *tmp = nullptr;
      CK2(cudaMalloc(&tmp, (size_t)std::min<int64_t>(chunk, ix->n) * ix->dim * sizeof(float)));
      for (int64_t r = 0; r < ix->n; r += chunk) {
        const int64_t m = std::min<int64_t>(chunk, ix->n - r);
        CK2(cudaMemcpyAsync(tmp, d->emb + (size_t)r * ix->dim, (size_t)m * ix->dim * sizeof(float),
                            cudaMemcpyHostToDevice, s));
        CK2(launch_sign_encode(tmp, m, ix->dim, ix->dim, ix->sign_bits, ix->sign_bin, ix->sign_idx_d,
                               ix->sign_sgn_d, ix->sign_codes + (size_t)r * ix->sign_W, ix->num_sms, s));
        CK2(cudaStreamSynchronize(s));
      }
      cudaFree(tmp);
    }
  }
  if (ix->elem != kElemF32) {  // low-precision copy read by the scan (precision form)
    const size_t qbytes = (size_t)ix->n * ix->d_pad * (ix->elem == kElemBF16 ? 2 : 1);
    if (cudaMalloc(&ix->Xq, qbytes) != cudaSuccess) {
      cudaGetLastError();
      return cleanup(fail(LR_ERR_NOMEM, "cannot allocate the low-precision embedding copy"));
    }
    ix->device_bytes += qbytes;
    if (ix->elem == kElemFP8) {
      CK2(cudaMalloc(&ix->xscale, (size_t)ix->n * sizeof(float)));
      ix->device_bytes += (size_t)ix->n * sizeof(float);
    }
    CK2(launch_quantize_rows(ix->X, ix->n, ix->d_pad, ix->elem, ix->Xq, ix->xscale, s));
  }

  // ---- term storage
  ix->term_dense.assign(ix->vocab, -1);
  const size_t bm_bytes = (size_t)ix->n_words * sizeof(uint32_t);
  if (have_bits) {
    ix->n_dense = ix->vocab;
    if (cudaMalloc(&ix->dense_bm, bm_bytes * ix->n_dense) != cudaSuccess) {
      cudaGetLastError();
      return cleanup(fail(LR_ERR_NOMEM, "cannot allocate term bitmaps"));
    }
    ix->device_bytes += bm_bytes * ix->n_dense;
    CK2(cudaMemsetAsync(ix->dense_bm, 0, bm_bytes * ix->n_dense, s));
    for (int t = 0; t < ix->vocab; ++t) ix->term_dense[t] = t;
    const int64_t W = (ix->vocab + 63) / 64;
    const uint64_t *bits = d->bitsets;
    uint64_t *tmpb = nullptr;
    if (!is_device_ptr(bits)) {
      CK2(cudaMalloc(&tmpb, (size_t)ix->n * W * sizeof(uint64_t)));
      CK2(cudaMemcpyAsync(tmpb, bits, (size_t)ix->n * W * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
      bits = tmpb;
    }
    // bits past vocab in the last word would name terms >= vocab
    CK2(launch_bitsets_to_termmajor(bits, ix->n, ix->vocab, ix->dense_bm, ix->n_words, s));
    CK2(cudaStreamSynchronize(s));
    if (tmpb) cudaFree(tmpb);
    {  // document frequencies for the plan choice
      int64_t *dfd = nullptr;
      CK2(cudaMalloc(&dfd, sizeof(int64_t) * (size_t)ix->vocab));
      std::vector<int64_t> df(ix->vocab);
      CK2(launch_term_counts(ix->dense_bm, ix->vocab, ix->n_words, dfd, s));
      CK2(cudaMemcpyAsync(df.data(), dfd, sizeof(int64_t) * (size_t)ix->vocab, cudaMemcpyDeviceToHost, s));
      CK2(cudaStreamSynchronize(s));
      cudaFree(dfd);
      ix->term_frac.resize(ix->vocab);
      for (int t = 0; t < ix->vocab; ++t) ix->term_frac[t] = (double)df[t] / (double)ix->n;
    }
  } else {
    ix->has_postings = true;
    ix->post_off_h.assign(d->post_off, d->post_off + ix->vocab + 1);
    const std::vector<int64_t> &po = ix->post_off_h;
    ix->term_frac.resize(ix->vocab);
    for (int t = 0; t < ix->vocab; ++t) ix->term_frac[t] = (double)(po[t + 1] - po[t]) / (double)ix->n;
    if (po[0] != 0) return cleanup(fail(LR_ERR_INVALID, "post_off[0] must be 0"));
    for (int t = 0; t < ix->vocab; ++t)
      if (po[t + 1] < po[t]) return cleanup(fail(LR_ERR_INVALID, "post_off must be non-decreasing"));
    const int64_t nnz = po[ix->vocab];
    std::vector<int32_t> order(ix->vocab);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return po[a + 1] - po[a] > po[b + 1] - po[b]; });
    ix->n_dense = d->n_dense_terms < 0 ? ix->vocab : std::min(d->n_dense_terms, ix->vocab);
    std::vector<int32_t> dense_terms(order.begin(), order.begin() + ix->n_dense);
    for (int i = 0; i < ix->n_dense; ++i) ix->term_dense[dense_terms[i]] = i;
    CK2(cudaMalloc(&ix->post_off_d, (size_t)(ix->vocab + 1) * sizeof(int64_t)));
    CK2(cudaMalloc(&ix->post_ids_d, (size_t)std::max<int64_t>(nnz, 1) * sizeof(uint32_t)));
    ix->device_bytes += (size_t)(ix->vocab + 1) * sizeof(int64_t) + (size_t)std::max<int64_t>(nnz, 1) * 4;
    CK2(cudaMemcpyAsync(ix->post_off_d, po.data(), (size_t)(ix->vocab + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                        s));
    if (nnz > 0)
      CK2(cudaMemcpyAsync(ix->post_ids_d, d->post_ids, (size_t)nnz * sizeof(uint32_t),
                          is_device_ptr(d->post_ids) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    if (ix->n_dense > 0) {
      if (cudaMalloc(&ix->dense_bm, bm_bytes * ix->n_dense) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(fail(LR_ERR_NOMEM, "cannot allocate dense term bitmaps"));
      }
      ix->device_bytes += bm_bytes * ix->n_dense;
      CK2(cudaMemsetAsync(ix->dense_bm, 0, bm_bytes * ix->n_dense, s));
      int32_t *terms_d = nullptr;
      CK2(cudaMalloc(&terms_d, sizeof(int32_t) * ix->n_dense));
      CK2(cudaMemcpyAsync(terms_d, dense_terms.data(), sizeof(int32_t) * ix->n_dense, cudaMemcpyHostToDevice, s));
      CK2(launch_scatter_postings(ix->post_off_d, ix->post_ids_d, terms_d, ix->n_dense, ix->dense_bm, ix->n_words,
                                  ix->n, err_tmp, s));
      CK2(cudaStreamSynchronize(s));
      cudaFree(terms_d);
    }
    // Span table for the per-batch expansion of the posting-list terms: when
    // every such list is sorted, a search writes each term's bitmap densely
    // (k_expand_postings) instead of clearing it and scattering with atomics.
    if (ix->n_dense < ix->vocab && nnz > 0 && !is_device_ptr(d->post_ids)) {
      bool sorted = true;
      for (int t = 0; t < ix->vocab && sorted; ++t) {
        if (ix->term_dense[t] >= 0) continue;
        for (int64_t p = po[t] + 1; p < po[t + 1]; ++p)
          if (d->post_ids[p] < d->post_ids[p - 1]) {
            sorted = false;
            break;
          }
      }
      int lg = 11;  // 2048 words (64K rows) per span, wider if the table would pass 256 MB
      auto spans_for = [&](int l) { return (ix->n_words + (int64_t(1) << l) - 1) >> l; };
      while (lg < 13 && (int64_t)ix->vocab * (spans_for(lg) + 1) * 4 > (int64_t(256) << 20)) ++lg;
      const int64_t ns = spans_for(lg);
      if (sorted && (int64_t)ix->vocab * (ns + 1) * 4 <= (int64_t(256) << 20)) {
        std::vector<int32_t> tab((size_t)ix->vocab * (size_t)(ns + 1), 0);
        for (int t = 0; t < ix->vocab; ++t) {
          if (ix->term_dense[t] >= 0) continue;
          const uint32_t *b = d->post_ids + po[t], *e = d->post_ids + po[t + 1];
          int32_t *row = tab.data() + (size_t)t * (size_t)(ns + 1);
          for (int64_t j = 0; j <= ns; ++j) {
            const uint64_t first_row = (uint64_t)j << (lg + 5);
            row[j] = (int32_t)(std::lower_bound(b, e, first_row, [](uint32_t x, uint64_t v) { return (uint64_t)x < v; }) - b);
          }
        }
        CK2(cudaMalloc(&ix->span_d, tab.size() * sizeof(int32_t)));
        ix->device_bytes += tab.size() * sizeof(int32_t);
        CK2(cudaMemcpyAsync(ix->span_d, tab.data(), tab.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        CK2(cudaStreamSynchronize(s));
        ix->n_spans = (int)ns;
        ix->span_log2 = lg;
      }
    }
  }

  {
    const lr_status wst = alloc_search_workspace(ix, s);
    if (wst != LR_OK) return cleanup(wst);
  }

  // ---- input validity recorded by the build kernels
  uint32_t e = 0;
  CK2(cudaMemcpyAsync(&e, err_tmp, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  CK2(cudaStreamSynchronize(s));
  cudaFree(err_tmp);
  if (e & 1u) return cleanup(fail(LR_ERR_INVALID, "non-finite value in the job embeddings"));
  if (e & 4u) return cleanup(fail(LR_ERR_INVALID, "posting list names a job id >= n_jobs"));
  ix->have_tmap = make_x_tensor_map(ix);
  ix->have_tmap_q = make_xq_tensor_map(ix);
  *out = ix;
  return LR_OK;
#undef CK2
}

}  // extern "C"

// --------------------------------------------------------------- filter compiler
namespace {

struct Compiled {
  std::vector<SubBatch> subs;
  std::vector<int32_t> sparse_terms;  // distinct posting-list terms of the batch
  size_t off_k = 0, off_kfin = 0, off_rank = 0, off_sparse = 0, bytes = 0;
};

// Estimated pass rate of every filter of the batch (terms independent):
//     s_q = prod_c (1 - prod_{t in c} (1 - df_t / n)).
// false when the index has no term statistics or the filters are malformed
// (which the filter compiler reports).
bool estimate_pass_rates(const lr_index *ix, const lr_filters *f, int B, std::vector<double> &s) {
  if (ix->term_frac.empty() || !f || !f->q_off || f->q_off[0] != 0) return false;
  for (int b = 0; b < B; ++b)
    if (f->q_off[b + 1] < f->q_off[b]) return false;
  if (f->q_off[B] > 0 && (!f->c_off || !f->terms || f->c_off[0] != 0)) return false;
  for (int c = 0; c < f->q_off[B]; ++c)
    if (f->c_off[c + 1] <= f->c_off[c]) return false;
  s.assign(B, 1.0);
  for (int b = 0; b < B; ++b) {
    for (int c = f->q_off[b]; c < f->q_off[b + 1]; ++c) {
      double none = 1.0;
      for (int i = f->c_off[c]; i < f->c_off[c + 1]; ++i) {
        const uint32_t t = f->terms[i];
        none *= 1.0 - (t < (uint32_t)ix->vocab ? ix->term_frac[t] : 0.0);
      }
      s[b] *= 1.0 - none;
    }
  }
  return true;
}

// Scan plan for LR_PLAN_AUTO from the estimated pass rates s_q: the union of a
// launch's queries is u = 1 - prod_q (1 - s_q).  Estimated times, fitted to
// the 10M x 128 FP32 selectivity sweep (each plan forced, batches 1 to 1,024)
// and scaled by the rows:
//   SIMT scan, per launch of up to 8 queries: ~55 us of threshold sample and
//     selections, the predicate's visit of every 256-row group (50 us + 2 us
//     per query per 10M rows), and the union's rows at 6.9 TB/s (up to four
//     queries) or 5.3 TB/s (more: the FMAs per row count), down to 60 % of
//     that when the rows are scattered (u -> 0), each passing row costing
//     ~18 ps more in the sample and the selections; a row costs at least the
//     FMAs of its d values per query, as an FP32 row of d values would;
//   tensor-core scan: the tile filter (60 us per 10M rows) plus, per launch of
//     up to 64 queries, the listed tiles (a tile is listed when one of its 128
//     rows passes: 1 - (1 - u)^128 of them) streamed at 5.2 TB/s; FP32 rows
//     above 64 queries run one 128-query launch at 2.0 TB/s of rows (up to
//     128 queries) or 96-query launches at 3.5 TB/s of rows, each with
//     ~0.25 ms per 10M rows of filters and selections;
//   and each plan's fixed launches (prep, expansion, sample, selection and the
//     exact fallback's early-exit launches): ~30 us.
// Without estimates the batch size decides (>= 16 queries: tensor cores).
double gemv_time_s(int64_t n, double rb, int dp, int B, const std::vector<double> &s) {
  const double scale = (double)n / 1e7;
  double t = 30e-6;
  for (int b0 = 0; b0 < B; b0 += kGemvMaxQ) {
    const int nq = std::min(B, b0 + kGemvMaxQ) - b0;
    double none = 1.0;
    for (int b = b0; b < b0 + nq; ++b) none *= 1.0 - s[b];
    const double u = 1.0 - none;
    const double bw = (nq <= 4 ? 6.9e12 : 5.3e12) * (u < 0.1 ? 0.6 + 4.0 * u : 1.0);
    const double row_bytes = std::max(rb, 0.5 * dp * nq);  // FMA floor: an FP32 row at eight queries
    t += 55e-6 + (50e-6 + 2e-6 * nq) * scale + u * (double)n * (row_bytes / bw + 1.8e-11);
  }
  return t;
}

double tc_time_s(int64_t n, double rb, bool fp32, int B, const std::vector<double> &s) {
  const double scale = (double)n / 1e7;
  double t = 30e-6 + 60e-6 * scale;
  const bool blocks = fp32 && B > kTcMaxQ;
  const int per = !blocks ? kTcMaxQ : B <= 2 * kTcMaxQ ? 2 * kTcMaxQ : 96;
  for (int b0 = 0; b0 < B; b0 += per) {
    double none = 1.0;
    for (int b = b0; b < std::min(B, b0 + per); ++b) none *= 1.0 - s[b];
    const double u = 1.0 - none;
    const double tiles = (1.0 - std::pow(1.0 - u, 128.0)) * (double)n * rb;
    if (!blocks)
      t += tiles / 5.2e12 + 10e-6;
    else
      t += tiles / (per == 96 ? 3.5e12 : 2.0e12) + 0.25e-3 * scale;
  }
  return t;
}

int choose_plan(const lr_index *ix, int B, bool tc_ok, bool have_est, const std::vector<double> &s) {
  if (!tc_ok) return LR_PLAN_GEMV;
  if (!have_est) return B >= kTcMinBatch ? LR_PLAN_TC : LR_PLAN_GEMV;
  const double rb = 4.0 * ix->d_pad * (ix->elem == kElemF32 ? 1.0 : ix->elem == kElemBF16 ? 0.5 : 0.25);
  const bool fp32 = ix->elem == kElemF32;
  return tc_time_s(ix->n, rb, fp32, B, s) < gemv_time_s(ix->n, rb, ix->d_pad, B, s) ? LR_PLAN_TC : LR_PLAN_GEMV;
}

// TBR-first choice per query: the clause whose distinct terms have the fewest
// postings (the smaller set of the paper's intersection argument).  ok is
// false when the index has no posting lists, a query has no clause, or a
// chosen clause has more postings than `cap`.
struct TbrPlan {
  bool ok = false;
  std::vector<int32_t> clause;     // [B] chosen clause (global clause index)
  std::vector<int64_t> postings;   // [B] postings of that clause
  int64_t max_postings = 0;
};

TbrPlan plan_tbr(const lr_index *ix, const lr_filters *f, int B, int64_t cap) {
  TbrPlan P;
  if (!ix->has_postings || !f || !f->q_off || !f->c_off || !f->terms) return P;
  P.clause.assign(B, -1);
  P.postings.assign(B, 0);
  const std::vector<int64_t> &po = ix->post_off_h;
  for (int b = 0; b < B; ++b) {
    const int c0 = f->q_off[b], c1 = f->q_off[b + 1];
    if (c1 <= c0) return P;
    int64_t best = -1;
    for (int c = c0; c < c1; ++c) {
      int64_t tot = 0;
      for (int i = f->c_off[c]; i < f->c_off[c + 1]; ++i) {
        const uint32_t t = f->terms[i];
        if (t >= (uint32_t)ix->vocab) return P;
        bool seen = false;  // a repeated term adds no rows
        for (int i2 = f->c_off[c]; i2 < i; ++i2) seen |= f->terms[i2] == t;
        if (!seen) tot += po[t + 1] - po[t];
      }
      if (best < 0 || tot < best) {
        best = tot;
        P.clause[b] = c;
      }
    }
    if (best > cap) return P;
    int distinct = 0;  // the collect kernel holds up to 16 ranges per query
    const int c = P.clause[b];
    for (int i = f->c_off[c]; i < f->c_off[c + 1]; ++i) {
      bool seen = false;
      for (int i2 = f->c_off[c]; i2 < i; ++i2) seen |= f->terms[i2] == f->terms[i];
      distinct += seen ? 0 : 1;
    }
    if (distinct > 16) return P;
    P.postings[b] = best;
    P.max_postings = std::max(P.max_postings, best);
  }
  P.ok = true;
  return P;
}

// Estimated time of the TBR-first plan against the scans' (choose_plan): the
// postings and their bit tests (term words mostly L2 hits: ~16 B of traffic
// per posting at 3.2 TB/s), the passing rows gathered in FP32 at 2 TB/s, the
// selection of every passing row as a candidate (one CTA per query, ~1.1 ns
// per candidate of the largest list: 0.14 ms for a 1 % filter over 10M rows),
// and a fixed 12 us (five launches, against the scans' dozen).  TBR first is
// taken when it is estimated at less than half the cheaper scan.
bool tbr_cheaper(const lr_index *ix, int B, const TbrPlan &T, const std::vector<double> &est, bool tc_ok) {
  const double rb = 4.0 * ix->d_pad, n = (double)ix->n;
  double tbr = 12e-6, cand_max = 0.0;
  for (int b = 0; b < B; ++b) {
    tbr += 16.0 * (double)T.postings[b] / 3.2e12 + est[b] * n * 4.0 * ix->d_pad / 2.0e12;
    cand_max = std::max(cand_max, est[b] * n);
  }
  tbr += 1.1e-9 * cand_max;
  const double rbs = rb * (ix->elem == kElemF32 ? 1.0 : ix->elem == kElemBF16 ? 0.5 : 0.25);
  const double gemv = gemv_time_s(ix->n, rbs, ix->d_pad, B, est);
  const double scan = tc_ok ? std::min(gemv, tc_time_s(ix->n, rbs, ix->elem == kElemF32, B, est)) : gemv;
  return tbr < 0.5 * scan;
}

// The batch's posting-list terms -> workspace bitmaps (step A1): a dense write
// of every word when the index has a span table, else clear + scatter.
cudaError_t expand_sparse_terms(lr_index *ix, const Compiled &C, cudaStream_t s) {
  const int32_t *terms = (const int32_t *)(ix->filt_d + C.off_sparse);
  const int nt = (int)C.sparse_terms.size();
  if (ix->span_d)
    return launch_expand_postings(ix->post_off_d, ix->post_ids_d, ix->span_d, ix->n_spans, ix->span_log2, terms, nt,
                                  ix->sparse_bm, ix->n_words, ix->n, s);
  const cudaError_t e = cudaMemsetAsync(ix->sparse_bm, 0, (size_t)ix->n_words * nt * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  return launch_scatter_postings(ix->post_off_d, ix->post_ids_d, terms, nt, ix->sparse_bm, ix->n_words, ix->n, ix->err,
                                 s);
}

// Validate the CNF batch and lay out, in the pinned staging buffer, the
// per-launch slot tables and clause lists.  Slot pointers are device addresses
// of dense index bitmaps or of workspace bitmaps for posting-list terms.
lr_status compile_filters(lr_index *ix, const lr_filters *f, int B, int max_q_per_launch, char *stage,
                          Compiled &C) {
  if (!f || !f->q_off || (!f->c_off && B > 0)) return fail(LR_ERR_INVALID, "filters: null arrays");
  const int32_t *qo = f->q_off, *co = f->c_off;
  if (qo[0] != 0) return fail(LR_ERR_INVALID, "filters: q_off[0] must be 0");
  for (int b = 0; b < B; ++b)
    if (qo[b + 1] < qo[b]) return fail(LR_ERR_INVALID, "filters: q_off must be non-decreasing");
  const int nC = qo[B];
  if (nC > 0 && !f->terms) return fail(LR_ERR_INVALID, "filters: terms is null");
  if (nC > 0 && co[0] != 0) return fail(LR_ERR_INVALID, "filters: c_off[0] must be 0");
  for (int c = 0; c < nC; ++c)
    if (co[c + 1] <= co[c]) return fail(LR_ERR_INVALID, "filters: a clause with zero terms can never pass");
  const int nT = nC > 0 ? co[nC] : 0;
  if (nT > ix->max_batch_terms) return fail(LR_ERR_WORKSPACE, "filters: more term occurrences than max_batch_terms");
  for (int i = 0; i < nT; ++i)
    if (f->terms[i] >= (uint32_t)ix->vocab) return fail(LR_ERR_INVALID, "filters: term id >= vocab");

  // batch-level: distinct posting-list terms get a workspace bitmap each
  const int32_t bgen = ++ix->gen;
  C.sparse_terms.clear();
  for (int i = 0; i < nT; ++i) {
    const int32_t t = (int32_t)f->terms[i];
    if (ix->term_dense[t] >= 0 || ix->sparse_stamp[t] == bgen) continue;
    ix->sparse_stamp[t] = bgen;
    ix->sparse_id[t] = (int32_t)C.sparse_terms.size();
    C.sparse_terms.push_back(t);
  }
  if ((int)C.sparse_terms.size() > ix->max_sparse)
    return fail(LR_ERR_WORKSPACE, "filters: more distinct posting-list terms than max_sparse_terms");

  size_t off = 0;
  auto take = [&](size_t bytes, size_t al) {
    off = align_up(off, al);
    size_t at = off;
    off += bytes;
    return at;
  };
  C.off_k = take(sizeof(int32_t) * B, 16);
  C.off_kfin = take(sizeof(int32_t) * B, 16);
  C.off_rank = take(sizeof(int32_t) * B, 16);
  C.off_sparse = take(sizeof(int32_t) * std::max<size_t>(C.sparse_terms.size(), 1), 16);
  if (off > ix->filt_bytes) return fail(LR_ERR_WORKSPACE, "filters: staging area too small");
  if (!C.sparse_terms.empty())
    std::memcpy(stage + C.off_sparse, C.sparse_terms.data(), sizeof(int32_t) * C.sparse_terms.size());

  // launch-level: runs of up to max_q_per_launch queries whose distinct terms
  // fit the kernel's shared-memory word table (kGemvMaxSlots)
  const size_t bm_words = (size_t)ix->n_words;
  C.subs.clear();
  int b = 0;
  while (b < B) {
    const int32_t lgen = ++ix->gen;
    std::vector<int32_t> slots;  // distinct terms of this launch in first-use order
    int e = b;
    while (e < B && e - b < max_q_per_launch) {
      const size_t before = slots.size();
      for (int c = qo[e]; c < qo[e + 1]; ++c)
        for (int i = co[c]; i < co[c + 1]; ++i) {
          const int32_t t = (int32_t)f->terms[i];
          if (ix->local_stamp[t] == lgen) continue;
          ix->local_stamp[t] = lgen;
          ix->local_id[t] = (int32_t)slots.size();
          slots.push_back(t);
        }
      if ((int)slots.size() > kGemvMaxSlots) {
        if (e == b) return fail(LR_ERR_UNSUPPORTED, "a single filter uses more than 256 distinct terms");
        for (size_t i = before; i < slots.size(); ++i) ix->local_stamp[slots[i]] = 0;  // query e starts the next run
        slots.resize(before);
        break;
      }
      ++e;
    }
    SubBatch sb;
    sb.q_base = b;
    sb.nq = e - b;
    sb.n_slots = (int)slots.size();
    const int ncl = qo[e] - qo[b];
    const int ntm = ncl > 0 ? co[qo[e]] - co[qo[b]] : 0;
    sb.n_cl = ncl;
    sb.n_tm = ntm;
    sb.off_slots = take(sizeof(uint64_t) * std::max<size_t>(slots.size(), 1), 16);
    sb.off_qc = take(sizeof(int32_t) * (sb.nq + 1), 16);
    sb.off_cl = take(sizeof(int32_t) * (ncl + 1), 16);
    sb.off_cs = take(sizeof(int32_t) * std::max(ntm, 1), 16);
    if (off > ix->filt_bytes) return fail(LR_ERR_WORKSPACE, "filters: staging area too small");
    uint64_t *sp = (uint64_t *)(stage + sb.off_slots);
    for (size_t i = 0; i < slots.size(); ++i) {
      const int32_t t = slots[i];
      const uint32_t *ptr = ix->term_dense[t] >= 0 ? ix->dense_bm + (size_t)ix->term_dense[t] * bm_words
                                                   : ix->sparse_bm + (size_t)ix->sparse_id[t] * bm_words;
      sp[i] = (uint64_t)(uintptr_t)ptr;
    }
    int32_t *qc = (int32_t *)(stage + sb.off_qc);
    int32_t *cl = (int32_t *)(stage + sb.off_cl);
    int32_t *cs = (int32_t *)(stage + sb.off_cs);
    int ci = 0, ti = 0;
    qc[0] = 0;
    cl[0] = 0;
    for (int qq = b; qq < e; ++qq) {
      for (int c = qo[qq]; c < qo[qq + 1]; ++c) {
        for (int i = co[c]; i < co[c + 1]; ++i) cs[ti++] = ix->local_id[(int32_t)f->terms[i]];
        cl[++ci] = ti;
      }
      qc[qq - b + 1] = ci;
    }
    C.subs.push_back(sb);
    b = e;
  }
  C.bytes = off;
  return LR_OK;
}

}  // namespace

// ------------------------------------------------------------------ search
namespace {

// Search with the sign-bit pre-selection (appendix "Quantization"): the CNF
// filter gives pass bitmaps, the Eq. 4 agreement of the passing jobs with the
// query's code is histogrammed, whole agreement levels from the top are kept
// down to about quant_mult * K jobs, and only those are scored exactly (FP32)
// and selected.  TBR -> Quant -> EBR, as the appendix chains them.
lr_status run_sign_search(lr_index *ix, const float *q, int B, const lr_filters *f, const int32_t *k, int k_all,
                          int32_t *out_ids, float *out_scores, int32_t *out_count, const lr_search_opts &o,
                          const lr_search_stats *stats, cudaStream_t s) {
  if (o.quant_mult < 0) return fail(LR_ERR_INVALID, "quant_mult must be >= 0");
  if (!ix->sign_codes) return fail(LR_ERR_UNSUPPORTED, "the index has no sign codes (sign_bits = 0)");
  if (ix->elem != kElemF32) return fail(LR_ERR_UNSUPPORTED, "sign-bit pre-selection needs an LR_F32 index");
  const int turn = ix->filt_turn;
  ix->filt_turn ^= 1;
  if (ix->filt_ev_live[turn]) LR_CK(cudaEventSynchronize(ix->filt_ev[turn]));
  char *stage = ix->filt_h[turn];
  Compiled C;
  lr_status st = compile_filters(ix, f, B, 32, stage, C);
  if (st != LR_OK) return st;
  int32_t *kf = (int32_t *)(stage + C.off_kfin);
  const size_t off_qk = align_up(C.bytes, 16);
  if (off_qk + sizeof(int64_t) * B > ix->filt_bytes) return fail(LR_ERR_WORKSPACE, "filters: staging area too small");
  int64_t *qk = (int64_t *)(stage + off_qk);
  for (int b = 0; b < B; ++b) {
    const int kb = k ? k[b] : k_all;
    if (kb < 1 || kb > ix->max_k || kb > k_all) return fail(LR_ERR_INVALID, "K must be in [1, min(max_k, k_all)]");
    kf[b] = kb;
    qk[b] = (int64_t)o.quant_mult * kb;
    if (qk[b] > ix->sign_max_qk) return fail(LR_ERR_WORKSPACE, "quant_mult * K exceeds the index's max_quant_k");
  }
  const size_t bytes = off_qk + sizeof(int64_t) * B;
  int32_t n_launch = 0;
  LR_CK(cudaMemcpyAsync(ix->filt_d, stage, bytes, cudaMemcpyHostToDevice, s));
  LR_CK(cudaEventRecord(ix->filt_ev[turn], s));
  ix->filt_ev_live[turn] = true;
  LR_CK(cudaMemsetAsync(ix->state, 0, ix->state_bytes, s));
  LR_CK(cudaMemsetAsync(ix->hist, 0, (size_t)B * kFbBins * sizeof(uint32_t), s));
  const int32_t *kfin_d = (const int32_t *)(ix->filt_d + C.off_kfin);
  const int64_t *qk_d = (const int64_t *)(ix->filt_d + off_qk);
  const float *qsrc = q;
  if (!is_device_ptr(q)) {
    LR_CK(cudaMemcpyAsync(ix->q_raw, q, sizeof(float) * (size_t)B * ix->dim, cudaMemcpyHostToDevice, s));
    qsrc = ix->q_raw;
  }
  LR_LAUNCH(launch_prep_queries(qsrc, ix->q_ws, B, ix->dim, ix->d_pad, ix->metric == LR_COSINE, ix->err, s));
  // the query codes come from the queries as given, like the rows' codes
  LR_LAUNCH(launch_sign_encode(qsrc, B, ix->dim, ix->dim, ix->sign_bits, ix->sign_bin, ix->sign_idx_d,
                               ix->sign_sgn_d, ix->sign_qcodes, ix->num_sms, s));
  if (!C.sparse_terms.empty()) {
    ++n_launch;
    LR_CK(expand_sparse_terms(ix, C, s));
  }
  // TBR: pass bitmaps and counts of every filter
  for (const SubBatch &sb : C.subs) {
    ScanArgs a{};
    a.n = ix->n;
    a.q_base = sb.q_base;
    a.nq = sb.nq;
    a.slot_bm = (const uint32_t *const *)(ix->filt_d + sb.off_slots);
    a.n_slots = sb.n_slots;
    a.qc_off = (const int32_t *)(ix->filt_d + sb.off_qc);
    a.cl_off = (const int32_t *)(ix->filt_d + sb.off_cl);
    a.cl_slot = (const int32_t *)(ix->filt_d + sb.off_cs);
    a.n_groups = ix->n_groups;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((ix->n_groups + 7) / 8, (int64_t)ix->num_sms * 4));
    LR_LAUNCH(launch_filter_eval(a, ix->pass, ix->sign_pass, ix->n_words, 0, grid, s));
  }
  // Quant: agreement levels, the level of each query, the kept jobs
  SignScanArgs g{};
  g.codes = ix->sign_codes;
  g.n = ix->n;
  g.nbits = ix->sign_bits;
  g.qcodes = ix->sign_qcodes;
  g.pass = ix->sign_pass;
  g.pass_words = ix->n_words;
  g.hist = ix->hist;
  g.hist_stride = kFbBins;
  g.level = ix->sign_level;
  g.buf = ix->sign_buf;
  g.cap = ix->sign_cap;
  g.cnt = ix->cnt;
  if (stats && stats->scan_start) LR_CK(cudaEventRecord((cudaEvent_t)stats->scan_start, s));
  int32_t n_scan = 0;
  for (const SubBatch &sb : C.subs) {
    g.q_base = sb.q_base;
    g.nq = sb.nq;
    g.mode = 0;
    LR_LAUNCH(launch_sign_scan(g, ix->num_sms, s));
    ++n_scan;
  }
  LR_LAUNCH(launch_sign_levels(ix->hist, kFbBins, ix->sign_bits, B, qk_d, ix->pass, ix->sign_cap, ix->sign_level,
                               ix->sign_ncand, s));
  for (const SubBatch &sb : C.subs) {
    g.q_base = sb.q_base;
    g.nq = sb.nq;
    g.mode = 1;
    LR_LAUNCH(launch_sign_scan(g, ix->num_sms, s));
    ++n_scan;
  }
  if (stats && stats->scan_stop) LR_CK(cudaEventRecord((cudaEvent_t)stats->scan_stop, s));
  // EBR: exact FP32 scores of the kept jobs, then the exact top K among them
  LR_LAUNCH(launch_sign_rescore(ix->X, ix->d_pad, ix->q_ws, ix->sign_buf, ix->sign_cap, ix->cnt, B, ix->num_sms, s));
  const bool dev_out = is_device_ptr(out_ids) && is_device_ptr(out_scores) &&
                       (out_count == nullptr || is_device_ptr(out_count));
  if (!dev_out && k_all > ix->max_k) return fail(LR_ERR_INVALID, "host outputs need k_all <= max_k");
  SelectArgs fa{};
  fa.mode = 1;
  fa.buf = ix->sign_buf;
  fa.cap = ix->sign_cap;
  fa.cnt = ix->cnt;
  fa.overflow = ix->ovf;
  fa.k = kfin_d;
  fa.pass_cnt = ix->sign_ncand;
  fa.k_stride = k_all;
  fa.out_ids = dev_out ? out_ids : ix->o_ids;
  fa.out_scores = dev_out ? out_scores : ix->o_sc;
  fa.out_count = dev_out ? out_count : ix->o_cnt;
  fa.flag = ix->flag;
  fa.n_flagged = ix->n_flag;
  fa.fb_prefix = ix->prefix;
  fa.fb_krem = ix->krem;
  fa.cand_count_out = ix->o_cand;
  fa.fallback_out = ix->o_fb;
  fa.err = ix->err;
  fa.id_base = ix->id_base;
  LR_LAUNCH(launch_select(fa, B, s));
  // the exact fallback of the plain search expects a clear histogram
  LR_CK(cudaMemsetAsync(ix->hist, 0, (size_t)B * kFbBins * sizeof(uint32_t), s));
  bool need_sync = false;
  if (!dev_out) {
    LR_CK(cudaMemcpyAsync(out_ids, ix->o_ids, sizeof(int32_t) * (size_t)B * k_all, cudaMemcpyDeviceToHost, s));
    LR_CK(cudaMemcpyAsync(out_scores, ix->o_sc, sizeof(float) * (size_t)B * k_all, cudaMemcpyDeviceToHost, s));
    if (out_count) LR_CK(cudaMemcpyAsync(out_count, ix->o_cnt, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, s));
    need_sync = host_out_sync((o.flags & LR_SEARCH_ASYNC_HOST) != 0, out_ids, out_scores, out_count);
  }
  if (stats) {
    if (stats->n_launches) *stats->n_launches = n_launch;
    if (stats->n_scan_launches) *stats->n_scan_launches = n_scan;
    if (stats->plan_used) *stats->plan_used = LR_PLAN_GEMV;
    struct { void *dst; const void *src; size_t bytes; } cp[3] = {
        {stats->pass_count, ix->pass, sizeof(int64_t) * B},
        {stats->cand_count, ix->o_cand, sizeof(int32_t) * B},
        {stats->fallback, ix->o_fb, sizeof(int32_t) * B}};
    for (auto &c : cp) {
      if (!c.dst) continue;
      LR_CK(cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyDefault, s));
      need_sync |= !is_device_ptr(c.dst);
    }
  }
  if (need_sync) LR_CK(cudaStreamSynchronize(s));
  return LR_OK;
}

// TBR-first search (Sec. 5.3, "EBR first or TBR first"): the postings of each
// query's chosen clause are the candidates; rows passing the whole CNF form the
// query's messenger list; only those rows are scored (FP32) and selected.
lr_status run_tbr_search(lr_index *ix, const float *q, int B, const lr_filters *f, const int32_t *k, int k_all,
                         int32_t *out_ids, float *out_scores, int32_t *out_count, const lr_search_stats *stats,
                         cudaStream_t s, const TbrPlan &T, int64_t cap, bool async_host) {
  const int turn = ix->filt_turn;
  ix->filt_turn ^= 1;
  if (ix->filt_ev_live[turn]) LR_CK(cudaEventSynchronize(ix->filt_ev[turn]));
  char *stage = ix->filt_h[turn];
  Compiled C;
  lr_status st = compile_filters(ix, f, B, kTcMaxQ, stage, C);
  if (st != LR_OK) return st;
  int32_t *kf = (int32_t *)(stage + C.off_kfin);
  for (int b = 0; b < B; ++b) {
    const int kb = k ? k[b] : k_all;
    if (kb < 1 || kb > ix->max_k || kb > k_all) return fail(LR_ERR_INVALID, "K must be in [1, min(max_k, k_all)]");
    kf[b] = kb;
  }
  // posting ranges of every query's chosen clause, with each term's bitmap
  const size_t off_roff = align_up(C.bytes, 16);
  const size_t off_rng = align_up(off_roff + sizeof(int32_t) * (B + 1), 16);
  int32_t *roff = (int32_t *)(stage + off_roff);
  TbrRange *rng = (TbrRange *)(stage + off_rng);
  const size_t bm_words = (size_t)ix->n_words;
  int R = 0;
  roff[0] = 0;
  for (int b = 0; b < B; ++b) {
    const int c = T.clause[b];
    for (int i = f->c_off[c]; i < f->c_off[c + 1]; ++i) {
      const int32_t t = (int32_t)f->terms[i];
      bool seen = false;
      for (int i2 = f->c_off[c]; i2 < i; ++i2) seen |= (int32_t)f->terms[i2] == t;
      if (seen) continue;
      if (off_rng + sizeof(TbrRange) * (R + 1) > ix->filt_bytes)
        return fail(LR_ERR_WORKSPACE, "filters: staging area too small");
      TbrRange r;
      r.begin = ix->post_off_h[t];
      r.end = ix->post_off_h[t + 1];
      r.bm = ix->term_dense[t] >= 0 ? ix->dense_bm + (size_t)ix->term_dense[t] * bm_words
                                    : ix->sparse_bm + (size_t)ix->sparse_id[t] * bm_words;
      std::memcpy(rng + R, &r, sizeof(TbrRange));
      ++R;
    }
    roff[b + 1] = R;
  }
  const size_t bytes = off_rng + sizeof(TbrRange) * std::max(R, 1);
  int32_t n_launch = 0;
  LR_CK(cudaMemcpyAsync(ix->filt_d, stage, bytes, cudaMemcpyHostToDevice, s));
  LR_CK(cudaEventRecord(ix->filt_ev[turn], s));
  ix->filt_ev_live[turn] = true;
  LR_CK(cudaMemsetAsync(ix->state, 0, ix->state_bytes, s));
  const int32_t *kfin_d = (const int32_t *)(ix->filt_d + C.off_kfin);
  const float *qsrc = q;
  if (!is_device_ptr(q)) {
    LR_CK(cudaMemcpyAsync(ix->q_raw, q, sizeof(float) * (size_t)B * ix->dim, cudaMemcpyHostToDevice, s));
    qsrc = ix->q_raw;
  }
  LR_LAUNCH(launch_prep_queries(qsrc, ix->q_ws, B, ix->dim, ix->d_pad, ix->metric == LR_COSINE, ix->err, s));
  if (!C.sparse_terms.empty()) {
    ++n_launch;
    LR_CK(expand_sparse_terms(ix, C, s));
  }
  if (stats && stats->scan_start) LR_CK(cudaEventRecord((cudaEvent_t)stats->scan_start, s));
  int32_t n_scan = 0;
  for (const SubBatch &sb : C.subs) {
    TbrArgs a{};
    a.n = ix->n;
    a.q_base = sb.q_base;
    a.nq = sb.nq;
    a.slot_bm = (const uint32_t *const *)(ix->filt_d + sb.off_slots);
    a.qc_off = (const int32_t *)(ix->filt_d + sb.off_qc);
    a.cl_off = (const int32_t *)(ix->filt_d + sb.off_cl);
    a.cl_slot = (const int32_t *)(ix->filt_d + sb.off_cs);
    a.r_off = (const int32_t *)(ix->filt_d + off_roff);
    a.ranges = (const TbrRange *)(ix->filt_d + off_rng);
    a.post_ids = ix->post_ids_d;
    a.buf = ix->cand_buf;
    a.cap = cap;
    a.cnt = ix->cnt;
    a.pass_cnt = ix->pass;
    a.err = ix->err;
    LR_LAUNCH(launch_tbr_collect(a, ix->num_sms, T.max_postings, s));
    ++n_scan;
  }
  LR_LAUNCH(launch_sign_rescore(ix->X, ix->d_pad, ix->q_ws, ix->cand_buf, cap, ix->cnt, B, ix->num_sms, s));
  ++n_scan;
  if (stats && stats->scan_stop) LR_CK(cudaEventRecord((cudaEvent_t)stats->scan_stop, s));
  const bool dev_out = is_device_ptr(out_ids) && is_device_ptr(out_scores) &&
                       (out_count == nullptr || is_device_ptr(out_count));
  if (!dev_out && k_all > ix->max_k) return fail(LR_ERR_INVALID, "host outputs need k_all <= max_k");
  SelectArgs fa{};
  fa.mode = 1;
  fa.buf = ix->cand_buf;
  fa.cap = cap;
  fa.cnt = ix->cnt;
  fa.overflow = ix->ovf;
  fa.k = kfin_d;
  fa.pass_cnt = ix->pass;
  fa.k_stride = k_all;
  fa.out_ids = dev_out ? out_ids : ix->o_ids;
  fa.out_scores = dev_out ? out_scores : ix->o_sc;
  fa.out_count = dev_out ? out_count : ix->o_cnt;
  fa.flag = ix->flag;
  fa.n_flagged = ix->n_flag;
  fa.fb_prefix = ix->prefix;
  fa.fb_krem = ix->krem;
  fa.cand_count_out = ix->o_cand;
  fa.fallback_out = ix->o_fb;
  fa.err = ix->err;
  fa.id_base = ix->id_base;
  LR_LAUNCH(launch_select(fa, B, s));
  bool need_sync = false;
  if (!dev_out) {
    LR_CK(cudaMemcpyAsync(out_ids, ix->o_ids, sizeof(int32_t) * (size_t)B * k_all, cudaMemcpyDeviceToHost, s));
    LR_CK(cudaMemcpyAsync(out_scores, ix->o_sc, sizeof(float) * (size_t)B * k_all, cudaMemcpyDeviceToHost, s));
    if (out_count) LR_CK(cudaMemcpyAsync(out_count, ix->o_cnt, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, s));
    need_sync = host_out_sync(async_host, out_ids, out_scores, out_count);
  }
  if (stats) {
    if (stats->n_launches) *stats->n_launches = n_launch;
    if (stats->n_scan_launches) *stats->n_scan_launches = n_scan;
    if (stats->plan_used) *stats->plan_used = LR_PLAN_TBR;
    struct { void *dst; const void *src; size_t bytes; } cp[3] = {
        {stats->pass_count, ix->pass, sizeof(int64_t) * B},
        {stats->cand_count, ix->o_cand, sizeof(int32_t) * B},
        {stats->fallback, ix->o_fb, sizeof(int32_t) * B}};
    for (auto &c : cp) {
      if (!c.dst) continue;
      LR_CK(cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyDefault, s));
      need_sync |= !is_device_ptr(c.dst);
    }
  }
  if (need_sync) LR_CK(cudaStreamSynchronize(s));
  return LR_OK;
}

lr_status run_search(lr_index *ix, const float *q, int B, const lr_filters *f, const int32_t *k, int k_all,
                     int32_t *out_ids, float *out_scores, int32_t *out_count, const lr_search_opts *opts,
                     const lr_search_stats *stats, cudaStream_t s, StageTimer &tm) {
  if (B < 1) return fail(LR_ERR_INVALID, "B must be >= 1");
  if (B > ix->max_batch) return fail(LR_ERR_WORKSPACE, "B exceeds max_batch");
  if (!q || !out_ids || !out_scores) return fail(LR_ERR_INVALID, "null query or output pointer");
  if (k_all < 1) return fail(LR_ERR_INVALID, "k_all must be >= 1");
  if (k_all > ix->max_k && k == nullptr) return fail(LR_ERR_INVALID, "K exceeds max_k");
  lr_search_opts o{};
  if (opts) o = *opts;
  // row range: groups [g0, g1) of the index
  const bool ranged = o.row_begin != 0 || o.row_end != 0;
  int64_t g0 = 0, g1 = ix->n_groups, range_rows = ix->n;
  if (ranged) {
    if (o.row_begin < 0 || o.row_end > ix->n || o.row_begin >= o.row_end || o.row_begin % kGroupRows != 0 ||
        (o.row_end % kGroupRows != 0 && o.row_end != ix->n))
      return fail(LR_ERR_INVALID, "row range: need 0 <= row_begin < row_end <= n, row_begin a multiple of 256 and "
                                  "row_end a multiple of 256 or n");
    if (o.quant_mult != 0 || o.plan == LR_PLAN_TBR)
      return fail(LR_ERR_UNSUPPORTED, "row range: not with sign pre-selection or the TBR-first plan");
    g0 = o.row_begin / kGroupRows;
    g1 = (o.row_end + kGroupRows - 1) / kGroupRows;
    range_rows = o.row_end - o.row_begin;
  }
  const int64_t range_groups = g1 - g0;
  if (o.quant_mult != 0) {
    tm.mark("sign");
    return run_sign_search(ix, q, B, f, k, k_all, out_ids, out_scores, out_count, o, stats, s);
  }

  // pick and wait for a staging buffer
  const int turn = ix->filt_turn;
  ix->filt_turn ^= 1;
  if (ix->filt_ev_live[turn]) LR_CK(cudaEventSynchronize(ix->filt_ev[turn]));
  char *stage = ix->filt_h[turn];
  Compiled C;
  // scoring plan: SIMT matrix-vector scan for small batches, tensor-core tiles
  // (3xTF32) once a launch serves enough queries to be a real contraction
  int plan = o.plan;
  if (plan != LR_PLAN_AUTO && plan != LR_PLAN_GEMV && plan != LR_PLAN_TC && plan != LR_PLAN_TBR)
    return fail(LR_ERR_INVALID, "plan must be LR_PLAN_AUTO, LR_PLAN_GEMV, LR_PLAN_TC or LR_PLAN_TBR");
  // LR_PLAN in the environment decides for the caller that left it to us
  // (not TBR first for a row range, which that plan does not serve)
  if (plan == LR_PLAN_AUTO && debug_env().plan > 0 && !(ranged && debug_env().plan == LR_PLAN_TBR))
    plan = debug_env().plan;
  const bool lowp = ix->elem != kElemF32;
  const bool tc_ok = lowp ? ix->have_tmap_q : ix->have_tmap;
  std::vector<double> est;  // estimated pass rate per filter
  const bool have_est = estimate_pass_rates(ix, f, B, est);
  // the automatic plan considers TBR first only when no scan option is forced
  const bool scan_opts = o.sample_stride != 0 || o.cand_cap != 0 || o.force_exact_fallback != 0;
  if (plan == LR_PLAN_TBR || (plan == LR_PLAN_AUTO && have_est && !scan_opts && !ranged)) {
    // the candidate buffer holds max_batch x cand_cap keys: a batch of B
    // queries gives each query an equal share of it for its messenger list
    int64_t tcap = ix->cand_cap * (int64_t)ix->max_batch / B;
    if (o.cand_cap > 0) tcap = std::min<int64_t>(tcap, o.cand_cap);
    const TbrPlan T = plan_tbr(ix, f, B, tcap);
    if (plan == LR_PLAN_TBR && !T.ok)
      return fail(LR_ERR_UNSUPPORTED, "TBR-first plan needs posting lists, a clause per query and a chosen clause "
                                      "with at most the candidate capacity of postings and 16 distinct terms");
    if (plan == LR_PLAN_TBR || (T.ok && tbr_cheaper(ix, B, T, est, tc_ok))) {
      tm.mark("tbr");
      return run_tbr_search(ix, q, B, f, k, k_all, out_ids, out_scores, out_count, stats, s, T, tcap,
                            (o.flags & LR_SEARCH_ASYNC_HOST) != 0);
    }
  }
  if (plan == LR_PLAN_AUTO) plan = choose_plan(ix, B, tc_ok, have_est, est);
  if (plan == LR_PLAN_TC && !tc_ok)
    return fail(LR_ERR_UNSUPPORTED, "tensor-core plan unavailable for this index (no TMA descriptor; "
                                    "low-precision rows need dim > 32)");
  // Above 64 queries consecutive sub-batches share several-block scans: FP32
  // rows two blocks, of 64 up to 128 queries and of 48 above (two
  // accumulators: fewer launches than blocks of 64 from there on); BF16 and
  // e4m3 rows up to four blocks of 64
  const bool pairs = plan == LR_PLAN_TC && ix->tile_msg2 != nullptr && B > kTcMaxQ;
  const int block_q = ix->elem == kElemF32 && B > kTc2MinBatch ? kTc2BlockQ : kTcMaxQ;
  const int group_max = ix->elem == kElemF32 ? 2 : kBf16Blocks;
  const int max_q = plan == LR_PLAN_TC ? (pairs ? block_q : ix->d_pad <= 128 ? kTcMaxQ : kTcMaxQ / 2) : kGemvMaxQ;
  lr_status st = compile_filters(ix, f, B, max_q, stage, C);
  if (st != LR_OK) return st;
  // ks: the K the scan and the selection work with (oversample x K for the
  // precision form); kf: the K the caller asked for
  int32_t *ks = (int32_t *)(stage + C.off_k);
  int32_t *kf = (int32_t *)(stage + C.off_kfin);
  for (int b = 0; b < B; ++b) {
    const int kb = k ? k[b] : k_all;
    if (kb < 1 || kb > ix->max_k || kb > k_all)
      return fail(LR_ERR_INVALID, "K must be in [1, min(max_k, k_all)]");
    kf[b] = kb;
    ks[b] = lowp ? std::min(kb * ix->oversample, ix->max_kq) : kb;
  }
  // threshold sample plan
  int stride = ix->auto_stride;
  if (o.sample_stride > 0) stride = o.sample_stride;
  if (o.sample_stride < 0) stride = 0;
  const SamplePlan sp = make_sample_plan(ix, stride, g0, g1);
  if (sp.stride > 0 && sp.sampled_rows > ix->samp_cap)
    return fail(LR_ERR_WORKSPACE, "sample stride too small for the sample workspace");
  int32_t *rk = (int32_t *)(stage + C.off_rank);
  // A filter expected to pass fewer than a quarter of what the final
  // selection holds in shared memory (and of the candidate buffer) collects
  // every passing key (rank 0: threshold 0) and needs no sample; when no filter
  // needs one the sample is skipped.  A wrong estimate overflows the buffer
  // and the exact fallback still gives the exact top K.  (Only with the
  // automatic stride: an explicit one always runs the sample.)
  int64_t cap = ix->cand_cap;
  if (o.cand_cap > 0) cap = std::min<int64_t>(cap, std::max<int64_t>(o.cand_cap, 1));
  const double direct = (double)std::min<int64_t>(cap, kThrScratchKeys);
  bool need_sample = false;
  for (int b = 0; b < B; ++b) {
    const bool small = o.sample_stride == 0 && have_est && est[b] * (double)range_rows * 4.0 < direct;
    rk[b] = small ? 0 : sample_rank(sp, ks[b]);
    need_sample |= rk[b] > 0;
  }

  // ---- device work
  tm.mark("upload+prep");
  int32_t n_launch = 0, n_scan = 0;
  LR_CK(cudaMemcpyAsync(ix->filt_d, stage, C.bytes, cudaMemcpyHostToDevice, s));
  LR_CK(cudaEventRecord(ix->filt_ev[turn], s));
  ix->filt_ev_live[turn] = true;
  LR_CK(cudaMemsetAsync(ix->state, 0, ix->state_bytes, s));
  // per-query K (scan and selection), final K and sample rank: read by the
  // kernels where they were uploaded
  const int32_t *kq_d = (const int32_t *)(ix->filt_d + C.off_k);
  const int32_t *kfin_d = (const int32_t *)(ix->filt_d + C.off_kfin);
  const int32_t *rank_d = (const int32_t *)(ix->filt_d + C.off_rank);
  const float *qsrc = q;
  if (!is_device_ptr(q)) {
    LR_CK(cudaMemcpyAsync(ix->q_raw, q, sizeof(float) * (size_t)B * ix->dim, cudaMemcpyHostToDevice, s));
    qsrc = ix->q_raw;
  }
  LR_LAUNCH(launch_prep_queries(qsrc, ix->q_ws, B, ix->dim, ix->d_pad, ix->metric == LR_COSINE, ix->err, s));
  if (!C.sparse_terms.empty()) {
    ++n_launch;
    LR_CK(expand_sparse_terms(ix, C, s));
  }

  auto scan_args = [&](const SubBatch &sb) {
    ScanArgs a{};
    a.X = ix->X;
    a.Xq = ix->Xq;
    a.xscale = ix->xscale;
    a.elem = ix->elem;
    a.n = ix->n;
    a.d_pad = ix->d_pad;
    a.Q = ix->q_ws;
    a.q_base = sb.q_base;
    a.nq = sb.nq;
    a.slot_bm = (const uint32_t *const *)(ix->filt_d + sb.off_slots);
    a.n_slots = sb.n_slots;
    a.qc_off = (const int32_t *)(ix->filt_d + sb.off_qc);
    a.cl_off = (const int32_t *)(ix->filt_d + sb.off_cl);
    a.cl_slot = (const int32_t *)(ix->filt_d + sb.off_cs);
    a.n_cl = sb.n_cl;
    a.n_tm = sb.n_tm;
    a.n_groups = g1;
    a.g_begin = g0;
    a.g_step = 1;
    a.mode = kCollect;
    a.err = ix->err;
    a.done_ctr = ix->done_ctr;
    a.work_ctr = ix->work_ctr;
    a.batch = B;
    a.tile_row = ix->tile_row;
    a.tile_msg = ix->tile_msg;
    a.tile_cnt = ix->tile_cnt;
    a.tile_cap = ix->tile_cap;
    return a;
  };
  const int vec = ix->d_pad / 32;
  auto nq_tmpl = [](int nq) { return nq <= 1 ? 1 : nq <= 2 ? 2 : nq <= 4 ? 4 : 8; };
  auto grid_for = [&](int64_t groups) {  // persistent: one CTA per SM, fewer for small scans
    const int64_t want = plan == LR_PLAN_TC ? groups : (groups + 3) / 4;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)ix->num_sms));
  };
  // Tensor-core plan: the tile filter (term predicate) writes the list of
  // tiles the scan reads.  With one sub-batch the main pass keeps its list and
  // the exact fallback's scans reuse it (masked to the flagged queries) instead
  // of filtering again.
  const bool reuse_list = plan == LR_PLAN_TC && C.subs.size() == 1;
  auto launch_scan = [&](ScanArgs a, int64_t groups, bool filter = true, bool keep = false) {
    if (plan != LR_PLAN_TC) return launch_scan_gemv(a, nq_tmpl(a.nq), vec, grid_for(groups), s);
    a.keep_list = keep ? 1 : 0;
    if (filter) {
      ++n_launch;
      const cudaError_t e = launch_tile_filter(a, ix->num_sms, s);
      if (e != cudaSuccess) return e;
    }
    return launch_scan_tc(a, lowp ? &ix->tmap_xq : &ix->tmap_x, grid_for(2 * groups), s);
  };

  auto main_args = [&](const SubBatch &sb) {
    ScanArgs a = scan_args(sb);
    a.tau = ix->tau;
    a.buf = ix->cand_buf;
    a.buf_cap = cap;
    a.buf_cnt = ix->cnt;
    a.overflow = ix->ovf;
    a.pass_cnt = ix->pass;
    return a;
  };
  // With one sub-batch the main pass's tile filter does not depend on the
  // threshold: it runs on the second stream while the threshold sample runs
  // here, and the main scan waits for it.
  const bool early_filter = reuse_list;
  if (early_filter) {
    LR_CK(cudaEventRecord(ix->ev_fork, s));
    LR_CK(cudaStreamWaitEvent(ix->aux, ix->ev_fork, 0));
    ++n_launch;
    LR_CK(launch_tile_filter(main_args(C.subs[0]), ix->num_sms, ix->aux));
    LR_CK(cudaEventRecord(ix->ev_join, ix->aux));
  }
  // 1. threshold sample
  tm.mark("sample");
  if (sp.stride > 0 && need_sample) {
    for (const SubBatch &sb : C.subs) {
      ScanArgs a = scan_args(sb);
      a.g_begin = g0 + sp.stride / 2;
      a.g_step = sp.stride;
      a.tile_row = ix->tile_row_s;  // the sample's own tile list
      a.tile_msg = ix->tile_msg_s;
      a.tile_cnt = ix->tile_cnt_s;
      a.tile_cap = ix->tile_cap_s;
      a.tau = nullptr;  // keep every passing key of the sampled groups
      a.buf = ix->samp_buf;
      a.buf_cap = ix->samp_cap;
      a.buf_cnt = ix->scnt;
      a.overflow = ix->sovf;
      LR_LAUNCH(launch_scan(a, sp.sampled_groups));
    }
    ThrArgs t{};
    t.buf = ix->samp_buf;
    t.cap = ix->samp_cap;
    t.cnt = ix->scnt;
    t.overflow = ix->sovf;
    t.rank = rank_d;
    t.tau = ix->tau;
    t.scratch = ix->thr_scratch;
    t.slice_n = ix->thr_slice_n;
    t.done = ix->thr_done;
    LR_LAUNCH(launch_threshold(t, B, s));
  }
  // 2. main scan: candidates at or above the threshold, pass counts
  tm.mark("scan");
  if (early_filter) LR_CK(cudaStreamWaitEvent(s, ix->ev_join, 0));
  if (stats && stats->scan_start) LR_CK(cudaEventRecord((cudaEvent_t)stats->scan_start, s));
  // Consecutive sub-batches (full ones of block_q queries, then one more)
  // share one scan that reads (and for FP32 converts) each tile once and
  // scores it against every block; their tile filters write every tile's
  // masks (no list), block b's into tile_msg2 + (b - 1) msg_block_stride
  const int64_t msg_stride = ix->tile_cap * 128;
  for (size_t i = 0; i < C.subs.size(); ++i) {
    const SubBatch &sb = C.subs[i];
    size_t g = 1;  // sub-batches in this launch
    while (pairs && !early_filter && g < (size_t)group_max && i + g < C.subs.size() &&
           C.subs[i + g - 1].nq == block_q && C.subs[i + g].q_base == C.subs[i + g - 1].q_base + block_q)
      ++g;
    if (g > 1) {
      ScanArgs a0 = main_args(sb);
      int nq = 0;
      for (size_t b = 0; b < g; ++b) {
        ScanArgs ab = main_args(C.subs[i + b]);
        ab.dense_tiles = 1;
        if (b > 0) ab.tile_msg = ix->tile_msg2 + (size_t)(b - 1) * (size_t)msg_stride;
        LR_LAUNCH(launch_tile_filter(ab, ix->num_sms, s));
        nq += C.subs[i + b].nq;
      }
      a0.dense_tiles = 1;
      a0.nq = nq;
      a0.tile_msg2 = ix->tile_msg2;
      a0.msg_block_stride = msg_stride;
      a0.block_q = block_q;
      LR_LAUNCH(launch_scan_tc2(a0, lowp ? &ix->tmap_xq : &ix->tmap_x, grid_for(2 * range_groups), s));
      ++n_scan;
      i += g - 1;
      continue;
    }
    LR_LAUNCH(launch_scan(main_args(sb), range_groups, !early_filter, reuse_list));
    ++n_scan;
  }
  if (stats && stats->scan_stop) LR_CK(cudaEventRecord((cudaEvent_t)stats->scan_stop, s));
  tm.mark("select");
  // 3. final selection into the caller's device outputs, or into workspace
  //    rows that are copied back when the outputs are host memory
  const bool dev_out = is_device_ptr(out_ids) && is_device_ptr(out_scores) &&
                       (out_count == nullptr || is_device_ptr(out_count));
  if (!dev_out && k_all > ix->max_k) return fail(LR_ERR_INVALID, "host outputs need k_all <= max_k");
  SelectArgs fa{};
  fa.mode = 1;
  fa.buf = ix->cand_buf;
  fa.cap = cap;
  fa.cnt = ix->cnt;
  fa.overflow = ix->ovf;
  fa.k = kq_d;
  fa.pass_cnt = ix->pass;
  fa.k_stride = lowp ? ix->max_kq : k_all;
  fa.out_ids = lowp ? ix->c_ids : dev_out ? out_ids : ix->o_ids;
  fa.out_scores = lowp ? ix->c_sc : dev_out ? out_scores : ix->o_sc;
  fa.out_count = lowp ? ix->c_cnt : dev_out ? out_count : ix->o_cnt;
  fa.flag = ix->flag;
  fa.n_flagged = ix->n_flag;
  fa.fb_prefix = ix->prefix;
  fa.fb_krem = ix->krem;
  fa.cand_count_out = ix->o_cand;
  fa.fallback_out = ix->o_fb;
  fa.fallback_round = 0;
  fa.force_flag = o.force_exact_fallback ? 1 : 0;
  fa.unsorted = lowp ? 1 : 0;  // the precision form re-ranks the candidates in FP32
  fa.err = ix->err;
  fa.id_base = lowp ? 0 : ix->id_base;  // the precision form's rescore reads rows by local id
  LR_LAUNCH(launch_select(fa, B, s));
  tm.mark("fallback");
  // 4. exact fallback for flagged queries (each launch returns at once when none
  //    is flagged): kFbPasses histogram passes, then the collect, per
  //    sub-batch; the sub-batch's first pass filters its tiles and the list
  //    serves the other passes (the collect's scan clears it for the next
  //    sub-batch; with one sub-batch the main pass's list serves all of them)
  for (const SubBatch &sb : C.subs) {
    for (int p = 0; p <= kFbPasses; ++p) {
      ScanArgs a = scan_args(sb);
      a.active = ix->flag;
      a.any_active = ix->n_flag;
      if (p < kFbPasses) {
        a.mode = kHist;
        a.hist_pass = p;
        a.prefix = ix->prefix;
        a.krem = ix->krem;
        a.hist = ix->hist;
        a.tau_out = ix->tau;
      } else {
        a.tau = ix->tau;
        a.buf = ix->cand_buf;
        a.buf_cap = ix->cand_cap;
        a.buf_cnt = ix->cnt;
        a.overflow = ix->ovf;
      }
      const bool filter = !reuse_list && p == 0;
      const bool keep = reuse_list || p < kFbPasses;
      LR_LAUNCH(launch_scan(a, range_groups, filter, keep));
    }
  }
  SelectArgs fb = fa;
  fb.cap = ix->cand_cap;
  fb.only = ix->flag;
  fb.any = ix->n_flag;
  fb.fallback_round = 1;
  fb.force_flag = 0;
  LR_LAUNCH(launch_select(fb, B, s));
  // 5. precision form: FP32 rescore of the candidates, FP64 re-rank of the near ties
  if (lowp) {
    tm.mark("rescore");
    RescoreArgs ra{};
    ra.X = ix->X;
    ra.d_pad = ix->d_pad;
    ra.dim = ix->dim;
    ra.Q = ix->q_ws;
    ra.cid = ix->c_ids;
    ra.ccnt = ix->c_cnt;
    ra.c_stride = ix->max_kq;
    ra.k = kfin_d;
    ra.k_stride = k_all;
    ra.out_ids = dev_out ? out_ids : ix->o_ids;
    ra.out_scores = dev_out ? out_scores : ix->o_sc;
    ra.out_count = dev_out ? out_count : ix->o_cnt;
    ra.tie_count = ix->o_ties;
    ra.err = ix->err;
    ra.keys = ix->rs_keys;
    ra.gmax = ix->rs_gmax;
    ra.id_base = ix->id_base;
    LR_LAUNCH(launch_rescore(ra, B, s));
  }

  // 6. host outputs and statistics
  tm.mark("outputs");
  bool need_sync = false;
  if (!dev_out) {
    LR_CK(cudaMemcpyAsync(out_ids, ix->o_ids, sizeof(int32_t) * (size_t)B * k_all, cudaMemcpyDeviceToHost, s));
    LR_CK(cudaMemcpyAsync(out_scores, ix->o_sc, sizeof(float) * (size_t)B * k_all, cudaMemcpyDeviceToHost, s));
    if (out_count) LR_CK(cudaMemcpyAsync(out_count, ix->o_cnt, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, s));
    need_sync = host_out_sync((o.flags & LR_SEARCH_ASYNC_HOST) != 0, out_ids, out_scores, out_count);
  }
  if (stats) {
    if (stats->n_launches) *stats->n_launches = n_launch;
    if (stats->n_scan_launches) *stats->n_scan_launches = n_scan;
    if (stats->plan_used) *stats->plan_used = plan;
    struct { void *dst; const void *src; size_t bytes; } cp[4] = {
        {stats->pass_count, ix->pass, sizeof(int64_t) * B},
        {stats->cand_count, ix->o_cand, sizeof(int32_t) * B},
        {stats->fallback, ix->o_fb, sizeof(int32_t) * B},
        {lowp ? stats->rescore_ties : nullptr, ix->o_ties, sizeof(int32_t) * B}};
    for (auto &c : cp) {
      if (!c.dst) continue;
      LR_CK(cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyDefault, s));
      need_sync |= !is_device_ptr(c.dst);
    }
  }
  if (need_sync) LR_CK(cudaStreamSynchronize(s));
  return LR_OK;
}

}  // namespace

extern "C" {

lr_status lr_search_ex(lr_index *index, const float *q, int32_t B, const lr_filters *f, const int32_t *k,
                       int32_t k_all, int32_t *out_ids, float *out_scores, int32_t *out_count,
                       const lr_search_opts *opts, const lr_search_stats *stats, void *stream) {
  if (!index) return fail(LR_ERR_INVALID, "index is null");
  StageTimer tm((cudaStream_t)stream, "lr_search");
  const lr_status st =
      run_search(index, q, B, f, k, k_all, out_ids, out_scores, out_count, opts, stats, (cudaStream_t)stream, tm);
  if (st == LR_OK) tm.report("B=" + std::to_string(B) + " K=" + std::to_string(k_all) + " ms");
  return st;
}

lr_status lr_search(lr_index *index, const float *q, int32_t B, const lr_filters *f, const int32_t *k,
                    int32_t k_all, int32_t *out_ids, float *out_scores, int32_t *out_count, void *stream) {
  return lr_search_ex(index, q, B, f, k, k_all, out_ids, out_scores, out_count, nullptr, nullptr, stream);
}

lr_status lr_filter_count(lr_index *index, const lr_filters *f, int32_t B, int64_t *out_pass, uint32_t *out_bitmap,
                          void *stream) {
  if (!index) return fail(LR_ERR_INVALID, "index is null");
  if (!out_pass) return fail(LR_ERR_INVALID, "out_pass is null");
  if (B < 1) return fail(LR_ERR_INVALID, "B must be >= 1");
  if (B > index->max_batch) return fail(LR_ERR_WORKSPACE, "B exceeds max_batch");
  lr_index *ix = index;
  cudaStream_t s = (cudaStream_t)stream;
  const int turn = ix->filt_turn;
  ix->filt_turn ^= 1;
  if (ix->filt_ev_live[turn]) LR_CK(cudaEventSynchronize(ix->filt_ev[turn]));
  char *stage = ix->filt_h[turn];
  Compiled C;
  lr_status st = compile_filters(ix, f, B, 32, stage, C);
  if (st != LR_OK) return st;
  LR_CK(cudaMemcpyAsync(ix->filt_d, stage, C.bytes, cudaMemcpyHostToDevice, s));
  LR_CK(cudaEventRecord(ix->filt_ev[turn], s));
  ix->filt_ev_live[turn] = true;
  LR_CK(cudaMemsetAsync(ix->state, 0, ix->state_bytes, s));
  if (!C.sparse_terms.empty()) LR_CK(expand_sparse_terms(ix, C, s));
  const int64_t out_words = (ix->n + 31) / 32;
  const bool bm_dev = out_bitmap && is_device_ptr(out_bitmap);
  // A host bitmap is staged, one sub-batch of at most 32 rows at a time, in the
  // index's tile-mask region (2 n_groups x 128 x 8 bytes >= 32 rows of n/8
  // bytes), so the call allocates nothing (appendix "Memory Pre-Allocation").
  uint32_t *stage_bm = reinterpret_cast<uint32_t *>(ix->tile_msg);
  for (const SubBatch &sb : C.subs) {
    ScanArgs a{};
    a.n = ix->n;
    a.q_base = sb.q_base;
    a.nq = sb.nq;
    a.slot_bm = (const uint32_t *const *)(ix->filt_d + sb.off_slots);
    a.n_slots = sb.n_slots;
    a.qc_off = (const int32_t *)(ix->filt_d + sb.off_qc);
    a.cl_off = (const int32_t *)(ix->filt_d + sb.off_cl);
    a.cl_slot = (const int32_t *)(ix->filt_d + sb.off_cs);
    a.n_groups = ix->n_groups;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((ix->n_groups + 7) / 8, (int64_t)ix->num_sms * 4));
    if (!out_bitmap || bm_dev) {
      LR_CK(launch_filter_eval(a, ix->pass, out_bitmap, out_words, 0, grid, s));
      continue;
    }
    if ((size_t)sb.nq * (size_t)out_words * 4 > (size_t)ix->tile_cap * 128 * sizeof(uint64_t))
      return fail(LR_ERR_WORKSPACE, "lr_filter_count: bitmap staging area too small");
    LR_CK(launch_filter_eval(a, ix->pass, stage_bm, out_words, sb.q_base, grid, s));
    LR_CK(cudaMemcpyAsync(out_bitmap + (size_t)sb.q_base * out_words, stage_bm,
                          sizeof(uint32_t) * (size_t)sb.nq * out_words, cudaMemcpyDeviceToHost, s));
    LR_CK(cudaStreamSynchronize(s));  // the next sub-batch reuses the staging rows
  }
  LR_CK(cudaMemcpyAsync(out_pass, ix->pass, sizeof(int64_t) * B, cudaMemcpyDefault, s));
  if (!is_device_ptr(out_pass) || (out_bitmap && !bm_dev)) LR_CK(cudaStreamSynchronize(s));
  return LR_OK;
}

lr_status lr_index_sync(lr_index *index, void *stream) {
  if (!index) return fail(LR_ERR_INVALID, "index is null");
  return check_err_word(index, (cudaStream_t)stream, "lr_index_sync");
}

}  // extern "C"

// ------------------------------------------------------------------ loss
namespace {

// Geometry and workspace of the loss passes for B queries, M jobs, dimension d.
struct LossPlan {
  int Bp = 0, Mp = 0, dp = 0, n_ctiles = 0, c_per_split = 0, splits = 0;
  int nj_ctiles = 0, cj_per_split = 0, splits_j = 0;  // the dJ pass: job tiles against query tiles
  size_t o_qp = 0, o_qt = 0, o_jp = 0, o_jt = 0, o_pm = 0, o_ps = 0, o_zp = 0, o_dq = 0, o_dj = 0, o_st = 0,
         o_bs = 0, total = 0;
};

// Split of the streamed range over CTAs: the count (at most 16) that minimises
// (waves of CTAs over the SMs) x (streamed tiles per CTA + a CTA's fixed cost,
// about two tiles: tensor-memory allocation and the resident tile's load).
// A CTA's range is a whole number of tile pairs where it can be (the score
// MMAs take the streamed tiles two at a time).
void choose_split(int rtiles, int ctiles, int sms, int &splits, int &per) {
  long best = -1;
  splits = 1;
  per = ctiles;
  for (int s = 1; s <= std::min(ctiles, 16); ++s) {
    const int p = ctiles >= 2 ? (ctiles + 2 * s - 1) / (2 * s) * 2 : ctiles;
    const int se = (ctiles + p - 1) / p;
    const long cost = (long)((rtiles * se + sms - 1) / sms) * (p + 2);
    if (best < 0 || cost < best) {
      best = cost;
      splits = se;
      per = p;
    }
  }
}

LossPlan loss_plan(int B, int M, int d, int sms) {
  LossPlan P;
  P.Bp = (B + 127) / 128 * 128;
  P.Mp = (M + 127) / 128 * 128;
  P.dp = d <= 64 ? 64 : 128;
  P.n_ctiles = P.Mp / 64;
  choose_split(P.Bp / 128, P.n_ctiles, sms, P.splits, P.c_per_split);
  P.nj_ctiles = P.Bp / 64;
  choose_split(P.Mp / 128, P.nj_ctiles, sms, P.splits_j, P.cj_per_split);
  Carver cv;
  P.o_qp = cv.take<uint16_t>((size_t)P.Bp * P.dp);
  P.o_qt = cv.take<uint16_t>((size_t)P.Bp * P.dp);
  P.o_jp = cv.take<uint16_t>((size_t)P.Mp * P.dp);
  P.o_jt = cv.take<uint16_t>((size_t)P.Mp * P.dp);
  P.o_pm = cv.take<float>((size_t)4 * P.splits * P.Bp);  // one partial per split and epilogue set
  P.o_ps = cv.take<float>((size_t)4 * P.splits * P.Bp);
  P.o_zp = cv.take<float>(P.Bp);
  P.o_dq = cv.take<float>((size_t)P.splits * P.Bp * P.dp);
  P.o_dj = cv.take<float>((size_t)P.splits_j * P.Mp * P.dp);
  P.o_st = cv.take<uint32_t>(4);  // status word, finished-block counter of the loss sum
  P.o_bs = cv.take<double>((size_t)loss_combine_blocks(P.Bp));
  P.total = align_up(cv.off, 256);
  return P;
}

int current_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
    cudaGetLastError();
    return 148;
  }
  return sms;
}

lr_status loss_check(const void *Q, const void *J, int B, int M, int d, int dtype, const int32_t *pos,
                     const uint32_t *mask, void *ws, size_t ws_bytes, const LossPlan &P) {
  if (B < 1 || M < 1) return fail(LR_ERR_INVALID, "B and M must be >= 1");
  if (d < 1 || d > 128) return fail(LR_ERR_UNSUPPORTED, "the loss kernels take d in [1, 128]");
  if (dtype != LR_BF16 && dtype != LR_F32) return fail(LR_ERR_INVALID, "dtype must be LR_BF16 or LR_F32");
  if (!is_device_ptr(Q) || !is_device_ptr(J) || !is_device_ptr(pos) || !is_device_ptr(ws) ||
      (mask && !is_device_ptr(mask)))
    return fail(LR_ERR_INVALID, "Q, J, pos, mask and workspace must be device memory");
  if (ws_bytes < P.total) return fail(LR_ERR_WORKSPACE, "workspace smaller than lr_score_workspace_size()");
  return LR_OK;
}

struct LossMaps {
  CUtensorMap qr, qc, qt, jr, jc, jt;
};

// Operand copies and TMA descriptors of the loss passes.  BF16 inputs whose
// rows are whole 16-byte words (d % 8 == 0, 16-byte aligned) are read in place
// (the descriptors' zero fill pads rows past B or M and columns past d);
// otherwise a BF16 copy padded to [rows_p][dp] is written.  The backward
// passes also read the transposed copies [dp][rows_p] (need_t).
lr_status loss_prepare(const void *Q, const void *J, int B, int M, int d, int dtype, char *w, const LossPlan &P,
                       LossMaps &T, bool need_t, cudaStream_t s) {
  const int elem = dtype == LR_BF16 ? kElemBF16 : kElemF32;
  const bool direct = dtype == LR_BF16 && d % 8 == 0 && ((uintptr_t)Q & 15u) == 0 && ((uintptr_t)J & 15u) == 0;
  LR_CK(cudaMemsetAsync(w + P.o_st, 0, 2 * sizeof(uint32_t), s));
  if (!direct || need_t) {
    LR_CK(launch_loss_prep(elem, d, P.dp, Q, B, P.Bp, direct ? nullptr : w + P.o_qp, need_t ? w + P.o_qt : nullptr, J, M,
                           P.Mp, direct ? nullptr : w + P.o_jp, need_t ? w + P.o_jt : nullptr, s));
  }
  const int bf = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, sw = CU_TENSOR_MAP_SWIZZLE_128B;
  const void *qs = direct ? Q : (const void *)(w + P.o_qp), *js = direct ? J : (const void *)(w + P.o_jp);
  const uint64_t inner = direct ? (uint64_t)d : (uint64_t)P.dp, rs = inner * 2;
  const uint64_t qrows = direct ? (uint64_t)B : (uint64_t)P.Bp, jrows = direct ? (uint64_t)M : (uint64_t)P.Mp;
  bool ok = encode_tmap_2d(&T.qr, bf, qs, inner, qrows, rs, 64, 128, sw) &&
            encode_tmap_2d(&T.qc, bf, qs, inner, qrows, rs, 64, 64, sw) &&
            encode_tmap_2d(&T.jr, bf, js, inner, jrows, rs, 64, 128, sw) &&
            encode_tmap_2d(&T.jc, bf, js, inner, jrows, rs, 64, 64, sw);
  if (ok && need_t)
    ok = encode_tmap_2d(&T.qt, bf, w + P.o_qt, P.Bp, P.dp, (uint64_t)P.Bp * 2, 64, P.dp, sw) &&
         encode_tmap_2d(&T.jt, bf, w + P.o_jt, P.Mp, P.dp, (uint64_t)P.Mp * 2, 64, P.dp, sw);
  if (!ok) return fail(LR_ERR_CUDA, "cannot encode the TMA descriptors of the loss operands");
  return LR_OK;
}

LossArgs loss_args(int B, int M, float inv_tau, const int32_t *pos, const uint32_t *mask, char *w,
                   const LossPlan &P) {
  LossArgs a{};
  a.B = B;
  a.M = M;
  a.dp = P.dp;
  a.rows_p = P.Bp;
  a.n_ctiles = P.n_ctiles;
  a.c_per_split = P.c_per_split;
  a.inv_tau = inv_tau;
  a.inv_b = 1.0f / (float)B;
  a.pos = pos;
  a.mask = mask;
  a.Mw = (M + 31) / 32;
  a.part_m = (float *)(w + P.o_pm);
  a.part_s = (float *)(w + P.o_ps);
  a.zpos = (float *)(w + P.o_zp);
  a.status = (uint32_t *)(w + P.o_st);
  return a;
}

}  // namespace

extern "C" {

size_t lr_score_workspace_size(int32_t B, int32_t M, int32_t d) {
  if (B < 1 || M < 1 || d < 1 || d > 128) return 0;
  return loss_plan(B, M, d, current_sms()).total;
}

lr_status lr_score_forward(const void *Q, const void *J, int32_t B, int32_t M, int32_t d, int32_t dtype,
                           const int32_t *pos, const uint32_t *mask_bits, float inv_tau, float *loss, float *lse,
                           void *workspace, size_t workspace_bytes, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const LossPlan P = loss_plan(B, M, d, current_sms());
  lr_status st = loss_check(Q, J, B, M, d, dtype, pos, mask_bits, workspace, workspace_bytes, P);
  if (st != LR_OK) return st;
  if (!is_device_ptr(loss) || !is_device_ptr(lse)) return fail(LR_ERR_INVALID, "loss and lse must be device memory");
  char *w = (char *)workspace;
  LossMaps T;
  st = loss_prepare(Q, J, B, M, d, dtype, w, P, T, false, s);
  if (st != LR_OK) return st;
  LossArgs a = loss_args(B, M, inv_tau, pos, mask_bits, w, P);
  LR_CK(launch_loss_pass(0, a, P.Bp / 128, P.splits, &T.qr, &T.jc, nullptr, s));
  LR_CK(launch_loss_combine(a, 4 * P.splits, lse, (double *)(w + P.o_bs), (uint32_t *)(w + P.o_st) + 1, loss, s));
  return LR_OK;
}

lr_status lr_score_backward(const void *Q, const void *J, int32_t B, int32_t M, int32_t d, int32_t dtype,
                            const int32_t *pos, const uint32_t *mask_bits, float inv_tau, const float *lse,
                            const float *dloss, float *dQ, float *dJ, void *workspace, size_t workspace_bytes,
                            void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const LossPlan P = loss_plan(B, M, d, current_sms());
  lr_status st = loss_check(Q, J, B, M, d, dtype, pos, mask_bits, workspace, workspace_bytes, P);
  if (st != LR_OK) return st;
  if (!is_device_ptr(lse) || !is_device_ptr(dQ) || !is_device_ptr(dJ) || (dloss && !is_device_ptr(dloss)))
    return fail(LR_ERR_INVALID, "lse, dloss, dQ and dJ must be device memory");
  char *w = (char *)workspace;
  LossMaps T;
  st = loss_prepare(Q, J, B, M, d, dtype, w, P, T, true, s);
  if (st != LR_OK) return st;
  // dQ: query tiles against job tiles, per-split partials, then their sum
  LossArgs a = loss_args(B, M, inv_tau, pos, mask_bits, w, P);
  a.lse = lse;
  a.dloss = dloss;
  a.out = (float *)(w + P.o_dq);
  a.out_split = (size_t)P.Bp * P.dp;
  a.out_ld = P.dp;
  a.out_cols = P.dp;
  LR_CK(launch_loss_pass(1, a, P.Bp / 128, P.splits, &T.qr, &T.jc, &T.jt, s));
  LR_CK(launch_loss_dq_reduce((const float *)(w + P.o_dq), P.splits, (size_t)P.Bp * P.dp, B, d, P.dp, dQ, s));
  // dJ: job tiles against query tiles, per-split partials, then their sum
  LossArgs b = a;
  b.n_ctiles = P.nj_ctiles;
  b.c_per_split = P.cj_per_split;
  b.out = (float *)(w + P.o_dj);
  b.out_split = (size_t)P.Mp * P.dp;
  b.out_ld = P.dp;
  b.out_cols = P.dp;
  LR_CK(launch_loss_pass(2, b, P.Mp / 128, P.splits_j, &T.jr, &T.qc, &T.qt, s));
  LR_CK(launch_loss_dq_reduce((const float *)(w + P.o_dj), P.splits_j, (size_t)P.Mp * P.dp, M, d, P.dp, dJ, s));
  return LR_OK;
}

// ---------------------------------------------------------------- hard negatives
// Workspace of lr_hard_negatives: the loss passes' operand copies, then the
// selection keys [Bp][Mp] and the per-query selection state.
struct HnLayout {
  size_t keys, negc, cnt, kq, ovf, flag, nflag, err, prefix, krem, zero_end, total;
};

HnLayout hn_layout(const LossPlan &P, int B) {
  HnLayout H{};
  Carver cv;
  cv.off = P.total;
  H.keys = cv.take<uint64_t>((size_t)P.Bp * P.Mp);
  H.negc = cv.take<unsigned long long>(B);
  H.cnt = cv.take<uint32_t>(B);
  H.ovf = cv.take<uint32_t>(B);
  H.flag = cv.take<uint32_t>(B);
  H.nflag = cv.take<uint32_t>(1);
  H.err = cv.take<uint32_t>(1);
  H.prefix = cv.take<uint64_t>(B);
  H.krem = cv.take<int32_t>(B);
  H.zero_end = cv.take<char>(0);
  H.kq = cv.take<int32_t>(B);
  H.total = align_up(cv.off, 256);
  return H;
}

size_t lr_hard_negatives_workspace_size(int32_t B, int32_t M, int32_t d) {
  if (B < 1 || M < 1 || d < 1 || d > 128) return 0;
  return hn_layout(loss_plan(B, M, d, current_sms()), B).total;
}

lr_status lr_hard_negatives(const void *Q, const void *J, int32_t B, int32_t M, int32_t d, int32_t dtype,
                            const int32_t *pos, const uint32_t *mask_bits, int32_t n_neg, int32_t *out_ids,
                            float *out_scores, int32_t *out_count, uint32_t *out_mask, void *workspace,
                            size_t workspace_bytes, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const LossPlan P = loss_plan(B, M, d, current_sms());
  lr_status st = loss_check(Q, J, B, M, d, dtype, pos, mask_bits, workspace, P.total, P);
  if (st != LR_OK) return st;
  const HnLayout H = hn_layout(P, B);
  if (workspace_bytes < H.total) return fail(LR_ERR_WORKSPACE, "workspace smaller than lr_hard_negatives_workspace_size()");
  if (n_neg < 1 || n_neg > kMaxK || n_neg > M) return fail(LR_ERR_INVALID, "n_neg must be in [1, min(4096, M)]");
  if (!out_ids || !out_scores || !is_device_ptr(out_ids) || !is_device_ptr(out_scores) ||
      (out_count && !is_device_ptr(out_count)) || (out_mask && !is_device_ptr(out_mask)))
    return fail(LR_ERR_INVALID, "outputs must be device memory");
  if (out_mask && !out_count) return fail(LR_ERR_INVALID, "out_mask needs out_count");
  char *w = (char *)workspace;
  LossMaps T;
  st = loss_prepare(Q, J, B, M, d, dtype, w, P, T, false, s);
  if (st != LR_OK) return st;
  LR_CK(cudaMemsetAsync(w + H.negc, 0, H.zero_end - H.negc, s));
  LossArgs a = loss_args(B, M, 1.0f, pos, mask_bits, w, P);
  a.keys = (uint64_t *)(w + H.keys);
  a.keys_ld = P.Mp;
  a.key_cnt = (uint32_t *)(w + H.cnt);
  LR_CK(launch_loss_pass(3, a, P.Bp / 128, P.splits, &T.qr, &T.jc, nullptr, s));
  LR_CK(launch_hn_setup(B, n_neg, a.key_cnt, (int32_t *)(w + H.kq), (unsigned long long *)(w + H.negc), s));
  SelectArgs fa{};
  fa.mode = 1;
  fa.buf = a.keys;
  fa.cap = P.Mp;
  fa.cnt = (uint32_t *)(w + H.cnt);
  fa.overflow = (uint32_t *)(w + H.ovf);
  fa.k = (const int32_t *)(w + H.kq);
  fa.pass_cnt = (const unsigned long long *)(w + H.negc);
  fa.k_stride = n_neg;
  fa.out_ids = out_ids;
  fa.out_scores = out_scores;
  fa.out_count = out_count;
  fa.flag = (uint32_t *)(w + H.flag);
  fa.n_flagged = (uint32_t *)(w + H.nflag);
  fa.fb_prefix = (uint64_t *)(w + H.prefix);
  fa.fb_krem = (int32_t *)(w + H.krem);
  fa.err = (uint32_t *)(w + H.err);
  LR_CK(launch_select(fa, B, s));
  if (out_mask) {
    const int Mw = (M + 31) / 32;
    LR_CK(cudaMemsetAsync(out_mask, 0, sizeof(uint32_t) * (size_t)B * Mw, s));
    LR_CK(launch_hn_mask(out_ids, out_count, B, n_neg, Mw, out_mask, s));
  }
  return LR_OK;
}

lr_status lr_score_status(void *workspace, int32_t B, int32_t M, int32_t d, void *stream) {
  if (!workspace) return fail(LR_ERR_INVALID, "workspace is null");
  const LossPlan P = loss_plan(B, M, d, current_sms());
  uint32_t e = 0;
  cudaStream_t s = (cudaStream_t)stream;
  LR_CK(cudaMemcpyAsync(&e, (char *)workspace + P.o_st, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  LR_CK(cudaStreamSynchronize(s));
  if (e & kErrTimeout) return fail(LR_ERR_TIMEOUT, "a bounded device wait of the loss kernels timed out");
  return LR_OK;
}

}  // extern "C"
