// lr_search_noalloc: exact top-K over caller-owned device arrays without any
// device allocation.
//
// Who needs it: callers that may not call cudaMalloc -- a plugin living inside a
// host framework that owns every device allocation through its own pool, or a
// latency-critical serving thread where an allocation could block on the
// driver or fail mid-request.  They cannot build an lr_index (which allocates
// its workspace), so this entry point takes the embeddings, queries, per-query
// pass bitmaps and outputs from the caller and keeps every intermediate in one
// fixed file-scope device array.
//
// The scratch array below is part of the library image: every GPU that loads
// the library holds it (about 10 MiB) until the process exits.  All calls share
// it, so two calls that overlap on the GPU (different streams, or different
// host threads) race on it and must be serialised by the caller.  Each call
// clears what has to start at zero before its first kernel, the device error
// word included: lr_search_noalloc_status reads that word for the last call.

#include "lr_internal.h"
#include "ptx.h"

namespace lr {
namespace {

constexpr int kNaMaxB = kGemvMaxQ;           // queries per call (one scan launch)
constexpr int kNaMaxK = 1024;
constexpr int64_t kNaMaxN = int64_t(1) << 24;  // jobs
constexpr int64_t kNaSampRows = 32768;       // rows in the threshold sample (upper bound)
constexpr int64_t kNaCandCap = 131072;       // candidate keys per query

constexpr size_t al(size_t v) { return (v + 255) / 256 * 256; }
// scratch layout (byte offsets)
constexpr size_t kOffTau = 0;
constexpr size_t kOffPrefix = kOffTau + 8 * kNaMaxB;
constexpr size_t kOffPass = kOffPrefix + 8 * kNaMaxB;
constexpr size_t kOffCnt = kOffPass + 8 * kNaMaxB;
constexpr size_t kOffOvf = kOffCnt + 4 * kNaMaxB;
constexpr size_t kOffScnt = kOffOvf + 4 * kNaMaxB;
constexpr size_t kOffSovf = kOffScnt + 4 * kNaMaxB;
constexpr size_t kOffFlag = kOffSovf + 4 * kNaMaxB;
constexpr size_t kOffKrem = kOffFlag + 4 * kNaMaxB;
constexpr size_t kOffNflag = kOffKrem + 4 * kNaMaxB;
constexpr size_t kStateBytes = kOffNflag + 4;        // cleared by every call
constexpr size_t kOffDone = al(kStateBytes);
constexpr size_t kOffErr = kOffDone + 4;
constexpr size_t kOffK = al(kOffErr + 8);  // after the error word and the work counter
constexpr size_t kOffRank = kOffK + 4 * kNaMaxB;
constexpr size_t kOffSlots = al(kOffRank + 4 * kNaMaxB);
constexpr size_t kOffQc = al(kOffSlots + 8 * kNaMaxB);
constexpr size_t kOffCl = kOffQc + 4 * (kNaMaxB + 1);
constexpr size_t kOffCs = kOffCl + 4 * (kNaMaxB + 1);
constexpr size_t kOffHist = al(kOffCs + 4 * kNaMaxB);
constexpr size_t kHistBytes = (size_t)kNaMaxB * kFbBins * 4;  // cleared by every call
constexpr size_t kOffSamp = al(kOffHist + kHistBytes);
constexpr size_t kOffCand = al(kOffSamp + (size_t)kNaMaxB * kNaSampRows * 8);
constexpr size_t kScratchBytes = al(kOffCand + (size_t)kNaMaxB * kNaCandCap * 8);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array on the current device.  Looked up on
// every call (no work is enqueued), so a module reloaded after a device reset
// never leaves a stale address behind.
lr_status scratch_address(unsigned char **base) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(lr_search_noalloc scratch)");
  *base = static_cast<unsigned char *>(p);
  return LR_OK;
}

// Device (or managed) memory?  cudaPointerGetAttributes allocates nothing.
bool na_device_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool aligned(const void *p, uintptr_t a) { return reinterpret_cast<uintptr_t>(p) % a == 0; }

// Filter tables for B one-term queries whose "terms" are the caller's bitmaps,
// plus per-query K and threshold rank.
__global__ void k_noalloc_setup(unsigned char *base, const uint32_t *bitmap, int64_t stride, int B, int K,
                                int rank) {
  const int t = threadIdx.x;
  uint64_t *slots = reinterpret_cast<uint64_t *>(base + kOffSlots);
  int32_t *qc = reinterpret_cast<int32_t *>(base + kOffQc);
  int32_t *cl = reinterpret_cast<int32_t *>(base + kOffCl);
  int32_t *cs = reinterpret_cast<int32_t *>(base + kOffCs);
  int32_t *kq = reinterpret_cast<int32_t *>(base + kOffK);
  int32_t *rk = reinterpret_cast<int32_t *>(base + kOffRank);
  const bool filtered = bitmap != nullptr;
  if (t <= B) {
    qc[t] = filtered ? t : 0;  // query b owns clause b (or no clause at all)
    cl[t] = t;                 // clause b holds slot b
  }
  if (t < B) {
    if (filtered) slots[t] = (uint64_t)(uintptr_t)(bitmap + (size_t)t * (size_t)stride);
    cs[t] = t;
    kq[t] = K;
    rk[t] = rank;
  }
}

}  // namespace
}  // namespace lr

using namespace lr;

extern "C" lr_status lr_search_noalloc(const float *X, int64_t n_jobs, int32_t dim, const float *q, int32_t B,
                                       const uint32_t *pass_bitmap, int64_t bitmap_stride_words, int32_t k,
                                       int32_t *out_ids, float *out_scores, int32_t *out_count, void *stream) {
  if (!X || !q || !out_ids || !out_scores) return fail(LR_ERR_INVALID, "lr_search_noalloc: null pointer");
  if (dim != 32 && dim != 64 && dim != 128 && dim != 256)
    return fail(LR_ERR_UNSUPPORTED, "lr_search_noalloc: dim must be 32, 64, 128 or 256");
  if (n_jobs < 1 || n_jobs > kNaMaxN)
    return fail(LR_ERR_WORKSPACE, "lr_search_noalloc: n_jobs must be in [1, 16777216] (fixed scratch)");
  if (B < 1 || B > kNaMaxB) return fail(LR_ERR_WORKSPACE, "lr_search_noalloc: B must be in [1, 8] (fixed scratch)");
  if (k < 1 || k > kNaMaxK) return fail(LR_ERR_WORKSPACE, "lr_search_noalloc: K must be in [1, 1024] (fixed scratch)");
  const int64_t n_groups = (n_jobs + kGroupRows - 1) / kGroupRows;
  if (pass_bitmap && (bitmap_stride_words < n_groups * kGroupWords || bitmap_stride_words % kGroupWords != 0))
    return fail(LR_ERR_INVALID, "lr_search_noalloc: bitmap row stride must be a multiple of 8 words and cover "
                                "ceil(n_jobs/256)*8 words");
  if (pass_bitmap && !aligned(pass_bitmap, 32))
    return fail(LR_ERR_INVALID, "lr_search_noalloc: pass_bitmap must be 32-byte aligned");
  // the scan copies rows in 16-byte pieces; queries and outputs are 4-byte words
  if (!aligned(X, 16)) return fail(LR_ERR_INVALID, "lr_search_noalloc: X must be 16-byte aligned");
  if (!aligned(q, 4) || !aligned(out_ids, 4) || !aligned(out_scores, 4) || (out_count && !aligned(out_count, 4)))
    return fail(LR_ERR_INVALID, "lr_search_noalloc: q and the outputs must be 4-byte aligned");
  // every array is read or written by kernels: a host pointer would fault the device
  if (!na_device_ptr(X) || !na_device_ptr(q) || !na_device_ptr(out_ids) || !na_device_ptr(out_scores) ||
      (out_count && !na_device_ptr(out_count)) || (pass_bitmap && !na_device_ptr(pass_bitmap)))
    return fail(LR_ERR_INVALID, "lr_search_noalloc: X, q, pass_bitmap and the outputs must be device memory");

  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
  unsigned char *base = nullptr;
  {
    const lr_status st = scratch_address(&base);
    if (st != LR_OK) return st;
  }
  cudaStream_t s = (cudaStream_t)stream;

  // threshold sample: every stride-th 256-row group, at most kNaSampRows rows;
  // no sample (every passing job is a candidate) when the index fits the buffer
  int stride = 0;
  int64_t samp_groups = 0, samp_rows = 0;
  int rank = 0;
  if (n_jobs > kNaCandCap) {
    stride = (int)((n_groups + (kNaSampRows / kGroupRows) - 1) / (kNaSampRows / kGroupRows));
    if (stride < 2) stride = 2;
    const int64_t begin = stride / 2;
    samp_groups = (n_groups - begin + stride - 1) / stride;
    const int64_t last = begin + (samp_groups - 1) * (int64_t)stride;
    samp_rows = (samp_groups - 1) * kGroupRows + ((n_jobs - last * kGroupRows) < kGroupRows
                                                      ? (n_jobs - last * kGroupRows) : kGroupRows);
    const double frac = (double)samp_rows / (double)n_jobs;
    double r = 4.0 * (double)k * frac;
    r = r < 64.0 ? 64.0 : (double)(int64_t)(r + 0.999999);
    rank = (int)r;
  }

  uint64_t *tau = (uint64_t *)(base + kOffTau), *prefix = (uint64_t *)(base + kOffPrefix);
  unsigned long long *pass = (unsigned long long *)(base + kOffPass);
  uint32_t *cnt = (uint32_t *)(base + kOffCnt), *ovf = (uint32_t *)(base + kOffOvf);
  uint32_t *scnt = (uint32_t *)(base + kOffScnt), *sovf = (uint32_t *)(base + kOffSovf);
  uint32_t *flag = (uint32_t *)(base + kOffFlag), *nflag = (uint32_t *)(base + kOffNflag);
  int32_t *krem = (int32_t *)(base + kOffKrem), *kq = (int32_t *)(base + kOffK), *rk = (int32_t *)(base + kOffRank);
  uint32_t *done = (uint32_t *)(base + kOffDone), *err = (uint32_t *)(base + kOffErr);
  uint32_t *hist = (uint32_t *)(base + kOffHist);
  uint64_t *samp = (uint64_t *)(base + kOffSamp), *cand = (uint64_t *)(base + kOffCand);

#define NA_CK(call)                                     \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

  NA_CK(cudaMemsetAsync(base, 0, kStateBytes, s));
  NA_CK(cudaMemsetAsync(done, 0, 12, s));  // completion counter, error word, work counter
  NA_CK(cudaMemsetAsync(hist, 0, kHistBytes, s));
  k_noalloc_setup<<<1, 32, 0, s>>>(base, pass_bitmap, bitmap_stride_words, B, k, rank);
  NA_CK(cudaGetLastError());

  ScanArgs a{};
  a.X = X;
  a.n = n_jobs;
  a.d_pad = dim;
  a.Q = q;
  a.q_base = 0;
  a.nq = B;
  a.slot_bm = (const uint32_t *const *)(base + kOffSlots);
  a.n_slots = pass_bitmap ? B : 0;
  a.qc_off = (const int32_t *)(base + kOffQc);
  a.cl_off = (const int32_t *)(base + kOffCl);
  a.cl_slot = (const int32_t *)(base + kOffCs);
  a.n_groups = n_groups;
  a.g_begin = 0;
  a.g_step = 1;
  a.mode = kCollect;
  a.err = err;
  a.done_ctr = done;
  a.work_ctr = done + 2;
  a.batch = B;
  const int vec = dim / 32;
  const int nqt = B <= 1 ? 1 : B <= 2 ? 2 : B <= 4 ? 4 : 8;
  auto grid_for = [&](int64_t groups) {
    int64_t want = (groups + 3) / 4;
    int64_t cap = (int64_t)sms;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
  };

  if (stride > 0) {
    ScanArgs t = a;
    t.g_begin = stride / 2;
    t.g_step = stride;
    t.tau = nullptr;
    t.buf = samp;
    t.buf_cap = kNaSampRows;
    t.buf_cnt = scnt;
    t.overflow = sovf;
    NA_CK(launch_scan_gemv(t, nqt, vec, grid_for(samp_groups), s));
    SelectArgs th{};
    th.mode = 0;
    th.buf = samp;
    th.cap = kNaSampRows;
    th.cnt = scnt;
    th.overflow = sovf;
    th.rank = rk;
    th.tau = tau;
    NA_CK(launch_select(th, B, s));
  }
  ScanArgs m = a;
  m.tau = tau;
  m.buf = cand;
  m.buf_cap = kNaCandCap;
  m.buf_cnt = cnt;
  m.overflow = ovf;
  m.pass_cnt = pass;
  NA_CK(launch_scan_gemv(m, nqt, vec, grid_for(n_groups), s));
  SelectArgs fa{};
  fa.mode = 1;
  fa.buf = cand;
  fa.cap = kNaCandCap;
  fa.cnt = cnt;
  fa.overflow = ovf;
  fa.k = kq;
  fa.pass_cnt = pass;
  fa.k_stride = k;
  fa.out_ids = out_ids;
  fa.out_scores = out_scores;
  fa.out_count = out_count;
  fa.flag = flag;
  fa.n_flagged = nflag;
  fa.fb_prefix = prefix;
  fa.fb_krem = krem;
  fa.err = err;
  NA_CK(launch_select(fa, B, s));
  // exact fallback for queries whose candidate set cannot prove exactness
  for (int p = 0; p < kFbPasses; ++p) {
    ScanArgs h = a;
    h.mode = kHist;
    h.hist_pass = p;
    h.prefix = prefix;
    h.krem = krem;
    h.hist = hist;
    h.tau_out = tau;
    h.active = flag;
    h.any_active = nflag;
    NA_CK(launch_scan_gemv(h, nqt, vec, grid_for(n_groups), s));
  }
  ScanArgs c = m;
  c.pass_cnt = nullptr;
  c.active = flag;
  c.any_active = nflag;
  NA_CK(launch_scan_gemv(c, nqt, vec, grid_for(n_groups), s));
  SelectArgs fb = fa;
  fb.only = flag;
  fb.any = nflag;
  fb.fallback_round = 1;
  NA_CK(launch_select(fb, B, s));
#undef NA_CK
  return LR_OK;
}

extern "C" lr_status lr_search_noalloc_status(void *stream) {
  unsigned char *base = nullptr;
  const lr_status st = scratch_address(&base);
  if (st != LR_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t e = 0;
  cudaError_t ce = cudaMemcpyAsync(&e, base + kOffErr, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return cuda_fail(ce, "lr_search_noalloc_status");
  if (e == 0u) return LR_OK;
  ce = cudaMemsetAsync(base + kOffErr, 0, sizeof(uint32_t), s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return cuda_fail(ce, "lr_search_noalloc_status");
  if (e & kErrTimeout) return fail(LR_ERR_TIMEOUT, "lr_search_noalloc: a bounded device wait timed out");
  return fail(LR_ERR_CUDA, "lr_search_noalloc: the selection state was inconsistent (device error word " +
                               std::to_string(e) + ")");
}
