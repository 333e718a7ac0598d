// Top-K of dense score rows (appendix "Fast Top K Selection").
//
// The appendix selects the top k of a long score vector without sorting it:
// every score goes to a bucket, bucketised score = (int)(score * G) + G for
// scores in [-1, 1] and a granularity G (100 in the paper), the buckets are
// counted, the counts are accumulated from the highest bucket down to the first
// bucket l at which at least k scores are gathered, and only the scores in
// buckets >= l are sorted.  The bounds of the scores must be known; here the
// caller passes them ([lo, hi] is mapped onto [-1, 1], which for cosine scores
// is the paper's formula itself) and scores outside go to the end buckets.
//
// B300 form: each row is split over many CTAs.  Pass 1 counts the buckets in
// shared memory and adds them to the row's histogram in the workspace; the
// last CTA of a row (completion counter) finds l.  Pass 2 appends the 64-bit
// keys (ordered score, ~index) of the scores in buckets >= l to the row's
// candidate list.  Pass 3 is the library's exact selection (radix select of
// the k-th key, bitonic sort of the top k), so equal scores order by index.
// LR_TOPK_RADIX skips the buckets (l = 0: every score is a candidate) and
// leaves the whole row to the radix selection, the library's bound-free way.
#include <cmath>

#include "lr_internal.h"

namespace lr {
namespace {

constexpr int kTkThreads = 256;
constexpr int kTkMaxG = 2048;  // granularity: 2G + 1 buckets in shared memory

struct TopkWs {
  uint32_t *hist;               // [B][nb]
  uint32_t *ctr;                // [B] CTAs of pass 1 finished
  int32_t *thr;                 // [B] bucket l
  uint32_t *cnt;                // [B] candidates gathered
  uint32_t *ovf;                // [B] zero (the candidate list holds a whole row)
  int32_t *kq;                  // [B] k
  unsigned long long *npass;    // [B] n
  uint32_t *flag, *n_flag, *err;
  uint64_t *prefix;             // [B]
  int32_t *krem;                // [B]
  uint64_t *cand;               // [B][n]
};

size_t al256(size_t v) { return (v + 255) / 256 * 256; }

// Workspace layout for B rows of n scores; offsets in bytes.
struct TopkLayout {
  size_t hist, ctr, thr, cnt, ovf, kq, npass, flag, nflag, err, prefix, krem, cand, clear_end, total;
};

TopkLayout topk_layout(int B, int64_t n) {
  TopkLayout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = al256(o + bytes);
    return at;
  };
  L.hist = take((size_t)B * (2 * kTkMaxG + 1) * 4);
  L.ctr = take((size_t)B * 4);
  L.cnt = take((size_t)B * 4);
  L.ovf = take((size_t)B * 4);
  L.flag = take((size_t)B * 4);
  L.nflag = take(4);
  L.err = take(4);
  L.clear_end = o;  // everything above starts at zero
  L.thr = take((size_t)B * 4);
  L.kq = take((size_t)B * 4);
  L.npass = take((size_t)B * 8);
  L.prefix = take((size_t)B * 8);
  L.krem = take((size_t)B * 4);
  L.cand = take((size_t)B * (size_t)n * 8);
  L.total = o;
  return L;
}

// The appendix's bucketised score of s, with [lo, hi] mapped onto [-1, 1]
// (t = (s - c) * scale); truncation toward zero as the (int) cast does, clamped
// to the 2G + 1 buckets.  Non-decreasing in s, so a bucket threshold keeps every
// score above it.
__device__ __forceinline__ int bucket_of(float s, float c, float scale, int G) {
  const float t = (s - c) * scale;
  const int b = __float2int_rz(t * (float)G) + G;
  return b < 0 ? 0 : (b > 2 * G ? 2 * G : b);
}

__global__ void __launch_bounds__(kTkThreads) k_topk_hist(const float *S, int64_t n, int64_t stride, float c,
                                                          float scale, int G, int k, TopkWs w) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
  extern __shared__ uint32_t h[];
  __shared__ bool last;
  const int row = blockIdx.y, nb = 2 * G + 1, tid = threadIdx.x;
  for (int i = tid; i < nb; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  const float *r = S + (size_t)row * (size_t)stride;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + tid; i < n; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&h[bucket_of(__ldg(r + i), c, scale, G)], 1u);
  __syncthreads();
  uint32_t *gh = w.hist + (size_t)row * nb;
  for (int i = tid; i < nb; i += blockDim.x)
    if (h[i]) atomicAdd(&gh[i], h[i]);
  __threadfence();
  __syncthreads();
  if (tid == 0) last = atomicAdd(&w.ctr[row], 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last || tid >= 32) return;
  __threadfence();
  // the last CTA of the row: from the top bucket down, the first bucket at
  // which at least min(k, n) scores are gathered.  Each lane owns a run of
  // buckets counted from the top; a prefix sum over lanes finds the run.
  const int lane = tid;
  const uint32_t need = (uint32_t)((int64_t)k < n ? (int64_t)k : n);
  const int per = (nb + 31) / 32;
  const int top0 = nb - 1 - lane * per;  // this lane's first (highest) bucket
  uint32_t sum = 0;
  for (int j = 0; j < per; ++j) {
    const int b = top0 - j;
    if (b >= 0) sum += __ldcg(gh + b);
  }
  uint32_t incl = sum;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, off);
    if (lane >= off) incl += t;
  }
  const uint32_t excl = incl - sum;
  const unsigned hit = __ballot_sync(0xFFFFFFFFu, excl < need && need <= incl);
  if (hit == 0u) {  // need == 0 cannot happen (k >= 1, n >= 1); keep every bucket
    if (lane == 0) w.thr[row] = 0;
  } else if (lane == __ffs(hit) - 1) {
    uint32_t cum = excl;
    int l = 0;
    for (int j = 0; j < per; ++j) {
      const int b = top0 - j;
      if (b < 0) break;
      cum += __ldcg(gh + b);
      if (cum >= need) {
        l = b;
        break;
      }
    }
    w.thr[row] = l;
  }
  if (lane == 0) {
    w.kq[row] = k;
    w.npass[row] = (unsigned long long)n;
  }
}

// Keys of the scores in buckets >= l (every score with l = 0), appended with
// one shared atomic per warp.
__global__ void __launch_bounds__(kTkThreads) k_topk_gather(const float *S, int64_t n, int64_t stride, float c,
                                                            float scale, int G, int use_buckets, TopkWs w,
                                                            int32_t *thr_or_null) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
  const int row = blockIdx.y, lane = threadIdx.x & 31;
  const int l = use_buckets ? w.thr[row] : 0;
  const float *r = S + (size_t)row * (size_t)stride;
  uint64_t *dst = w.cand + (size_t)row * (size_t)n;
  for (int64_t b0 = (int64_t)blockIdx.x * blockDim.x; b0 < n; b0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = b0 + threadIdx.x;  // whole warps every trip
    const float s = i < n ? __ldg(r + i) : 0.f;
    const bool take = i < n && (!use_buckets || bucket_of(s, c, scale, G) >= l);
    const unsigned m = __ballot_sync(0xFFFFFFFFu, take);
    if (m == 0u) continue;
    const int lead = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == lead) base = atomicAdd(&w.cnt[row], (uint32_t)__popc(m));
    base = __shfl_sync(0xFFFFFFFFu, base, lead);
    if (take) dst[base + (uint32_t)__popc(m & ((1u << lane) - 1u))] = make_key(s, (uint32_t)i);
  }
  if (thr_or_null != nullptr && blockIdx.x == 0 && threadIdx.x == 0) thr_or_null[row] = l;
}

// LR_TOPK_RADIX: no buckets; K and the row length for the selection.
__global__ void k_topk_setup(int B, int k, int64_t n, TopkWs w) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= B) return;
  w.thr[row] = 0;
  w.kq[row] = k;
  w.npass[row] = (unsigned long long)n;
}

bool topk_dev_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace lr

using namespace lr;

extern "C" size_t lr_topk_workspace_size(int32_t B, int64_t n) {
  if (B < 1 || n < 1) return 0;
  return topk_layout(B, n).total;
}

extern "C" lr_status lr_topk(const float *scores, int32_t B, int64_t n, int64_t row_stride, int32_t k,
                             int32_t method, float lo, float hi, int32_t granularity, int32_t *out_ids,
                             float *out_scores, int32_t *out_threshold_bucket, void *workspace,
                             size_t workspace_bytes, void *stream) {
  if (!scores || !out_ids || !out_scores || !workspace) return fail(LR_ERR_INVALID, "lr_topk: null pointer");
  if (B < 1 || n < 1 || n > 0x7FFFFFFFll) return fail(LR_ERR_INVALID, "lr_topk: need B >= 1 and 1 <= n < 2^31");
  if (row_stride < n) return fail(LR_ERR_INVALID, "lr_topk: row_stride must be >= n");
  if (k < 1 || k > kMaxK) return fail(LR_ERR_INVALID, "lr_topk: k must be in [1, 4096]");
  if (method != LR_TOPK_BUCKET && method != LR_TOPK_RADIX) return fail(LR_ERR_INVALID, "lr_topk: unknown method");
  if (method == LR_TOPK_BUCKET && (granularity < 1 || granularity > kTkMaxG || !(hi > lo) || !std::isfinite(lo) ||
                                   !std::isfinite(hi)))
    return fail(LR_ERR_INVALID, "lr_topk: bucket method needs finite lo < hi and granularity in [1, 2048]");
  const TopkLayout L = topk_layout(B, n);
  if (workspace_bytes < L.total) return fail(LR_ERR_WORKSPACE, "lr_topk: workspace smaller than lr_topk_workspace_size()");
  if (!topk_dev_ptr(scores) || !topk_dev_ptr(out_ids) || !topk_dev_ptr(out_scores) || !topk_dev_ptr(workspace) ||
      (out_threshold_bucket && !topk_dev_ptr(out_threshold_bucket)))
    return fail(LR_ERR_INVALID, "lr_topk: scores, outputs and workspace must be device memory");
  cudaStream_t s = (cudaStream_t)stream;
  char *w0 = static_cast<char *>(workspace);
  TopkWs w{};
  w.hist = (uint32_t *)(w0 + L.hist);
  w.ctr = (uint32_t *)(w0 + L.ctr);
  w.thr = (int32_t *)(w0 + L.thr);
  w.cnt = (uint32_t *)(w0 + L.cnt);
  w.ovf = (uint32_t *)(w0 + L.ovf);
  w.kq = (int32_t *)(w0 + L.kq);
  w.npass = (unsigned long long *)(w0 + L.npass);
  w.flag = (uint32_t *)(w0 + L.flag);
  w.n_flag = (uint32_t *)(w0 + L.nflag);
  w.err = (uint32_t *)(w0 + L.err);
  w.prefix = (uint64_t *)(w0 + L.prefix);
  w.krem = (int32_t *)(w0 + L.krem);
  w.cand = (uint64_t *)(w0 + L.cand);
#define TK_CK(call)                                     \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)
  TK_CK(cudaMemsetAsync(w0, 0, L.clear_end, s));
  int dev = 0, sms = 148;
  TK_CK(cudaGetDevice(&dev));
  TK_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // chunks per row: enough CTAs to cover the SMs a few times over all rows
  const int64_t per_cta = (int64_t)kTkThreads * 16;
  int64_t chunks = (n + per_cta - 1) / per_cta;
  const int64_t want = (4 * (int64_t)sms + B - 1) / B;
  if (chunks > want) chunks = want;
  if (chunks < 1) chunks = 1;
  const dim3 grid((unsigned)chunks, (unsigned)B);
  const bool buckets = method == LR_TOPK_BUCKET;
  const int G = buckets ? granularity : 1;
  const float c = buckets ? 0.5f * (lo + hi) : 0.f;
  const float scale = buckets ? 2.0f / (hi - lo) : 1.f;
  if (buckets) {
    const size_t smem = (size_t)(2 * G + 1) * sizeof(uint32_t);
    TK_CK(launch_pdl(k_topk_hist, dim3(grid), dim3(kTkThreads), smem, s, scores, n, row_stride, c, scale, G, k, w));
  } else {
    TK_CK(launch_pdl(k_topk_setup, dim3((unsigned)((B + 127) / 128)), dim3(128), 0, s, B, k, n, w));
  }
  TK_CK(launch_pdl(k_topk_gather, dim3(grid), dim3(kTkThreads), 0, s, scores, n, row_stride, c, scale, G,
                   buckets ? 1 : 0, w, out_threshold_bucket));
  SelectArgs a{};
  a.mode = 1;
  a.buf = w.cand;
  a.cap = n;
  a.cnt = w.cnt;
  a.overflow = w.ovf;
  a.k = w.kq;
  a.pass_cnt = w.npass;
  a.k_stride = k;
  a.out_ids = out_ids;
  a.out_scores = out_scores;
  a.flag = w.flag;
  a.n_flagged = w.n_flag;
  a.fb_prefix = w.prefix;
  a.fb_krem = w.krem;
  a.err = w.err;
  TK_CK(launch_select(a, B, s));
#undef TK_CK
  return LR_OK;
}
