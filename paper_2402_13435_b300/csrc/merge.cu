// Exact merge of per-part top-K lists (Sec. 5.3, "Communication cost"): the
// search is split by contiguous job-row ranges, each part returns its own top
// K' rows per query, and one exchange brings the G lists of every query
// together.  Because the parts hold disjoint jobs and every list is sorted by
// the same total order (score desc, id asc), the merged top K is the unsharded
// top K.
//
// Merge by rank: entry i of list g has exactly i entries of its own list above
// it, and in every other list h the number of entries above it is found by a
// binary search.  Its rank in the union is the sum, so each entry that ranks
// below k writes itself straight to its output position -- no sort and no
// block-wide barrier beyond staging.  Keys are the library's 64-bit (ordered
// score, ~id) keys, so equal scores order by ascending id.
#include "lr_internal.h"

namespace lr {
namespace {

constexpr int kMergeThreads = 256;
constexpr int kMergeMaxG = 64;

__device__ __forceinline__ uint64_t list_key(const int32_t *ids, const float *sc, int i) {
  return make_key(sc[i], (uint32_t)ids[i]);
}

// Entries of list (ids, sc, n) whose key is larger than `key` (the list is
// sorted by descending key).
__device__ __forceinline__ int count_above(const int32_t *ids, const float *sc, int n, uint64_t key) {
  int lo = 0, hi = n;  // answer in [lo, hi]
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (list_key(ids, sc, mid) > key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kMergeThreads) k_merge_topk(const int32_t *ids, const float *scores,
                                                              const int32_t *counts, int G, int B, int k_in, int k,
                                                              int32_t *out_ids, float *out_scores,
                                                              int32_t *out_count) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
  const int b = blockIdx.x;
  __shared__ int cnt[kMergeMaxG];
  __shared__ int total;
  if (threadIdx.x == 0) total = 0;
  __syncthreads();
  for (int g = threadIdx.x; g < G; g += blockDim.x) {
    int c = counts[(size_t)g * B + b];
    c = c < 0 ? 0 : (c > k_in ? k_in : c);
    cnt[g] = c;
    atomicAdd(&total, c);
  }
  __syncthreads();
  const int kout = total < k ? total : k;
  int32_t *oi = out_ids + (size_t)b * k;
  float *os = out_scores + (size_t)b * k;
  for (int i = kout + threadIdx.x; i < k; i += blockDim.x) {
    oi[i] = -1;
    os[i] = -INFINITY;
  }
  // every valid entry of every list: its rank in the union
  for (int g = 0; g < G; ++g) {
    const int32_t *gi = ids + ((size_t)g * B + b) * k_in;
    const float *gs = scores + ((size_t)g * B + b) * k_in;
    const int n = cnt[g] < k ? cnt[g] : k;  // entries past k of one list rank past k
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const uint64_t key = list_key(gi, gs, i);
      int rank = i;
      for (int h = 0; h < G && rank < k; ++h) {
        if (h == g) continue;
        const int32_t *hi = ids + ((size_t)h * B + b) * k_in;
        const float *hs = scores + ((size_t)h * B + b) * k_in;
        const int nh = cnt[h] < k ? cnt[h] : k;
        rank += count_above(hi, hs, nh, key);
      }
      if (rank < kout) {
        oi[rank] = gi[i];
        os[rank] = gs[i];
      }
    }
  }
  if (threadIdx.x == 0 && out_count) out_count[b] = kout;
}

}  // namespace

cudaError_t launch_merge_topk(const int32_t *ids, const float *scores, const int32_t *counts, int G, int B, int k_in,
                              int k, int32_t *out_ids, float *out_scores, int32_t *out_count, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  return launch_pdl(k_merge_topk, dim3((unsigned)B), dim3(kMergeThreads), 0, s, ids, scores, counts, G, B, k_in, k,
                    out_ids, out_scores, out_count);
}

namespace {

// Rotating scan: batch row b of a chunk's result (c_cnt[b] entries, sorted)
// merged into the running top-K of its query's lane (run_cnt entries, sorted,
// from the chunks before; the two hold disjoint rows).  Each entry's rank in
// the union is its index plus the entries of the other list above it; the
// first k_of[b] are staged in shared memory and written back to the lane.
__global__ void __launch_bounds__(kMergeThreads) k_lane_merge(const int32_t *c_ids, const float *c_sc,
                                                              const int32_t *c_cnt, int c_stride,
                                                              const int32_t *lane_of, const int32_t *k_of,
                                                              int32_t *run_ids, float *run_sc, int32_t *run_cnt,
                                                              int run_stride) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
  extern __shared__ __align__(16) unsigned char lm_smem[];
  const int b = blockIdx.x;
  const int lane = lane_of[b];
  const int k = k_of[b];
  int32_t *oi = reinterpret_cast<int32_t *>(lm_smem);
  float *os = reinterpret_cast<float *>(lm_smem) + run_stride;
  const int32_t *ci = c_ids + (size_t)b * c_stride;
  const float *cs = c_sc + (size_t)b * c_stride;
  int32_t *ri = run_ids + (size_t)lane * run_stride;
  float *rs = run_sc + (size_t)lane * run_stride;
  const int nc = min(min(c_cnt[b], c_stride), k), nr = min(run_cnt[lane], k);
  const int kout = min(nc + nr, k);
  for (int i = threadIdx.x; i < nr; i += blockDim.x) {
    const int rank = i + count_above(ci, cs, nc, list_key(ri, rs, i));
    if (rank < kout) {
      oi[rank] = ri[i];
      os[rank] = rs[i];
    }
  }
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    const int rank = i + count_above(ri, rs, nr, list_key(ci, cs, i));
    if (rank < kout) {
      oi[rank] = ci[i];
      os[rank] = cs[i];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kout; i += blockDim.x) {
    ri[i] = oi[i];
    rs[i] = os[i];
  }
  if (threadIdx.x == 0) run_cnt[lane] = kout;
}

__global__ void k_lane_reset(const int32_t *lanes, int n, int32_t *run_cnt) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) run_cnt[lanes[i]] = 0;
}

// Rows of finished lanes into a compact [n][k_stride] result block (-1 / -inf
// past each lane's count).
__global__ void __launch_bounds__(kMergeThreads) k_lane_gather(const int32_t *lanes, const int32_t *run_ids,
                                                               const float *run_sc, const int32_t *run_cnt,
                                                               int run_stride, int k_stride, int32_t *out_ids,
                                                               float *out_sc, int32_t *out_cnt) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
  const int j = blockIdx.x;
  const int lane = lanes[j];
  const int c = min(run_cnt[lane], k_stride);
  for (int i = threadIdx.x; i < k_stride; i += blockDim.x) {
    out_ids[(size_t)j * k_stride + i] = i < c ? run_ids[(size_t)lane * run_stride + i] : -1;
    out_sc[(size_t)j * k_stride + i] = i < c ? run_sc[(size_t)lane * run_stride + i] : -INFINITY;
  }
  if (threadIdx.x == 0) out_cnt[j] = c;
}

}  // namespace

cudaError_t launch_lane_merge(const int32_t *c_ids, const float *c_sc, const int32_t *c_cnt, int B, int c_stride,
                              const int32_t *lane_of, const int32_t *k_of, int32_t *run_ids, float *run_sc,
                              int32_t *run_cnt, int run_stride, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const size_t smem = (size_t)run_stride * 8;
  if (smem > 48u * 1024u) {
    const cudaError_t e = allow_dynamic_smem((const void *)k_lane_merge, smem);
    if (e != cudaSuccess) return e;
  }
  return launch_pdl(k_lane_merge, dim3((unsigned)B), dim3(kMergeThreads), smem, s, c_ids, c_sc, c_cnt, c_stride, lane_of,
                    k_of, run_ids, run_sc, run_cnt, run_stride);
}

cudaError_t launch_lane_reset(const int32_t *lanes, int n, int32_t *run_cnt, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  return launch_pdl(k_lane_reset, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, s, lanes, n, run_cnt);
}

cudaError_t launch_lane_gather(const int32_t *lanes, int n, const int32_t *run_ids, const float *run_sc,
                               const int32_t *run_cnt, int run_stride, int k_stride, int32_t *out_ids, float *out_sc,
                               int32_t *out_cnt, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  return launch_pdl(k_lane_gather, dim3((unsigned)n), dim3(kMergeThreads), 0, s, lanes, run_ids, run_sc, run_cnt,
                    run_stride, k_stride, out_ids, out_sc, out_cnt);
}

}  // namespace lr

using namespace lr;

namespace {
bool merge_dev_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}
}  // namespace

extern "C" lr_status lr_merge_topk(const int32_t *ids, const float *scores, const int32_t *counts, int32_t G,
                                   int32_t B, int32_t k_in, int32_t k, int32_t *out_ids, float *out_scores,
                                   int32_t *out_count, void *stream) {
  if (!ids || !scores || !counts || !out_ids || !out_scores) return fail(LR_ERR_INVALID, "lr_merge_topk: null pointer");
  if (G < 1 || G > kMergeMaxG) return fail(LR_ERR_INVALID, "lr_merge_topk: G must be in [1, 64]");
  if (B < 1 || k_in < 1) return fail(LR_ERR_INVALID, "lr_merge_topk: B and k_in must be >= 1");
  if (k < 1 || k > kMaxK || (int64_t)k > (int64_t)G * k_in)
    return fail(LR_ERR_INVALID, "lr_merge_topk: k must be in [1, min(4096, G * k_in)]");
  if (!merge_dev_ptr(ids) || !merge_dev_ptr(scores) || !merge_dev_ptr(counts) || !merge_dev_ptr(out_ids) ||
      !merge_dev_ptr(out_scores) || (out_count && !merge_dev_ptr(out_count)))
    return fail(LR_ERR_INVALID, "lr_merge_topk: every array must be device memory");
  const cudaError_t e =
      launch_merge_topk(ids, scores, counts, G, B, k_in, k, out_ids, out_scores, out_count, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "lr_merge_topk");
  return LR_OK;
}
