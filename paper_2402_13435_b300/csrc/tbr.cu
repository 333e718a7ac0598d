// TBR-first plan (Sec. 5.3, "EBR first or TBR first" and "F-TBR vs H-TBR"):
// when a query's term constraint is selective, its candidates come from the
// inverted index instead of a scan of every row.  The host picks, per query,
// the clause whose posting lists are shortest (the "smaller set" of the
// paper's intersection argument); every posting of that clause is a candidate
// row, kept when no earlier term of the clause already produced it and when
// the row satisfies the whole CNF (bit tests on the term bitmaps).  The kept
// rows form the query's messenger list (appendix "Message Passing between
// Layers"); EBR then scores exactly those rows (k_sign_rescore's warp-per-row
// FP32 dot products) and the library's exact selection returns the top K.
#include "lr_internal.h"

namespace lr {
namespace {

constexpr int kTbrThreads = 256;
constexpr int kTbrMaxRanges = 16;

__device__ __forceinline__ bool has_bit(const uint32_t *bm, uint32_t j) { return (__ldg(bm + (j >> 5)) >> (j & 31)) & 1u; }

__global__ void __launch_bounds__(kTbrThreads) k_tbr_collect(const TbrArgs a) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
  __shared__ int64_t pre[kTbrMaxRanges + 1];
  __shared__ int64_t beg[kTbrMaxRanges];
  __shared__ const uint32_t *bms[kTbrMaxRanges];
  const int ql = blockIdx.y, q = a.q_base + ql, lane = threadIdx.x & 31;
  const int r0 = a.r_off[q], nr = a.r_off[q + 1] - r0;
  if (nr <= 0 || nr > kTbrMaxRanges) return;
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int r = 0; r < nr; ++r) {
      pre[r] = t;
      beg[r] = a.ranges[r0 + r].begin;
      bms[r] = a.ranges[r0 + r].bm;
      t += a.ranges[r0 + r].end - a.ranges[r0 + r].begin;
    }
    pre[nr] = t;
  }
  __syncthreads();
  const int64_t T = pre[nr];
  const int c0 = a.qc_off[ql], c1 = a.qc_off[ql + 1];
  unsigned long long kept = 0;
  for (int64_t p0 = (int64_t)blockIdx.x * blockDim.x; p0 < T; p0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = p0 + threadIdx.x;  // whole warps every trip
    bool take = false;
    uint32_t j = 0;
    if (p < T) {
      int r = 0;
      while (r + 1 < nr && pre[r + 1] <= p) ++r;
      j = __ldg(a.post_ids + beg[r] + (p - pre[r]));
      take = j < (uint32_t)a.n;
      for (int e = 0; e < r && take; ++e) take = !has_bit(bms[e], j);  // an earlier term of the clause has it
      for (int c = c0; c < c1 && take; ++c) {
        bool any = false;
        for (int t = a.cl_off[c]; t < a.cl_off[c + 1] && !any; ++t) any = has_bit(a.slot_bm[a.cl_slot[t]], j);
        take = any;
      }
    }
    const unsigned m = __ballot_sync(0xFFFFFFFFu, take);
    if (m == 0u) continue;
    const int lead = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == lead) base = atomicAdd(&a.cnt[q], (uint32_t)__popc(m));
    base = __shfl_sync(0xFFFFFFFFu, base, lead);
    const uint32_t pos = base + (uint32_t)__popc(m & ((1u << lane) - 1u));
    if (take) {
      if (pos < (uint32_t)a.cap)
        a.buf[(size_t)q * a.cap + pos] = (uint64_t)j;
      else
        atomicOr(a.err, 64u);  // the planner bounds the list by the clause's postings: unreachable
    }
    kept += take ? 1ull : 0ull;
  }
  for (int off = 16; off >= 1; off >>= 1) kept += __shfl_xor_sync(0xFFFFFFFFu, kept, off);
  if (lane == 0 && kept) atomicAdd(&a.pass_cnt[q], kept);
}

}  // namespace

cudaError_t launch_tbr_collect(const TbrArgs &a, int num_sms, int64_t max_postings, cudaStream_t s) {
  if (a.nq <= 0) return cudaSuccess;
  int64_t gx = (max_postings + kTbrThreads - 1) / kTbrThreads;
  const int64_t cap_x = (4 * (int64_t)num_sms + a.nq - 1) / a.nq;
  if (gx > cap_x) gx = cap_x;
  if (gx < 1) gx = 1;
  return launch_pdl(k_tbr_collect, dim3((unsigned)gx, (unsigned)a.nq), dim3(kTbrThreads), 0, s, a);
}

}  // namespace lr
