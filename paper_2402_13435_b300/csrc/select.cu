// Per-query selection over candidate buffers (appendix "Fast Top K Selection").
//
// The paper selects with a score-bucket histogram that needs known score bounds.
// Here every candidate is a distinct 64-bit key (ordered score, ~job id), so an
// exact radix selection needs no bounds: 8 passes of an 8-bit digit histogram
// in shared memory find the r-th largest key; the keys at or above it are then
// gathered and sorted by a bitonic network in shared memory.
//
//   mode 0 (threshold): tau[q] = r-th largest key of the sample buffer, or 0
//                       when the sample holds fewer than r keys.
//   mode 1 (final):     top min(K, #passing) keys of the candidate buffer,
//                       written as (id, score) rows; a query whose buffer cannot
//                       prove it holds the top K (overflow, or fewer than K
//                       candidates above a non-zero threshold) is flagged for the
//                       exact fallback instead.
#include "lr_internal.h"

namespace lr {
namespace {

constexpr int kSelThreads = 512;
constexpr int kSmemKeys = 8192;  // candidate keys staged in shared memory when they fit

constexpr uint32_t kFew = 32;  // a bin this small is finished by one warp

struct SelShared {
  uint32_t hist[256];
  uint32_t digit;
  uint32_t krem;
  uint32_t bin;  // keys in the chosen bin
  uint32_t n_out;
  uint32_t n_few;
  uint64_t result;
  uint64_t few[kFew];
};

// r-th largest (1-based) of n distinct keys; keys may be in shared or global memory.
// Radix select on 8-bit digits from the top; as soon as the bin that holds the
// r-th largest key has at most kFew keys, those keys are gathered and one warp
// finds the one with exactly krem - 1 of them above it, instead of running the
// remaining digit passes.
__device__ uint64_t block_kth(const uint64_t *keys, int64_t n, uint32_t r, SelShared &sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint64_t prefix = 0;
  uint32_t krem = r;
  for (int shift = 56; shift >= 0; shift -= 8) {
    const int top = shift + 8;
    for (int i = tid; i < 256; i += blockDim.x) sh.hist[i] = 0u;
    __syncthreads();
    for (int64_t i = tid; i < n; i += blockDim.x) {
      const uint64_t key = keys[i];
      if (top >= 64 || (key >> top) == (prefix >> top)) atomicAdd(&sh.hist[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (warp == 0) {
      uint32_t c[8], cs = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) { c[j] = sh.hist[255 - 8 * lane - j]; cs += c[j]; }
      uint32_t incl = cs;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, off);
        if (lane >= off) incl += t;
      }
      const uint32_t excl = incl - cs;
      const unsigned hit = __ballot_sync(0xFFFFFFFFu, excl < krem && krem <= incl);
      if (hit == 0u) {
        if (lane == 0) { sh.digit = 0u; sh.krem = 1u; sh.bin = 0xFFFFFFFFu; }  // unreachable for r <= n
      } else if (lane == __ffs(hit) - 1) {
        uint32_t cum = excl, bin = c[7];
        int d = 255 - 8 * lane - 7;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (cum + c[j] >= krem) { d = 255 - 8 * lane - j; bin = c[j]; break; }
          cum += c[j];
        }
        sh.digit = (uint32_t)d;
        sh.krem = krem - cum;
        sh.bin = bin;
      }
    }
    __syncthreads();
    prefix |= (uint64_t)sh.digit << shift;
    krem = sh.krem;
    const uint32_t bin = sh.bin;
    __syncthreads();
    if (shift > 0 && bin <= kFew) {  // the rest is decided inside one small bin
      if (tid == 0) {
        sh.n_few = 0u;
        sh.result = prefix;
      }
      __syncthreads();
      for (int64_t i = tid; i < n; i += blockDim.x) {
        const uint64_t key = keys[i];
        if ((key >> shift) == (prefix >> shift)) {
          const uint32_t pos = atomicAdd(&sh.n_few, 1u);
          if (pos < kFew) sh.few[pos] = key;
        }
      }
      __syncthreads();
      if (warp == 0) {
        const uint32_t m = sh.n_few < kFew ? sh.n_few : kFew;
        const uint64_t v = (uint32_t)lane < m ? sh.few[lane] : 0ull;
        uint32_t above = 0;
        for (uint32_t j = 0; j < m; ++j) above += __shfl_sync(0xFFFFFFFFu, v, (int)j) > v ? 1u : 0u;
        if ((uint32_t)lane < m && above == krem - 1u) sh.result = v;
      }
      __syncthreads();
      return sh.result;
    }
  }
  return prefix;
}

// Append `key` at dst[*cnt] (stored while below cap) when `take`: the taking
// lanes of a warp claim their places with one shared atomic.  Called by whole,
// converged warps.
__device__ __forceinline__ void warp_append(bool take, uint64_t key, uint64_t *dst, uint32_t cap, uint32_t *cnt) {
  const unsigned m = __ballot_sync(0xFFFFFFFFu, take);
  if (m == 0u) return;
  const int lane = threadIdx.x & 31, lead = __ffs(m) - 1;
  uint32_t base = 0;
  if (lane == lead) base = atomicAdd(cnt, (uint32_t)__popc(m));
  base = __shfl_sync(0xFFFFFFFFu, base, lead);
  if (take) {
    const uint32_t pos = base + (uint32_t)__popc(m & ((1u << lane) - 1u));
    if (pos < cap) dst[pos] = key;
  }
}

constexpr int kPilot = 4096;  // keys of the strided pilot sample (kPilot <= kSmemKeys)

// r-th largest of n > kSmemKeys distinct keys in global memory.  The r-th largest
// key of a strided pilot of kPilot keys, taken with a margin of three standard
// deviations, gives a bound t0 that usually has between r and kSmemKeys keys at
// or above it; those keys are gathered into shared memory (one coalesced pass)
// and selected there.  When the gathered count misses that window the radix
// passes run over global memory, so the result is exact either way.
__device__ uint64_t kth_large(const uint64_t *g, int64_t n, uint32_t r, uint64_t *sbuf, SelShared &sh) {
  const int tid = threadIdx.x;
  constexpr int kPu = kPilot / kSelThreads;  // pilot loads per thread, all in flight together
  static_assert(kPilot % kSelThreads == 0, "pilot split");
  uint64_t pv[kPu];
#pragma unroll
  for (int u = 0; u < kPu; ++u) pv[u] = __ldcg(g + (int64_t)(tid + u * kSelThreads) * n / kPilot);
#pragma unroll
  for (int u = 0; u < kPu; ++u) sbuf[tid + u * kSelThreads] = pv[u];
  __syncthreads();
  const double e = (double)r * (double)kPilot / (double)n;
  double want = ceil(e + 3.0 * sqrt(e) + 8.0);
  const uint32_t rp = want > (double)kPilot ? (uint32_t)kPilot : (uint32_t)want;
  const uint64_t t0 = block_kth(sbuf, kPilot, rp, sh);
  if (tid == 0) sh.n_out = 0u;
  __syncthreads();
  constexpr int kU = 16;  // loads in flight per thread (64 KB per CTA)
  for (int64_t b0 = 0; b0 < n; b0 += (int64_t)kU * blockDim.x) {  // whole warps every trip
    const int64_t b = b0 + tid;
    uint64_t v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = b + (int64_t)u * blockDim.x;
      v[u] = i < n ? __ldcg(g + i) : 0ull;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u)
      warp_append(b + (int64_t)u * blockDim.x < n && v[u] >= t0, v[u], sbuf, (uint32_t)kSmemKeys, &sh.n_out);
  }
  __syncthreads();
  const uint32_t c = sh.n_out;
  __syncthreads();
  if (c >= r && c <= (uint32_t)kSmemKeys) return block_kth(sbuf, c, r, sh);
  return block_kth(g, n, r, sh);
}

__device__ void bitonic_desc(uint64_t *s, int P) {
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
        const int pos = 2 * i - (i & (stride - 1));
        const int par = pos + stride;
        const bool desc = (pos & size) == 0;
        const uint64_t x = s[pos], y = s[par];
        if ((x < y) == desc) { s[pos] = y; s[par] = x; }
      }
      __syncthreads();
    }
  }
}

// Compare-exchange of the key at index i (this lane) with the one `st` lanes
// away, inside bitonic merge step `size`; st < 32.
__device__ __forceinline__ void cx_lanes(uint64_t &e, int i, int st, int size, int lane) {
  const uint64_t y = __shfl_xor_sync(0xFFFFFFFFu, e, st);
  const bool keep_max = ((lane & st) == 0) == ((i & size) == 0);
  e = keep_max ? (e > y ? e : y) : (e < y ? e : y);
}

// Strides min(size/2, 32) .. 1 of bitonic merge step `size` on one 64-key chunk
// held by a warp: lane l holds the keys at indices i0 = base + l and i0 + 32.
__device__ __forceinline__ void merge_in_warp(uint64_t &e0, uint64_t &e1, int i0, int size, int lane) {
  int st = size / 2;
  if (size >= 64) {
    const bool desc = (i0 & size) == 0;
    const uint64_t hi = e0 > e1 ? e0 : e1, lo = e0 > e1 ? e1 : e0;
    e0 = desc ? hi : lo;
    e1 = desc ? lo : hi;
    st = 16;
  }
  for (; st > 0; st >>= 1) {
    cx_lanes(e0, i0, st, size, lane);
    cx_lanes(e1, i0 + 32, st, size, lane);
  }
}

// Descending bitonic sort of s[0, P), P a power of two of at least 64.  Merge
// strides of 64 and more go through shared memory with one barrier each; the
// strides below run in registers, one warp per 64-key chunk, so a sort of P
// keys takes log2(P / 64) (log2(P / 64) + 1) / 2 + log2(P / 32) barriers.
__device__ void bitonic_desc_chunks(uint64_t *s, int P) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int chunks = P / 64;
  for (int ch = warp; ch < chunks; ch += nw) {
    const int i0 = ch * 64 + lane;
    uint64_t e0 = s[i0], e1 = s[i0 + 32];
    for (int size = 2; size <= 64; size <<= 1) merge_in_warp(e0, e1, i0, size, lane);
    s[i0] = e0;
    s[i0 + 32] = e1;
  }
  __syncthreads();
  for (int size = 128; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride >= 64; stride >>= 1) {
      for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
        const int pos = 2 * i - (i & (stride - 1));
        const int par = pos + stride;
        const bool desc = (pos & size) == 0;
        const uint64_t x = s[pos], y = s[par];
        if ((x < y) == desc) { s[pos] = y; s[par] = x; }
      }
      __syncthreads();
    }
    for (int ch = warp; ch < chunks; ch += nw) {
      const int i0 = ch * 64 + lane;
      uint64_t e0 = s[i0], e1 = s[i0 + 32];
      merge_in_warp(e0, e1, i0, size, lane);
      s[i0] = e0;
      s[i0 + 32] = e1;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kSelThreads) k_select(const SelectArgs a) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
  const int q = blockIdx.x;
  if (a.any != nullptr && *reinterpret_cast<const volatile uint32_t *>(a.any) == 0u) return;
  if (a.only != nullptr && a.only[q] == 0u) return;
  extern __shared__ __align__(16) uint64_t sbuf[];  // [kSmemKeys] keys, then [kMaxK] sort area
  __shared__ SelShared sh;
  const int tid = threadIdx.x;
  const uint32_t cnt = a.cnt[q];
  const bool ovf = a.overflow[q] != 0u;
  const int64_t n = (int64_t)cnt < a.cap ? (int64_t)cnt : a.cap;
  const uint64_t *gkeys = a.buf + (size_t)q * (size_t)a.cap;

  const uint64_t *keys = gkeys;
  if (n <= kSmemKeys) {
    for (int64_t i = tid; i < n; i += blockDim.x) sbuf[i] = __ldcg(gkeys + i);
    __syncthreads();
    keys = sbuf;
  }

  if (a.mode == 0) {
    const int32_t r = a.rank[q];
    uint64_t t = 0;
    if (r > 0 && !ovf && n >= r)
      t = n <= kSmemKeys ? block_kth(keys, n, (uint32_t)r, sh) : kth_large(gkeys, n, (uint32_t)r, sbuf, sh);
    if (tid == 0) a.tau[q] = t;
    return;
  }

  const int32_t K = a.k[q];
  const unsigned long long P = a.pass_cnt[q];
  const int32_t kp = (int32_t)((unsigned long long)K < P ? (unsigned long long)K : P);
  const bool exact = !ovf && (n >= K || (unsigned long long)n == P);
  int32_t *ids = a.out_ids + (size_t)q * (size_t)a.k_stride;
  float *sc = a.out_scores + (size_t)q * (size_t)a.k_stride;
  if (a.fallback_round == 0 && (!exact || a.force_flag)) {
    if (tid == 0) {  // hand the query to the exact fallback: no digit fixed, rank min(K, P), empty list
      a.flag[q] = 1u;
      a.fb_prefix[q] = 0ull;
      a.fb_krem[q] = kp;
      a.cnt[q] = 0u;
      a.overflow[q] = 0u;
      atomicAdd(a.n_flagged, 1u);
    }
    return;
  }
  if (!exact) {  // the exact fallback always gathers exactly min(K, #passing) keys
    if (tid == 0) atomicOr(a.err, 2u);
    return;
  }
  uint64_t *sort = sbuf + kSmemKeys;
  int P2 = 1;
  while (P2 < kp) P2 <<= 1;
  if (kp > 0) {
    const uint64_t kth =
        n <= kSmemKeys ? block_kth(keys, n, (uint32_t)kp, sh) : kth_large(gkeys, n, (uint32_t)kp, sbuf, sh);
    if (tid == 0) sh.n_out = 0u;
    for (int i = tid; i < P2; i += blockDim.x) sort[i] = 0ull;
    __syncthreads();
    for (int64_t b = 0; b < n; b += blockDim.x) {  // whole warps every trip
      const int64_t i = b + tid;
      const uint64_t key = i < n ? keys[i] : 0ull;
      warp_append(i < n && key >= kth, key, sort, (uint32_t)P2, &sh.n_out);
    }
    __syncthreads();
    if (!a.unsorted) {
      if (P2 >= 64)
        bitonic_desc_chunks(sort, P2);
      else
        bitonic_desc(sort, P2);
    }
  }
  for (int i = tid; i < a.k_stride; i += blockDim.x) {
    if (i < kp) {
      const uint64_t key = sort[i];
      ids[i] = (int32_t)((int64_t)key_id(key) + a.id_base);
      sc[i] = key_score((uint32_t)(key >> 32));
    } else {
      ids[i] = -1;
      sc[i] = -INFINITY;
    }
  }
  if (tid == 0) {
    if (a.out_count) a.out_count[q] = kp;
    if (a.cand_count_out) a.cand_count_out[q] = (int32_t)cnt;
    if (a.fallback_out) a.fallback_out[q] = a.fallback_round;
  }
}

// ---------------------------------------------------------------- threshold
// Threshold of a query's sample (mode 0 of the selection, split over CTAs):
// a large sample is cut into P <= kThrSlices slices of at most kSmemKeys keys;
// CTA (q, p) finds the top r keys of its slice (the r-th largest key of the
// whole sample is among the union of the slices' top r), and the last CTA of
// the query selects the r-th largest of that union.  Samples that fit one
// slice, or whose union would not fit shared memory, take one CTA.
constexpr int kThrSlices = 32;
static_assert(kSmemKeys == kThrScratchKeys, "scratch per query = shared-memory key capacity");

__global__ void __launch_bounds__(kSelThreads) k_threshold(const ThrArgs a) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
  extern __shared__ __align__(16) uint64_t sbuf[];  // [kSmemKeys] keys
  __shared__ SelShared sh;
  __shared__ bool s_last;
  __shared__ uint32_t s_off[kThrSlices + 1];
  const int q = blockIdx.x, p = blockIdx.y, tid = threadIdx.x;
  const int64_t n = (int64_t)a.cnt[q] < a.cap ? (int64_t)a.cnt[q] : a.cap;
  const int32_t r = a.rank[q];
  if (r <= 0 || a.overflow[q] != 0u || n < r) {
    if (p == 0 && tid == 0) a.tau[q] = 0ull;
    return;
  }
  const uint64_t *g = a.buf + (size_t)q * (size_t)a.cap;
  const int64_t P64 = (n + kSmemKeys - 1) / kSmemKeys;
  const int P = (int)(P64 < kThrSlices ? P64 : kThrSlices);
  if (P == 1 || (int64_t)P * r > kSmemKeys || P64 > kThrSlices) {  // one CTA takes the whole sample
    if (p != 0) return;
    uint64_t t;
    if (n <= kSmemKeys) {
      for (int64_t i = tid; i < n; i += blockDim.x) sbuf[i] = __ldcg(g + i);
      __syncthreads();
      t = block_kth(sbuf, n, (uint32_t)r, sh);
    } else {
      t = kth_large(g, n, (uint32_t)r, sbuf, sh);
    }
    if (tid == 0) a.tau[q] = t;
    return;
  }
  if (p >= P) return;
  const int64_t per = (n + P - 1) / P, lo = (int64_t)p * per, hi = lo + per < n ? lo + per : n;
  const int64_t m = hi > lo ? hi - lo : 0;
  constexpr int kU = 16;  // loads in flight per thread
  for (int64_t b = tid; b < m; b += (int64_t)kU * blockDim.x) {
    uint64_t v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = b + (int64_t)u * blockDim.x;
      v[u] = i < m ? __ldcg(g + lo + i) : 0ull;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = b + (int64_t)u * blockDim.x;
      if (i < m) sbuf[i] = v[u];
    }
  }
  __syncthreads();
  uint64_t *out = a.scratch + (size_t)q * kSmemKeys + (size_t)p * (size_t)r;  // r places for this slice
  uint32_t kept;
  if (m <= r) {
    for (int64_t i = tid; i < m; i += blockDim.x) out[i] = sbuf[i];
    kept = (uint32_t)m;
  } else {
    const uint64_t kth = block_kth(sbuf, m, (uint32_t)r, sh);
    if (tid == 0) sh.n_out = 0u;
    __syncthreads();
    for (int64_t b = 0; b < m; b += blockDim.x) {  // exactly r keys (keys are distinct)
      const int64_t i = b + tid;
      const uint64_t key = i < m ? sbuf[i] : 0ull;
      warp_append(i < m && key >= kth, key, out, (uint32_t)r, &sh.n_out);
    }
    kept = (uint32_t)r;
  }
  if (tid == 0) a.slice_n[(size_t)q * kThrSlices + p] = kept;
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(&a.done[q], 1u) == (uint32_t)(P - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (tid == 0) {  // the union of the slices' top keys, gathered in slice order
    uint32_t off = 0;
    for (int pp = 0; pp < P; ++pp) {
      s_off[pp] = off;
      off += __ldcg(a.slice_n + (size_t)q * kThrSlices + pp);
    }
    s_off[P] = off;
  }
  __syncthreads();
  const uint64_t *src = a.scratch + (size_t)q * kSmemKeys;
  for (int pp = 0; pp < P; ++pp) {
    const uint32_t kn = s_off[pp + 1] - s_off[pp];
    for (uint32_t i = tid; i < kn; i += blockDim.x) sbuf[s_off[pp] + i] = __ldcg(src + (size_t)pp * r + i);
  }
  __syncthreads();
  const uint64_t t = block_kth(sbuf, s_off[P], (uint32_t)r, sh);
  if (tid == 0) {
    a.tau[q] = t;
    a.done[q] = 0u;  // ready for the next launch
  }
}

// ---------------------------------------------------------------- rescore
// Precision form: the low-precision scan has gathered each query's top c
// candidates (c = oversample x K, by the scaled BF16/FP8 score).  Here every
// candidate is rescored in FP32 from the FP32 copy of its row, and the top K
// are kept by (FP32 score desc, id asc).  Candidates whose FP32 score lies
// within w of the K-th FP32 score s_K are re-ranked by an FP64 dot product:
//   w = max(1e-5 max(|s_K|, 1e-6), 2 g),  g = (d + 8) 2^-24 max_j sum_k |q_k x_jk|
// g bounds the FP32 rounding error of any candidate's dot product, so every
// candidate above the band truly outscores every candidate below it, and only
// the order inside the band needs more precision.  Band members' FP64 scores
// are reported rounded to FP32 (capped by the last score above the band so the
// reported scores stay non-increasing).
constexpr int kRsThreads = 512;
constexpr int kMaxTie = 1024;
constexpr int kRsSplit = 8;  // scoring CTAs per query
constexpr int kRsRows = 4;   // candidates a warp scores at once (their rows in flight together)

// FP32 dot product p = q.x and bound m = sum_k |q_k x_k| of every candidate:
// CTA (q, s) takes candidates s * 16 + w (warp w) in steps of kRsSplit * 16
// warps, kRsRows at a time; lane-strided partial sums, tree reductions.
__global__ void __launch_bounds__(kRsThreads) k_rescore_scores(const RescoreArgs a) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
  const int q = blockIdx.x, sl = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n = a.ccnt[q] < a.c_stride ? a.ccnt[q] : a.c_stride;
  const int32_t *cid = a.cid + (size_t)q * a.c_stride;
  const float *qv = a.Q + (size_t)q * a.d_pad;
  const int step = kRsSplit * nw * kRsRows;
  uint32_t mx = 0u;
  for (int i0 = (sl * nw + warp) * kRsRows; i0 < n; i0 += step) {
    int32_t id[kRsRows];
    float p[kRsRows], m[kRsRows];
#pragma unroll
    for (int u = 0; u < kRsRows; ++u) {
      id[u] = i0 + u < n ? cid[i0 + u] : -1;
      p[u] = 0.f;
      m[u] = 0.f;
    }
    for (int k = lane; k < a.d_pad; k += 32) {
      const float v = qv[k];
      float xv[kRsRows];
#pragma unroll
      for (int u = 0; u < kRsRows; ++u) xv[u] = id[u] >= 0 ? a.X[(size_t)id[u] * a.d_pad + k] : 0.f;
#pragma unroll
      for (int u = 0; u < kRsRows; ++u) {
        p[u] = fmaf(v, xv[u], p[u]);
        m[u] = fmaf(fabsf(v), fabsf(xv[u]), m[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < kRsRows; ++u) {
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) {
        p[u] += __shfl_xor_sync(0xFFFFFFFFu, p[u], off);
        m[u] += __shfl_xor_sync(0xFFFFFFFFu, m[u], off);
      }
      if (id[u] >= 0) {
        if (lane == 0) a.keys[(size_t)q * a.c_stride + i0 + u] = make_key(p[u], (uint32_t)id[u]);
        mx = max(mx, __float_as_uint(m[u]));  // non-negative floats order as their bits
      }
    }
  }
  if (lane == 0 && mx != 0u) atomicMax(a.gmax + q, mx);
}


struct TieShared {
  double s[kMaxTie];
  int32_t id[kMaxTie];
  uint32_t n_tie, n_above, gmax_bits;
};

__global__ void __launch_bounds__(kRsThreads) k_rescore(const RescoreArgs a) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
  const int q = blockIdx.x;
  extern __shared__ __align__(16) uint64_t sbuf[];  // [kMaxK] FP32 keys, then [kMaxK] sort area
  __shared__ SelShared sh;
  __shared__ TieShared ts;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int n = a.ccnt[q] < a.c_stride ? a.ccnt[q] : a.c_stride;
  const int K = a.k[q] < n ? a.k[q] : n;
  const float *qv = a.Q + (size_t)q * a.d_pad;
  uint64_t *keys = sbuf;
  uint64_t *sortb = sbuf + kMaxK;
  int32_t *ids = a.out_ids + (size_t)q * a.k_stride;
  float *sc = a.out_scores + (size_t)q * a.k_stride;
  if (tid == 0) {
    ts.n_tie = 0u;
    ts.n_above = 0u;
    ts.gmax_bits = 0u;
  }
  __syncthreads();
  // 1. the candidates' FP32 keys, computed by the scoring launch
  for (int i = tid; i < n; i += blockDim.x) keys[i] = __ldcg(a.keys + (size_t)q * a.c_stride + i);
  if (tid == 0) ts.gmax_bits = __ldcg(a.gmax + q);
  __syncthreads();
  int n_tie = 0, n_above = 0;
  float s_above_last = INFINITY;
  if (K > 0) {
    // 2. the K-th FP32 key and the near-tie band around it
    const uint64_t kth = block_kth(keys, n, (uint32_t)K, sh);
    const float sK = key_score((uint32_t)(kth >> 32));
    const float g = (float)(a.dim + 8) * 5.9604645e-8f * __uint_as_float(ts.gmax_bits) * 1.0001f;
    const float w = fmaxf(1e-5f * fmaxf(fabsf(sK), 1e-6f), 2.f * g);
    for (int i = tid; i < n; i += blockDim.x) {
      const float si = key_score((uint32_t)(keys[i] >> 32));
      if (si > sK + w) {
        const uint32_t pos = atomicAdd(&ts.n_above, 1u);
        if (pos < (uint32_t)kMaxK) sortb[pos] = keys[i];
      } else if (si >= sK - w) {
        const uint32_t t = atomicAdd(&ts.n_tie, 1u);
        if (t < (uint32_t)kMaxTie) ts.id[t] = (int32_t)key_id(keys[i]);
      }
    }
    __syncthreads();
    n_above = (int)ts.n_above;
    const int ties_all = (int)ts.n_tie;
    n_tie = ties_all < kMaxTie ? ties_all : kMaxTie;
    // 3. candidates above the band: FP32 order
    int P2 = 1;
    while (P2 < n_above) P2 <<= 1;
    for (int i = n_above + tid; i < P2; i += blockDim.x) sortb[i] = 0ull;
    __syncthreads();
    if (n_above > 1) {
      if (P2 >= 64)
        bitonic_desc_chunks(sortb, P2);
      else
        bitonic_desc(sortb, P2);
    }
    for (int i = tid; i < n_above; i += blockDim.x) {
      ids[i] = (int32_t)((int64_t)key_id(sortb[i]) + a.id_base);
      sc[i] = key_score((uint32_t)(sortb[i] >> 32));
    }
    if (n_above > 0) s_above_last = key_score((uint32_t)(sortb[n_above - 1] >> 32));
    // 4. the band: FP64 dot products, then (score desc, id asc)
    if (ties_all > kMaxTie && tid == 0) atomicOr(a.err, 32u);  // band larger than the FP64 re-rank holds
    for (int t = warp; t < n_tie; t += nw) {
      const float *x = a.X + (size_t)ts.id[t] * a.d_pad;
      double p = 0.0;
      for (int k = lane; k < a.d_pad; k += 32) p = fma((double)qv[k], (double)x[k], p);
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) p += __shfl_xor_sync(0xFFFFFFFFu, p, off);
      if (lane == 0) ts.s[t] = p;
    }
    int T2 = 1;
    while (T2 < n_tie) T2 <<= 1;
    for (int i = n_tie + tid; i < T2; i += blockDim.x) {
      ts.s[i] = -INFINITY;
      ts.id[i] = 0x7FFFFFFF;
    }
    __syncthreads();
    for (int size = 2; size <= T2; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int i = tid; i < T2 / 2; i += blockDim.x) {
          const int pos = 2 * i - (i & (stride - 1));
          const int par = pos + stride;
          const bool desc = (pos & size) == 0;
          const double x0 = ts.s[pos], x1 = ts.s[par];
          const int32_t i0 = ts.id[pos], i1 = ts.id[par];
          const bool first_better = x0 > x1 || (x0 == x1 && i0 < i1);
          if (first_better != desc) {
            ts.s[pos] = x1;
            ts.s[par] = x0;
            ts.id[pos] = i1;
            ts.id[par] = i0;
          }
        }
        __syncthreads();
      }
    }
    const int need = K - n_above;
    for (int i = tid; i < need; i += blockDim.x) {
      const bool have = i < n_tie;
      ids[n_above + i] = have ? (int32_t)((int64_t)ts.id[i] + a.id_base) : -1;
      sc[n_above + i] = have ? fminf((float)ts.s[i], s_above_last) : -INFINITY;
    }
  }
  for (int i = K + tid; i < a.k_stride; i += blockDim.x) {
    ids[i] = -1;
    sc[i] = -INFINITY;
  }
  if (tid == 0) {
    if (a.out_count) a.out_count[q] = K;
    if (a.tie_count) a.tie_count[q] = n_tie;
  }
}

// Fallback set-up: for flagged queries start the radix selection of the
// min(K, #passing)-th key from an empty prefix and clear the candidate buffer.
}  // namespace

cudaError_t launch_threshold(const ThrArgs &a, int B, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const size_t smem = (size_t)kSmemKeys * sizeof(uint64_t);
  cudaError_t e = allow_dynamic_smem((const void *)k_threshold, (size_t)smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_threshold, dim3((unsigned)B, (unsigned)kThrSlices), dim3(kSelThreads), smem, s, a);
}

cudaError_t launch_select(const SelectArgs &a, int B, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const size_t smem = (size_t)(kSmemKeys + kMaxK) * sizeof(uint64_t);
  cudaError_t e = allow_dynamic_smem((const void *)k_select, (size_t)smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_select, dim3((unsigned)B), dim3(kSelThreads), smem, s, a);
}

cudaError_t launch_rescore(const RescoreArgs &a, int B, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const cudaError_t e0 = launch_pdl(k_rescore_scores, dim3((unsigned)B, (unsigned)kRsSplit), dim3(kRsThreads), 0, s, a);
  if (e0 != cudaSuccess) return e0;
  const size_t smem = (size_t)2 * kMaxK * sizeof(uint64_t);
  cudaError_t e = allow_dynamic_smem((const void *)k_rescore, (size_t)smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_rescore, dim3((unsigned)B), dim3(kRsThreads), smem, s, a);
}

}  // namespace lr
