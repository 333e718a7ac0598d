// Scan for small query batches: fused term predicate (F-TBR) + FP32 scoring
// (F-EBR) + candidate gathering, one pass over the job embeddings.
//
// Sec. 5.3 ("F-TBR and F-EBR are integrated in the same program") and the
// appendix paragraphs "TBR", "EBR" ("skip rows"), "Message Passing between
// Layers" and "Batch Inference" describe the method; this kernel is a B300
// design of it:
//
//   * The index is cut into 256-row groups handed out by a global work counter.
//     For each distinct term of the launch the group's 8 bitmap words (32
//     contiguous bytes of a term-major bitmap) are prefetched into shared
//     memory, and lane q evaluates query q's CNF (AND over clauses of OR over
//     terms) word-wise.
//   * Rows nobody passes are never read from HBM ("skip rows").  Passing rows
//     are compacted into 32-row lists (the messenger: job id + mask of the
//     queries that pass it) in shared memory.
//   * Rows go straight from HBM into registers: lane l holds dimensions
//     [l d/32, (l + 1) d/32) of every row and of every query, so one row is one
//     coalesced warp-wide load (d x element bytes).  A round takes R rows
//     (R x NQ <= 32 row-query pairs); each lane forms its partial dot product of
//     every pair (a sequential FP32 FMA chain over its d/32 values), and a
//     butterfly over the lanes (offsets 16, 8, 4, 2, 1, each step halving the
//     pairs a lane carries) leaves every pair's full sum in one lane.  The
//     butterfly always combines lanes in the same order, so a pair's score does
//     not depend on which other queries or rows share the launch or the round.
//     The next round's rows are loaded while the current one is reduced.
//   * No row data sits in shared memory (only the 32-row list and the term
//     words), so many warps fit on an SM and keep rows in flight.
//   * Candidates (mode kCollect): the 64-bit key (score, ~id) of each passing
//     pair is compared with the query's threshold and appended to the query's
//     buffer when it is not below it.  Mode kHist instead histograms one 11-bit
//     digit of the keys that match the query's prefix (exact radix selection);
//     the last CTA to finish fixes the digit for every query.
#include <atomic>

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "lr_internal.h"
#include "ptx.h"
#include "scan_common.cuh"

namespace lr {
namespace {

constexpr int kChunkGroups = 2;  // groups handed out per work-counter grab
constexpr int kWarps = 8;        // warps per CTA (each runs its own pipeline)

__host__ __device__ constexpr int elem_bytes(int e) { return e == kElemF32 ? 4 : e == kElemBF16 ? 2 : 1; }

// Rows per round: R x NQ row-query pairs per lane before the butterfly.
template <int NQ>
__host__ __device__ constexpr int rows_per_round() {
  return NQ >= 8 ? 4 : 8;
}

// Per-warp shared memory: the 32-row list (job ids, then query masks) and two
// term-word tables of n_slots x 8 words (the group being evaluated and the next).
__host__ __device__ inline size_t warp_bytes(int n_slots) {
  const size_t b = 256 + (size_t)2 * (n_slots > 0 ? n_slots : 1) * 32;
  return (b + 127) / 128 * 128;
}

// V consecutive row values (E) at p as FP32 (exact: BF16 and e4m3 values are
// FP32 values); p is aligned to V x element bytes.
template <int E, int V>
__device__ __forceinline__ void load_vals(const unsigned char *p, float (&x)[V]) {
  if constexpr (E == kElemF32) {
    if constexpr (V == 1) {
      x[0] = __ldg(reinterpret_cast<const float *>(p));
    } else if constexpr (V == 2) {
      const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
      x[0] = v.x;
      x[1] = v.y;
    } else {
#pragma unroll
      for (int i = 0; i < V; i += 4) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(p) + i / 4);
        x[i] = v.x;
        x[i + 1] = v.y;
        x[i + 2] = v.z;
        x[i + 3] = v.w;
      }
    }
  } else if constexpr (E == kElemBF16) {
    if constexpr (V == 1) {
      x[0] = __uint_as_float((uint32_t)__ldg(reinterpret_cast<const unsigned short *>(p)) << 16);
    } else {
      uint32_t w[V / 2];
      if constexpr (V == 2) {
        w[0] = __ldg(reinterpret_cast<const uint32_t *>(p));
      } else if constexpr (V == 4) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
        w[0] = v.x;
        w[1] = v.y;
      } else {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
        w[0] = v.x;
        w[1] = v.y;
        w[2] = v.z;
        w[3] = v.w;
      }
#pragma unroll
      for (int i = 0; i < V / 2; ++i) {
        x[2 * i] = __uint_as_float(w[i] << 16);
        x[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
      }
    }
  } else {
    // e4m3: pairs of bytes through the FP8 -> half conversion
    uint32_t h[V > 1 ? V / 2 : 1];
    if constexpr (V == 1) {
      h[0] = (uint32_t)__ldg(reinterpret_cast<const unsigned char *>(p));
    } else if constexpr (V == 2) {
      h[0] = (uint32_t)__ldg(reinterpret_cast<const unsigned short *>(p));
    } else if constexpr (V == 4) {
      const uint32_t w = __ldg(reinterpret_cast<const uint32_t *>(p));
      h[0] = w & 0xFFFFu;
      h[1] = w >> 16;
    } else {
      const uint2 w = __ldg(reinterpret_cast<const uint2 *>(p));
      h[0] = w.x & 0xFFFFu;
      h[1] = w.x >> 16;
      h[2] = w.y & 0xFFFFu;
      h[3] = w.y >> 16;
    }
#pragma unroll
    for (int i = 0; i < (V > 1 ? V / 2 : 1); ++i) {
      const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)h[i], __NV_E4M3);
      const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&hr));
      x[2 * i] = f.x;
      if constexpr (V > 1) x[2 * i + 1] = f.y;
    }
  }
}

// Butterfly over the warp: on entry v[p] is this lane's partial sum of pair p
// (p < P, P a power of two <= 32); on return every lane holds the full sum of
// pair lane >> (5 - log2 P).  Step o halves the pairs a lane carries (the lane
// with bit o set keeps the upper half) until one is left, then plain xor
// steps finish the remaining offsets; either way lanes differing in bit 4 are
// added first, then bit 3, ..., bit 0, for every pair.
template <int P>
__device__ __forceinline__ float lane_sum(float (&v)[P], int lane) {
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int o = 16 >> s;
    const int cnt = P >> s;  // pairs carried before this step
    if (cnt > 1) {
      const int h = cnt / 2;
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int i = 0; i < h; ++i) {
        const float send = up ? v[i] : v[i + h];
        const float keep = up ? v[i + h] : v[i];
        v[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, o);
      }
    } else {
      v[0] += __shfl_xor_sync(0xFFFFFFFFu, v[0], o);
    }
  }
  return v[0];
}

// A packed CNF (scan_common.cuh) over one group's words, four terms per step:
// the step's slot ids come from one register and its loads are independent,
// while the loop itself stays rolled (fewer registers than eval_packed).
__device__ __forceinline__ void eval_packed_steps(const PackedCnf &p, const uint32_t *sw, uint32_t (&pw)[8]) {
  uint32_t cw[8];
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    pw[w] = 0xFFFFFFFFu;
    cw[w] = 0u;
  }
#pragma unroll 1
  for (int t0 = 0; t0 < p.nt; t0 += 4) {
    const uint32_t ids = t0 < 4 ? p.slot[0] : t0 < 8 ? p.slot[1] : t0 < 12 ? p.slot[2] : p.slot[3];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int t = t0 + j;
      if (t < p.nt) {
        if (t > 0 && ((p.start >> t) & 1u)) {  // term t opens the next clause
#pragma unroll
          for (int w = 0; w < 8; ++w) {
            pw[w] &= cw[w];
            cw[w] = 0u;
          }
        }
        const uint4 *src = reinterpret_cast<const uint4 *>(sw + ((ids >> (8 * j)) & 0xFFu) * 8);
        const uint4 lo = src[0], hi = src[1];
        cw[0] |= lo.x; cw[1] |= lo.y; cw[2] |= lo.z; cw[3] |= lo.w;
        cw[4] |= hi.x; cw[5] |= hi.y; cw[6] |= hi.z; cw[7] |= hi.w;
      }
    }
  }
  if (p.nt > 0)
#pragma unroll
    for (int w = 0; w < 8; ++w) pw[w] &= cw[w];
}

template <int P>
__host__ __device__ constexpr int log2_of() {
  return P >= 32 ? 5 : P >= 16 ? 4 : P >= 8 ? 3 : P >= 4 ? 2 : P >= 2 ? 1 : 0;
}

template <int DP, int NQ, int E>
__global__ void __launch_bounds__(kWarps * 32) k_scan_gemv(const ScanArgs a) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
  if (a.any_active != nullptr && *reinterpret_cast<const volatile uint32_t *>(a.any_active) == 0u) return;
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int kV = DP / 32;  // values of a row (and of a query) per lane
  constexpr int kEsz = elem_bytes(E);
  constexpr int kRowBytes = DP * kEsz;
  constexpr int kR = rows_per_round<NQ>();
  constexpr int kP = kR * NQ;  // row-query pairs per round
  constexpr int kLg = log2_of<kP>();
  static_assert(kP <= 32 && (kP & (kP - 1)) == 0, "pairs per round: a power of two up to 32");
  const unsigned char *xsrc =
      reinterpret_cast<const unsigned char *>(E == kElemF32 ? static_cast<const void *>(a.X) : a.Xq);
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  unsigned char *wbase = smem + (size_t)warp * warp_bytes(a.n_slots);
  uint32_t *mrow = reinterpret_cast<uint32_t *>(wbase);  // [32] job ids of the list
  uint32_t *mqm = mrow + 32;                             // [32] their query masks
  uint32_t *slot_tab = reinterpret_cast<uint32_t *>(wbase + 256);
  __shared__ bool s_last;

  // this lane's values of every query of the launch
  float qv[NQ][kV];
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int v = 0; v < kV; ++v)
      qv[q][v] = q < a.nq ? a.Q[(size_t)(a.q_base + q) * DP + (size_t)lane * kV + v] : 0.f;

  const int top = 64 - kFbBits * a.hist_pass;
  const int shift = top - kFbBits > 0 ? top - kFbBits : 0;
  const uint32_t dmask = (1u << (top - shift)) - 1u;
  // predicate layout: lane q evaluates query q
  const int gq = a.q_base + lane;
  const bool qlive = lane < a.nq && (a.active == nullptr || a.active[gq] != 0u);
  // One- and two-query launches (latency-bound: few rows, the per-group chain
  // sets the pace) pack the lane's CNF in registers once (up to 16 terms), so
  // each group's evaluation issues only independent shared-memory loads
  // instead of walking the clause lists in global memory, and keep the pass
  // words in registers; wider launches, bound by instruction issue, keep the
  // lists (measured: the packed form cost 8-query launches 1-7 %)
  constexpr bool kPackedEval = NQ <= 2;
  PackedCnf pcnf{};
  bool packed = false;
  if (kPackedEval && qlive) {
    pcnf = pack_cnf(a, lane);
    packed = pcnf.ok;
  }
  // scoring layout: after the butterfly this lane holds pair pidx = (row my_r
  // of the round, query my_q); of the 32 / kP lanes holding it the first reports it
  const int pidx = lane >> (5 - kLg);
  const int my_r = pidx / NQ, my_q = pidx % NQ;
  const bool rep = (lane & ((1 << (5 - kLg)) - 1)) == 0;
  const int g2 = a.q_base + my_q;
  const bool my_live = my_q < a.nq && (a.active == nullptr || a.active[g2] != 0u);
  const uint64_t my_t = !my_live ? 0ull : (a.mode == kCollect ? (a.tau ? a.tau[g2] : 0ull) : a.prefix[g2]);

  const int64_t n_items = a.g_begin < a.n_groups ? (a.n_groups - a.g_begin + a.g_step - 1) / a.g_step : 0;
  int64_t item = 0, item_end = 0;
  auto next_group = [&]() -> int64_t {
    if (item + 1 < item_end) return a.g_begin + (++item) * a.g_step;
    uint32_t c = 0;
    if (lane == 0) c = atomicAdd(a.work_ctr, 1u);
    c = __shfl_sync(0xFFFFFFFFu, c, 0);
    item = (int64_t)c * kChunkGroups;
    item_end = item + kChunkGroups < n_items ? item + kChunkGroups : n_items;
    return item < n_items ? a.g_begin + item * a.g_step : -1;
  };
  auto prefetch = [&](int64_t g, int t) {
    uint32_t *dst = slot_tab + (size_t)t * a.n_slots * 8;
    for (int i = lane; i < 2 * a.n_slots; i += 32) {
      const int s = i >> 1, h = i & 1;
      cp_async16(dst + s * 8 + h * 4, a.slot_bm[s] + g * kGroupWords + h * 4);
    }
    cp_async_commit();
  };

  // score the list's first n rows: rounds of kR rows, the next round's rows
  // loaded before the current round is reduced
  auto score_rows = [&](uint32_t n) {
    float xa[kR][kV], xb[kR][kV];
    auto load = [&](uint32_t base, float(&x)[kR][kV]) {
#pragma unroll
      for (int r = 0; r < kR; ++r) {
        const uint32_t i = base + (uint32_t)r;
        if (i < n) {
          load_vals<E, kV>(xsrc + (size_t)mrow[i] * kRowBytes + (size_t)lane * (kV * kEsz), x[r]);
        } else {
#pragma unroll
          for (int v = 0; v < kV; ++v) x[r][v] = 0.f;
        }
      }
    };
    auto process = [&](uint32_t base, const float(&x)[kR][kV]) {
      float part[kP];
#pragma unroll
      for (int r = 0; r < kR; ++r)
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          float acc = 0.f;
#pragma unroll
          for (int v = 0; v < kV; ++v) acc = fmaf(x[r][v], qv[q][v], acc);
          part[r * NQ + q] = acc;
        }
      float s = lane_sum<kP>(part, lane);
      const uint32_t i = base + (uint32_t)my_r;
      const bool valid = i < n;
      const uint32_t row = valid ? mrow[i] : 0u;
      const uint32_t qm = valid ? mqm[i] : 0u;
      const bool pass = rep && ((qm >> my_q) & 1u);
      if constexpr (E == kElemFP8) s *= pass ? __ldg(a.xscale + row) : 0.f;  // per-row scale of the e4m3 row
      const uint64_t key = make_key(s, row);
      if (a.mode == kCollect) {
        // one counter reservation per warp and query
        const bool take = pass && key >= my_t;
        if (__any_sync(0xFFFFFFFFu, take)) {
          const uint32_t grp = __match_any_sync(0xFFFFFFFFu, take ? (uint32_t)my_q : 64u + (uint32_t)lane);
          const int leader = __ffs(grp) - 1;
          uint32_t pos0 = 0;
          if (take && lane == leader) pos0 = atomicAdd(&a.buf_cnt[g2], (uint32_t)__popc(grp));
          pos0 = __shfl_sync(0xFFFFFFFFu, pos0, leader);
          if (take) {
            const uint32_t p = pos0 + (uint32_t)__popc(grp & ((1u << lane) - 1u));
            if ((int64_t)p < a.buf_cap)
              a.buf[(size_t)g2 * (size_t)a.buf_cap + p] = key;
            else
              atomicOr(&a.overflow[g2], 1u);
          }
        }
      } else if (pass && (top >= 64 || (key >> top) == (my_t >> top))) {
        atomicAdd(&a.hist[(size_t)g2 * kFbBins + (uint32_t)((key >> shift) & dmask)], 1u);
      }
    };
    load(0u, xa);
    for (uint32_t b = 0; b < n; b += 2 * kR) {
      if (b + kR < n) load(b + kR, xb);
      process(b, xa);
      if (b + kR < n) {
        if (b + 2 * kR < n) load(b + 2 * kR, xa);
        process(b + kR, xb);
      }
    }
  };

  unsigned long long my_pass = 0;
  uint32_t fill = 0;  // rows in the list
  int t = 0;
  int64_t g = next_group();
  if (g >= 0) prefetch(g, 0);
  int64_t gn = g >= 0 ? next_group() : -1;
  if (gn >= 0) prefetch(gn, 1);
  else cp_async_commit();
  while (g >= 0) {
    cp_async_wait_group<1>();  // term words of g have landed
    __syncwarp();
    uint32_t pw[8];
    if (qlive) {
      if (kPackedEval && packed)
        eval_packed_steps(pcnf, slot_tab + (size_t)t * a.n_slots * 8, pw);
      else
        eval_cnf(a, lane, slot_tab + (size_t)t * a.n_slots * 8, pw);
    } else {
#pragma unroll
      for (int w = 0; w < 8; ++w) pw[w] = 0u;
    }
    __syncwarp();
    const int64_t gnn = gn >= 0 ? next_group() : -1;
    if (gnn >= 0) prefetch(gnn, t);  // the table of g is free again
    else cp_async_commit();
    const int64_t r0 = g * kGroupRows;
#pragma unroll 1
    for (int w = 0; w < 8; ++w) {
      const int64_t left = a.n - (r0 + w * 32);
      // packed form: word w is pw[0], the words shifting down one place per
      // iteration, so the array stays in registers (no indexing by the rolled
      // loop's counter)
      const uint32_t pw_w = kPackedEval ? pw[0] : pw[w];
      const uint32_t p = pw_w & (left >= 32 ? 0xFFFFFFFFu : (left > 0 ? ((1u << left) - 1u) : 0u));
      if constexpr (kPackedEval) {
#pragma unroll
        for (int i = 0; i < 7; ++i) pw[i] = pw[i + 1];
      }
      my_pass += (unsigned long long)__popc(p);
      const uint32_t U = __reduce_or_sync(0xFFFFFFFFu, p);
      if (U == 0u) continue;
      uint32_t qm = 0;  // lane r: mask of the queries that pass row r of the word
#pragma unroll
      for (int q = 0; q < NQ; ++q) qm |= ((__shfl_sync(0xFFFFFFFFu, p, q) >> lane) & 1u) << q;
      const uint32_t n = __popc(U);
      const uint32_t rank = __popc(U & ((1u << lane) - 1u));
      const int64_t wrow = r0 + w * 32;
      uint32_t done = 0;
      while (done < n) {
        const uint32_t take = (32u - fill) < (n - done) ? (32u - fill) : (n - done);
        if (((U >> lane) & 1u) && rank >= done && rank < done + take) {
          mrow[fill + rank - done] = (uint32_t)(wrow + lane);
          mqm[fill + rank - done] = qm;
        }
        __syncwarp();  // the list is visible to every lane
        fill += take;
        done += take;
        if (fill == 32u) {
          score_rows(32u);
          __syncwarp();  // every lane has read the list
          fill = 0;
        }
      }
    }
    g = gn;
    gn = gnn;
    t ^= 1;
  }
  if (fill > 0u) score_rows(fill);
  cp_async_wait_all();
  if (qlive && a.pass_cnt != nullptr) atomicAdd(&a.pass_cnt[gq], my_pass);

  // grid completion: the last CTA resets the work counter and, in kHist mode,
  // fixes this pass's digit for every participating query
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(a.done_ctr, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    if (a.mode == kHist) hist_step(a, top, shift);
    __syncthreads();
    if (threadIdx.x == 0) {
      *a.work_ctr = 0u;
      *a.done_ctr = 0u;
    }
  }
}

template <int DP, int NQ, int E>
cudaError_t launch_one(const ScanArgs &a, int grid, cudaStream_t s) {
  const size_t smem = (size_t)kWarps * warp_bytes(a.n_slots);
  if (a.n_slots > kGemvMaxSlots || smem > 220u * 1024u) return cudaErrorInvalidValue;
  auto *fn = k_scan_gemv<DP, NQ, E>;
  cudaError_t e = allow_dynamic_smem((const void *)fn, smem);
  if (e != cudaSuccess) return e;
  // CTAs an SM holds at this shared-memory size (looked up once per slot count)
  static std::atomic<int> per_sm[kGemvMaxSlots + 1];
  const int ns = a.n_slots > 0 ? a.n_slots : 0;
  int nb = per_sm[ns].load(std::memory_order_relaxed);
  if (nb <= 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kWarps * 32, smem);
    if (e != cudaSuccess) return e;
    if (nb < 1) nb = 1;
    per_sm[ns].store(nb, std::memory_order_relaxed);
  }
  // grid: the caller's CTAs per pass (at most one per SM) x CTAs per SM, no
  // more than the work counter hands out chunks to
  const int64_t n_items = a.g_begin < a.n_groups ? (a.n_groups - a.g_begin + a.g_step - 1) / a.g_step : 0;
  const int64_t want = (n_items + (int64_t)kChunkGroups * kWarps - 1) / ((int64_t)kChunkGroups * kWarps);
  int64_t total = (int64_t)grid * nb;
  if (total > want) total = want;
  if (total < 1) total = 1;
  return launch_pdl(fn, dim3((unsigned)total), dim3(kWarps * 32), smem, s, a);
}

template <int DP, int E>
cudaError_t dispatch_nq(const ScanArgs &a, int nq_tmpl, int grid, cudaStream_t s) {
  switch (nq_tmpl) {
    case 1: return launch_one<DP, 1, E>(a, grid, s);
    case 2: return launch_one<DP, 2, E>(a, grid, s);
    case 4: return launch_one<DP, 4, E>(a, grid, s);
    case 8: return launch_one<DP, 8, E>(a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int DP>
cudaError_t dispatch_elem(const ScanArgs &a, int nq_tmpl, int grid, cudaStream_t s) {
  switch (a.elem) {
    case kElemF32: return dispatch_nq<DP, kElemF32>(a, nq_tmpl, grid, s);
    case kElemBF16: return dispatch_nq<DP, kElemBF16>(a, nq_tmpl, grid, s);
    case kElemFP8: return dispatch_nq<DP, kElemFP8>(a, nq_tmpl, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_scan_gemv(const ScanArgs &a, int nq_tmpl, int vec, int grid, cudaStream_t s) {
  switch (vec) {
    case 1: return dispatch_elem<32>(a, nq_tmpl, grid, s);
    case 2: return dispatch_elem<64>(a, nq_tmpl, grid, s);
    case 4: return dispatch_elem<128>(a, nq_tmpl, grid, s);
    case 8: return dispatch_elem<256>(a, nq_tmpl, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lr
