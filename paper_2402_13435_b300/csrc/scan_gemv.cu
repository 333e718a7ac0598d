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
//     are compacted into 32-row batches (the messenger: job id + mask of the
//     queries that pass it) and fetched asynchronously.
//   * Lane i scores row i of a batch against every query of the launch: a
//     sequential FP32 FMA chain over the dimensions, row data from shared
//     memory (rows sit 16 bytes apart beyond their length, so the 32 lanes'
//     16-byte loads hit distinct banks) and query values broadcast from shared
//     memory.  A score is therefore computed the same way whatever other
//     queries share the launch.
//   * Candidates (mode kCollect): the 64-bit key (score, ~id) of each passing
//     pair is compared with the query's threshold and appended to the query's
//     buffer when it is not below it.  Mode kHist instead histograms one 11-bit
//     digit of the keys that match the query's prefix (exact radix selection);
//     the last CTA to finish fixes the digit for every query.
//
// Every mbarrier wait is bounded (ptx.h); a wait that gives up records
// LR_ERR_TIMEOUT in the error word.
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "lr_internal.h"
#include "ptx.h"
#include "scan_common.cuh"

namespace lr {
namespace {

constexpr int kChunkGroups = 2;  // groups handed out per work-counter grab

// Per-warp pipeline (every warp of the CTA runs one independently):
//   * take 256-row groups from the global work counter (chunks of kChunkGroups);
//   * term words of the next group are prefetched with cp.async while the
//     current group is processed (one commit group per prefetch);
//   * lane q evaluates query q's CNF over the group's 8 words;
//   * passing rows are packed into 32-row batches -- the paper's messenger: a
//     slot holds the job id and the bit mask of the queries that pass it -- and
//     each row is fetched by one warp-wide cp.async (16 bytes per lane, one
//     coalesced request per row) into a padded shared-memory slot;
//   * completion of a batch's copies is counted on the batch buffer's mbarrier
//     (cp.async.mbarrier.arrive.noinc from every lane), and the previous batch is
//     scored while the current one is in flight (double buffering).
struct WarpLayout {
  size_t row_stride, buf_bytes, per_warp, bars, meta, slots, rows, queries, total;
};

__host__ __device__ inline size_t w_align(size_t v, size_t a) { return (v + a - 1) / a * a; }

__host__ __device__ constexpr int elem_bytes(int e) { return e == kElemF32 ? 4 : e == kElemBF16 ? 2 : 1; }

__host__ __device__ inline WarpLayout warp_layout(int d_pad, int esz, int nq_tmpl, int n_slots, int warps) {
  WarpLayout L;
  L.row_stride = (size_t)d_pad * esz + 16;  // +16 bytes: the 32 lanes' 16-byte loads hit distinct banks
  L.buf_bytes = 32 * L.row_stride;
  // per-warp region: 2 barriers | meta (row, qmask) x 2 buffers | 2 term tables | 2 row buffers
  L.bars = 0;
  L.meta = 16;
  L.slots = w_align(L.meta + 2 * 32 * 8, 16);
  L.rows = w_align(L.slots + (size_t)2 * (n_slots > 0 ? n_slots : 1) * 32, 16);
  L.per_warp = w_align(L.rows + 2 * L.buf_bytes, 128);
  L.queries = (size_t)warps * L.per_warp;
  L.total = L.queries + (size_t)nq_tmpl * d_pad * 4;
  return L;
}

// Row element (E) values of one 16-byte chunk as FP32 (exact: BF16 and e4m3
// values are FP32 values).
template <int E>
__device__ __forceinline__ void chunk_to_f32(const uint4 &r, float (&x)[16 / elem_bytes(E)]) {
  const uint32_t w[4] = {r.x, r.y, r.z, r.w};
  if constexpr (E == kElemF32) {
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] = __uint_as_float(w[i]);
  } else if constexpr (E == kElemBF16) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      x[2 * i] = __uint_as_float(w[i] << 16);
      x[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const __half2_raw hr =
            __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)((w[i] >> (16 * h)) & 0xFFFFu), __NV_E4M3);
        const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&hr));
        x[4 * i + 2 * h] = f.x;
        x[4 * i + 2 * h + 1] = f.y;
      }
    }
  }
}

template <int DP, int NQ, int E>
__device__ __forceinline__ void score_batch(const ScanArgs &a, const unsigned char *buf, const uint32_t *meta_row,
                                            const uint32_t *meta_qm, uint32_t n, const float *qs,
                                            const uint64_t (&tq)[NQ], int lane, int top, int shift,
                                            uint32_t dmask, size_t row_stride) {
  // every lane takes part (the appends below are warp-aggregated); lanes past
  // the batch score a stale slot of the buffer and pass no query
  const bool live = (uint32_t)lane < n;
  const uint32_t row = live ? meta_row[lane] : 0u;
  const uint32_t qm = live ? meta_qm[lane] : 0u;
  constexpr int kPer = 16 / elem_bytes(E);  // values per 16-byte chunk
  const unsigned char *xr = buf + (size_t)lane * row_stride;
  float acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.f;
#pragma unroll 4
  for (int k = 0; k < DP; k += kPer) {
    float x[kPer];
    chunk_to_f32<E>(*reinterpret_cast<const uint4 *>(xr + (size_t)k * elem_bytes(E)), x);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
#pragma unroll
      for (int v4 = 0; v4 < kPer / 4; ++v4) {
        const float4 v = *reinterpret_cast<const float4 *>(qs + q * DP + k + 4 * v4);
        acc[q] = fmaf(x[4 * v4 + 0], v.x, acc[q]);
        acc[q] = fmaf(x[4 * v4 + 1], v.y, acc[q]);
        acc[q] = fmaf(x[4 * v4 + 2], v.z, acc[q]);
        acc[q] = fmaf(x[4 * v4 + 3], v.w, acc[q]);
      }
    }
  }
  if constexpr (E == kElemFP8) {  // per-row scale of the e4m3 row
    const float sc = live ? __ldg(a.xscale + row) : 0.f;
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] *= sc;
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const bool pass = (qm >> q) & 1u;
    const uint64_t key = make_key(acc[q], row);
    const int g2 = a.q_base + q;
    if (a.mode == kCollect) {
      // one counter reservation per warp and query
      const bool take = pass && key >= tq[q];
      const uint32_t want = __ballot_sync(0xFFFFFFFFu, take);
      if (want == 0u) continue;
      uint32_t base = 0;
      if (lane == __ffs(want) - 1) base = atomicAdd(&a.buf_cnt[g2], (uint32_t)__popc(want));
      base = __shfl_sync(0xFFFFFFFFu, base, __ffs(want) - 1);
      if (take) {
        const uint32_t p = base + (uint32_t)__popc(want & ((1u << lane) - 1u));
        if ((int64_t)p < a.buf_cap)
          a.buf[(size_t)g2 * (size_t)a.buf_cap + p] = key;
        else
          atomicOr(&a.overflow[g2], 1u);
      }
    } else if (pass && (top >= 64 || (key >> top) == (tq[q] >> top))) {
      atomicAdd(&a.hist[(size_t)g2 * kFbBins + (uint32_t)((key >> shift) & dmask)], 1u);
    }
  }
}

template <int DP, int NQ, int E>
__global__ void __launch_bounds__(256, 1) k_scan_gemv(const ScanArgs a) {
  if (a.any_active != nullptr && *reinterpret_cast<const volatile uint32_t *>(a.any_active) == 0u) return;
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int kRowBytes = DP * elem_bytes(E);
  constexpr int kChunks = kRowBytes / 16;  // 16-byte chunks per row
  const int warps = blockDim.x >> 5;
  const WarpLayout L = warp_layout(DP, elem_bytes(E), NQ, a.n_slots, warps);
  const unsigned char *xsrc =
      reinterpret_cast<const unsigned char *>(E == kElemF32 ? static_cast<const void *>(a.X) : a.Xq);
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  unsigned char *wbase = smem + (size_t)warp * L.per_warp;
  uint64_t *bar = reinterpret_cast<uint64_t *>(wbase + L.bars);
  uint32_t *meta = reinterpret_cast<uint32_t *>(wbase + L.meta);  // [buf][row 32 | qmask 32]
  uint32_t *slot_tab = reinterpret_cast<uint32_t *>(wbase + L.slots);
  unsigned char *rows = wbase + L.rows;
  float *qs = reinterpret_cast<float *>(smem + L.queries);
  __shared__ bool s_last;

  for (int i = threadIdx.x; i < NQ * DP; i += blockDim.x) {
    const int q = i / DP;
    qs[i] = q < a.nq ? a.Q[(size_t)(a.q_base + q) * DP + (i % DP)] : 0.f;
  }
  if (lane == 0) {
    mbar_init(&bar[0], 32);
    mbar_init(&bar[1], 32);
    fence_mbar_init();
  }
  __syncthreads();

  const int top = 64 - kFbBits * a.hist_pass;
  const int shift = top - kFbBits > 0 ? top - kFbBits : 0;
  const uint32_t dmask = (1u << (top - shift)) - 1u;
  const int gq = a.q_base + lane;
  const bool qlive = lane < a.nq && (a.active == nullptr || a.active[gq] != 0u);
  uint64_t tq[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int g2 = a.q_base + q;
    const bool live = q < a.nq && (a.active == nullptr || a.active[g2] != 0u);
    tq[q] = !live ? 0ull : (a.mode == kCollect ? (a.tau ? a.tau[g2] : 0ull) : a.prefix[g2]);
  }

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

  unsigned long long my_pass = 0;
  bool ok = true;
  int fb = 0;          // buffer being filled
  uint32_t fill = 0;   // rows placed in it
  bool prev = false;   // a closed batch waits in buffer fb ^ 1
  uint32_t prev_n = 0;
  uint32_t phase[2] = {0u, 0u};
  auto close_and_score_prev = [&]() {
    // hand the filled buffer's copies to its barrier, then score the previous batch
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar[fb])) : "memory");
    if (prev) {
      const int pb = fb ^ 1;
      if (!mbar_wait(&bar[pb], phase[pb])) ok = false;
      phase[pb] ^= 1u;
      __syncwarp();
      score_batch<DP, NQ, E>(a, rows + (size_t)pb * L.buf_bytes, meta + pb * 64, meta + pb * 64 + 32, prev_n, qs,
                             tq, lane, top, shift, dmask, L.row_stride);
      __syncwarp();
    }
    prev = true;
    prev_n = fill;
    fb ^= 1;
    fill = 0;
  };

  int t = 0;
  int64_t g = next_group();
  if (g >= 0) prefetch(g, 0);
  int64_t gn = g >= 0 ? next_group() : -1;
  if (gn >= 0) prefetch(gn, 1);
  else cp_async_commit();
  while (g >= 0 && ok) {
    cp_async_wait_group<1>();  // term words of g have landed
    __syncwarp();
    uint32_t pw[8];
    if (qlive) {
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
      uint32_t p = pw[w] & (left >= 32 ? 0xFFFFFFFFu : (left > 0 ? ((1u << left) - 1u) : 0u));
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
        uint32_t *mrow = meta + fb * 64;
        if (((U >> lane) & 1u) && rank >= done && rank < done + take) {
          mrow[fill + rank - done] = (uint32_t)(wrow + lane);
          mrow[32 + fill + rank - done] = qm;
        }
        __syncwarp();  // the slots' job ids are visible to every lane
        unsigned char *dst = rows + (size_t)fb * L.buf_bytes;
        for (uint32_t i = lane; i < take * kChunks; i += 32) {
          const uint32_t k = i / kChunks, c = i % kChunks;
          cp_async16(dst + (size_t)(fill + k) * L.row_stride + c * 16,
                     xsrc + (size_t)mrow[fill + k] * kRowBytes + (size_t)c * 16);
        }
        fill += take;
        done += take;
        if (fill == 32u) close_and_score_prev();
      }
    }
    g = gn;
    gn = gnn;
    t ^= 1;
  }
  // drain: close the partial batch, score what remains
  if (fill > 0u) close_and_score_prev();
  if (prev) {
    const int pb = fb ^ 1;
    if (!mbar_wait(&bar[pb], phase[pb])) ok = false;
    __syncwarp();
    score_batch<DP, NQ, E>(a, rows + (size_t)pb * L.buf_bytes, meta + pb * 64, meta + pb * 64 + 32, prev_n, qs, tq,
                           lane, top, shift, dmask, L.row_stride);
  }
  cp_async_wait_all();
  if (!ok && lane == 0) atomicOr(a.err, kErrTimeout);
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
  const size_t budget = 220u * 1024u;
  int warps = 8;
  while (warps > 1 && warp_layout(DP, elem_bytes(E), NQ, a.n_slots, warps).total > budget) --warps;
  const WarpLayout L = warp_layout(DP, elem_bytes(E), NQ, a.n_slots, warps);
  if (L.total > budget) return cudaErrorInvalidValue;
  auto *fn = k_scan_gemv<DP, NQ, E>;
  cudaError_t e = allow_dynamic_smem((const void *)fn, (size_t)L.total);
  if (e != cudaSuccess) return e;
  fn<<<grid, warps * 32, L.total, s>>>(a);
  return cudaGetLastError();
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
