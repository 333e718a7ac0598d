// Tensor-core scan for larger query batches: fused term predicate (F-TBR) +
// scoring (F-EBR) on tcgen05 + candidate gathering, one pass over the index.
//
// Sec. 5.3 turns each query embedding into a multiplication against the dense
// job matrix; with many queries in a batch ("Batch Inference") that product is
// a real dense contraction S = X Q^T, so it runs on the 5th-generation tensor
// cores: M = 128 jobs x N = queries x K = d per tile, accumulated in tensor
// memory.  FP32 accuracy comes from the 3xTF32 split
//     x = x_hi + x_lo,  x_hi = x with the low 13 mantissa bits cleared,
//     x.q ~= x_hi.q_hi + x_hi.q_lo + x_lo.q_hi     (x_lo.q_lo dropped, < 2^-20 |x q|)
// where x_hi and q_hi are exact in TF32; the unit truncates x_lo and q_lo to
// TF32 (11 significant bits of their 13), an error below 2^-22 |x q| per term.
//
// One CTA per SM, eleven warps with fixed roles:
//   warp 0     predicate: takes 256-row groups from the work counter (read one
//              chunk ahead), prefetches the groups' term words (cp.async),
//              evaluates every query's CNF (held in registers when it has at
//              most 16 terms) and publishes per-tile row messages (the mask of
//              the queries that pass each row); tiles nobody passes are not
//              published and never read ("skip rows").
//   warp 10    loader: issues the 2-D TMA loads (128 rows x 32 floats, 128-byte
//              swizzle) of every published tile into a ring of raw stages.
//   warp 1     owns the tensor memory and issues the MMAs from one thread.  The
//              job operand comes from tensor memory: per 8-wide K step one MMA
//              of width 2N with x_hi against [q_hi ; q_lo] and one of width N
//              with x_lo against q_hi, so accumulator columns [0, N) and
//              [N, 2N) add up to the 3xTF32 product.
//   warps 2-5  converters, one per tensor-memory lane quarter: each thread
//              reads its row of a landed chunk, releases the raw stage at once,
//              and writes x_hi and x_lo into tensor memory (tcgen05.st).  Raw
//              stages therefore never wait on the tensor core, and shared
//              memory holds little besides them.
//   warps 6-9  epilogue: read the accumulator (warp w owns lanes 32*(w%4) ..),
//              test every passing (row, query) against the query's threshold
//              without branches, and record the few candidates in a per-warp
//              shared-memory list flushed to the query buffers in bulk.
// All waits are bounded; on a timeout the error word gets LR_ERR_TIMEOUT, the
// loader lets issued copies land, the MMA warp waits for its MMAs, and the
// tensor memory is freed before the CTA exits.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "lr_internal.h"
#include "ptx.h"
#include "scan_common.cuh"

namespace lr {
namespace {

constexpr int kTcThreads = 352;
constexpr int kEpiWarp0 = 6;
constexpr int kLoadWarp = 10;
constexpr int kMetaDepth = 4;
constexpr int kTileRows = 128;
constexpr int kChunkBytes = kTileRows * 128;  // one raw stage: a 128-row tile of 128-byte rows

// Row elements per raw chunk and the bytes of a chunk's row: FP32 rows come in
// 32-float (128-byte) column blocks; BF16 in 64-value (128-byte) blocks; FP8
// e4m3 in 64-value (64-byte) blocks.
__host__ __device__ constexpr int tc_epc(int e) { return e == kElemF32 ? 32 : 64; }
__host__ __device__ constexpr int tc_row_bytes(int e) { return e == kElemFP8 ? 64 : 128; }
constexpr int kTcGroupChunk = 2;              // groups per work-counter grab
constexpr int kWarpCand = 512;                // candidates staged per epilogue warp (flushed past 256)
constexpr int kABufs = 4;                     // x_hi/x_lo chunk buffers in tensor memory
constexpr uint32_t kTmemCols = 512;           // the whole tensor memory: one CTA per SM

// Messenger of one 128-row tile: for each row, the mask of the launch's queries
// that pass it (bit q).
struct TileMeta {
  int64_t row0;
  uint32_t done;
  uint32_t pad;
  uint64_t qm[kTileRows];
};

struct TcLayout {
  int S, C, C32, N;
  size_t raw, q, meta, slots, taus, cand, ccnt, cq, bars, holder, total;
};

__host__ __device__ inline size_t tc_align(size_t v, size_t a) { return (v + a - 1) / a * a; }

__host__ __device__ inline TcLayout tc_layout(int d_pad, int epc, int N, int n_slots, int S) {
  TcLayout T;
  T.S = S;
  T.C = d_pad / epc;   // raw chunks per tile
  T.C32 = d_pad / 32;  // 32-value chunks of the query operand
  T.N = N;
  size_t off = 0;
  T.raw = off;
  off += (size_t)S * kChunkBytes;
  T.q = off;  // per chunk: 2N rows (N rows of q_hi, then N rows of q_lo), 128 bytes each
  off += (size_t)T.C32 * 2 * N * 128;
  T.meta = tc_align(off, 16);
  off = T.meta + (size_t)kMetaDepth * sizeof(TileMeta);
  T.slots = tc_align(off, 16);
  off = T.slots + (size_t)2 * (n_slots > 0 ? n_slots : 1) * 32;
  T.taus = tc_align(off, 16);
  off = T.taus + (size_t)N * 12;  // 64-bit thresholds, then their score words as floats
  T.cand = tc_align(off, 16);     // per epilogue warp: keys, then query indices (bytes)
  off = T.cand + (size_t)4 * kWarpCand * 9;
  T.ccnt = tc_align(off, 16);
  off = T.ccnt + 16;
  T.cq = off;  // per epilogue warp: per-query counts, then reserved bases, of one flush
  off = T.cq + (size_t)4 * 2 * N * 4;
  T.bars = tc_align(off, 16);
  off = T.bars + (size_t)(2 * S + 2 * kABufs + 4 + 2 * kMetaDepth + 1) * 8;
  T.holder = tc_align(off, 16);
  T.total = T.holder + 16;
  return T;
}

// 32x32 bit-matrix transpose across the warp: lane i holds row i on entry
// (bit c = column c) and column i on exit (bit r = row r).  Five stages swap
// the off-diagonal blocks of size 16, 8, 4, 2, 1.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
  const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int j = 16 >> st;
    const uint32_t m = masks[st];
    const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, j);
    x = (lane & j) ? (((y >> j) & m) | (x & ~m)) : ((x & m) | ((y & m) << j));
  }
  return x;
}

// Leader-lane wait broadcast to the warp.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, int lane) {
  bool got = true;
  if (lane == 0) got = mbar_wait(bar, parity);
  return __shfl_sync(0xFFFFFFFFu, got ? 1 : 0, 0) != 0;
}

template <int N, int E>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_scan_tc(const ScanArgs a, const __grid_constant__ CUtensorMap tmap, int S) {
  if (a.any_active != nullptr && *reinterpret_cast<const volatile uint32_t *>(a.any_active) == 0u) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem =
      smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);  // 1024-byte aligned for the swizzle atoms
  const TcLayout T = tc_layout(a.d_pad, tc_epc(E), N, a.n_slots, S);
  const int C = T.C;
  const int C32 = T.C32;
  unsigned char *raw = smem + T.raw;
  float *qop = reinterpret_cast<float *>(smem + T.q);
  TileMeta *meta = reinterpret_cast<TileMeta *>(smem + T.meta);
  uint32_t *slot_tab = reinterpret_cast<uint32_t *>(smem + T.slots);
  uint64_t *taus = reinterpret_cast<uint64_t *>(smem + T.taus);
  float *thr = reinterpret_cast<float *>(taus + N);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + T.bars);
  uint64_t *raw_full = bars, *raw_empty = bars + S;
  uint64_t *a_full = bars + 2 * S, *a_empty = a_full + kABufs;
  uint64_t *acc_full = a_empty + kABufs, *acc_empty = acc_full + 2;
  uint64_t *meta_full = acc_empty + 2, *meta_empty = meta_full + kMetaDepth;
  uint64_t *drain = meta_empty + kMetaDepth;
  uint32_t *holder = reinterpret_cast<uint32_t *>(smem + T.holder);
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const uint32_t acol0 = 4u * (uint32_t)N;  // first tensor-memory column of the x_hi/x_lo buffers
  __shared__ bool s_last;

  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&raw_full[i], 1);
      mbar_init(&raw_empty[i], 4);
    }
    for (int i = 0; i < kABufs; ++i) {
      mbar_init(&a_full[i], 4);
      mbar_init(&a_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 4);
    }
    for (int i = 0; i < kMetaDepth; ++i) {
      mbar_init(&meta_full[i], 1);
      mbar_init(&meta_empty[i], 4);
    }
    mbar_init(drain, 1);
    fence_mbar_init();
  }
  // queries of the launch in the K-major 128-byte swizzle layout, split into hi/lo
  for (int i = threadIdx.x; i < C32 * N * 32; i += blockDim.x) {
    const int c = i / (N * 32), rem = i % (N * 32), r = rem / 32, k = rem % 32;
    const float v = r < a.nq ? a.Q[(size_t)(a.q_base + r) * a.d_pad + c * 32 + k] : 0.f;
    const float h = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
    const int rl = r + N;  // row of q_lo in the combined operand
    const size_t base = (size_t)c * 2 * N * 128;
    qop[(base + (size_t)r * 128 + ((((k >> 2) ^ (r & 7)) & 7) << 4) + (k & 3) * 4) / 4] = h;
    qop[(base + (size_t)rl * 128 + ((((k >> 2) ^ (rl & 7)) & 7) << 4) + (k & 3) * 4) / 4] = v - h;
  }
  for (int q = threadIdx.x; q < N; q += blockDim.x) {
    const int g2 = a.q_base + q;
    const bool live = q < a.nq && (a.active == nullptr || a.active[g2] != 0u);
    taus[q] = !live ? 0ull : (a.mode == kCollect ? (a.tau ? a.tau[g2] : 0ull) : a.prefix[g2]);
    // score_key(s) >= h  <=>  s >= thr[q] for every non-NaN score s
    const uint32_t h = (uint32_t)(taus[q] >> 32);
    thr[q] = h <= score_key(-INFINITY) ? -INFINITY
             : h > score_key(INFINITY) ? __uint_as_float(0x7FFFFFFFu)  // NaN: no score passes
                                       : key_score(h);
  }
  fence_proxy_async();
  if (warp == 1) {
    tmem_alloc(holder, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *holder;

  const int top = 64 - kFbBits * a.hist_pass;
  const int shift = top - kFbBits > 0 ? top - kFbBits : 0;
  const uint32_t dmask = (1u << (top - shift)) - 1u;
  bool ok = true;

  if (warp == 0) {
    // ------------------------------------------------------------- producer
    const int q0 = lane, q1 = lane + 32;
    const bool live0 = q0 < a.nq && (a.active == nullptr || a.active[a.q_base + q0] != 0u);
    const bool live1 = q1 < a.nq && (a.active == nullptr || a.active[a.q_base + q1] != 0u);
    const int64_t n_items = a.g_begin < a.n_groups ? (a.n_groups - a.g_begin + a.g_step - 1) / a.g_step : 0;
    int64_t item = 0, item_end = 0;
    // work counter read one chunk ahead: the atomic of the next chunk is in
    // flight while the current one is processed
    uint32_t pref = 0;
    if (lane == 0) pref = atomicAdd(a.work_ctr, 1u);
    auto next_group = [&]() -> int64_t {
      if (item + 1 < item_end) return a.g_begin + (++item) * a.g_step;
      const uint32_t c = __shfl_sync(0xFFFFFFFFu, pref, 0);
      item = (int64_t)c * kTcGroupChunk;
      item_end = item + kTcGroupChunk < n_items ? item + kTcGroupChunk : n_items;
      if (item >= n_items) return -1;
      if (lane == 0) pref = atomicAdd(a.work_ctr, 1u);
      return a.g_begin + item * a.g_step;
    };
    auto prefetch = [&](int64_t g, int t) {
      uint32_t *dst = slot_tab + (size_t)t * a.n_slots * 8;
      for (int i = lane; i < 2 * a.n_slots; i += 32) {
        const int s = i >> 1, h = i & 1;
        cp_async16(dst + s * 8 + h * 4, a.slot_bm[s] + g * kGroupWords + h * 4);
      }
      cp_async_commit();
    };
    // each lane's queries' CNFs in registers (queries with more than 16 terms use the lists)
    const PackedCnf pk0 = live0 ? pack_cnf(a, q0) : PackedCnf{};
    const PackedCnf pk1 = live1 ? pack_cnf(a, q1) : PackedCnf{};
    unsigned long long pass0 = 0, pass1 = 0;
    uint64_t pm = 0;
    int t = 0;
    int64_t g = next_group();
    if (g >= 0) prefetch(g, 0);
    int64_t gn = g >= 0 ? next_group() : -1;
    if (gn >= 0) prefetch(gn, 1);
    else cp_async_commit();
    while (g >= 0 && ok) {
      cp_async_wait_group<1>();
      __syncwarp();
      uint32_t pw0[8], pw1[8];
      const uint32_t *tab = slot_tab + (size_t)t * a.n_slots * 8;
      if (live0 && pk0.ok) eval_packed(pk0, tab, pw0);
      else if (live0) eval_cnf(a, q0, tab, pw0);
      else
#pragma unroll
        for (int w = 0; w < 8; ++w) pw0[w] = 0u;
      if (live1 && pk1.ok) eval_packed(pk1, tab, pw1);
      else if (live1) eval_cnf(a, q1, tab, pw1);
      else
#pragma unroll
        for (int w = 0; w < 8; ++w) pw1[w] = 0u;
      __syncwarp();
      const int64_t gnn = gn >= 0 ? next_group() : -1;
      if (gnn >= 0) prefetch(gnn, t);
      else cp_async_commit();
      const int64_t r0 = g * kGroupRows;
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        const int64_t left = a.n - (r0 + w * 32);
        const uint32_t valid = left >= 32 ? 0xFFFFFFFFu : (left > 0 ? ((1u << left) - 1u) : 0u);
        pw0[w] &= valid;
        pw1[w] &= valid;
        pass0 += (unsigned long long)__popc(pw0[w]);
        pass1 += (unsigned long long)__popc(pw1[w]);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t any = 0;
#pragma unroll
        for (int w = 0; w < 4; ++w) any |= pw0[4 * h + w] | pw1[4 * h + w];
        if (__reduce_or_sync(0xFFFFFFFFu, any) == 0u || !ok) continue;
        const int m = (int)(pm % kMetaDepth);
        if (!warp_wait(&meta_empty[m], (uint32_t)((pm / kMetaDepth) & 1u) ^ 1u, lane)) {
          ok = false;
          break;
        }
        const int64_t row0 = r0 + h * kTileRows;
        if (lane == 0) {
          meta[m].row0 = row0;
          meta[m].done = 0u;
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) {  // lane r: queries passing row 32w + r of the tile
          const uint32_t lo32 = transpose32(pw0[4 * h + w], lane);
          const uint32_t hi32 = N > 32 ? transpose32(pw1[4 * h + w], lane) : 0u;
          meta[m].qm[w * 32 + lane] = ((uint64_t)hi32 << 32) | lo32;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&meta_full[m]);
        ++pm;
      }
      g = gn;
      gn = gnn;
      t ^= 1;
    }
    cp_async_wait_all();
    if (ok) {  // end-of-work marker for the other roles
      const int m = (int)(pm % kMetaDepth);
      if (warp_wait(&meta_empty[m], (uint32_t)((pm / kMetaDepth) & 1u) ^ 1u, lane)) {
        if (lane == 0) {
          meta[m].done = 1u;
          mbar_arrive(&meta_full[m]);
        }
        ++pm;
      } else {
        ok = false;
      }
    }
    if (!ok && lane == 0) atomicOr(a.err, kErrTimeout);
    if (a.pass_cnt != nullptr) {
      if (live0) atomicAdd(&a.pass_cnt[a.q_base + q0], pass0);
      if (live1) atomicAdd(&a.pass_cnt[a.q_base + q1], pass1);
    }
  } else if (warp == kLoadWarp) {
    // ------------------------------------------------------------- loader
    // issues the TMA loads of every published tile, in message order, into the
    // ring of raw stages; decoupled from the predicate warp so that neither
    // waits for the other's latencies
    if (lane == 0) {
      uint64_t pm = 0, pr = 0;
      while (ok) {
        const int m = (int)(pm % kMetaDepth);
        if (!mbar_wait(&meta_full[m], (uint32_t)((pm / kMetaDepth) & 1u))) {
          ok = false;
          break;
        }
        if (meta[m].done) break;
        const int row0 = (int)meta[m].row0;
        for (int c = 0; c < C; ++c) {
          const int s = (int)(pr % (uint64_t)S);
          if (!mbar_wait(&raw_empty[s], (uint32_t)((pr / S) & 1u) ^ 1u)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&raw_full[s], (uint32_t)(kTileRows * tc_row_bytes(E)));
          tma_load_2d(raw + (size_t)s * kChunkBytes, &tmap, c * tc_epc(E), row0, &raw_full[s]);
          ++pr;
        }
        if (!ok) break;
        ++pm;
      }
      if (!ok) {
        atomicOr(a.err, kErrTimeout);
        const uint64_t first = pr > (uint64_t)S ? pr - S : 0;  // let issued loads land
        for (uint64_t p = first; p < pr; ++p) mbar_wait(&raw_full[p % S], (uint32_t)((p / S) & 1u));
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc2 = idesc_tf32(kTileRows, 2 * N), idesc1 = idesc_tf32(kTileRows, N);
      uint64_t pm = 0, pr = 0, pa = 0;
      bool issued = false;
      while (ok) {
        const int m = (int)(pm % kMetaDepth);
        if (!mbar_wait(&meta_full[m], (uint32_t)((pm / kMetaDepth) & 1u))) {
          ok = false;
          break;
        }
        if (meta[m].done) break;
        const int ab = (int)(pa & 1u);
        if (!mbar_wait(&acc_empty[ab], (uint32_t)((pa >> 1) & 1u) ^ 1u)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(ab * 2 * N);
        for (int c = 0; c < C && ok; ++c) {
          const int l = (int)(pr % (uint64_t)kABufs);
          if (!mbar_wait(&a_full[l], (uint32_t)((pr / kABufs) & 1u))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t ah = tmem_base + acol0 + (uint32_t)(l * 64), al = ah + 32u;
          if constexpr (E == kElemF32) {
            const uint32_t qa = smem_u32(qop) + (uint32_t)(c * 2 * N * 128);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
              // D[0,2N) += x_hi . [q_hi ; q_lo]^T, then D[0,N) += x_lo . q_hi^T
              mma_tf32_tmem_a(d, ah + (uint32_t)(ks * 8), sw128_desc(qa + (uint32_t)ks * 32u), idesc2,
                              (c | ks) != 0 ? 1u : 0u);
              mma_tf32_tmem_a(d, al + (uint32_t)(ks * 8), sw128_desc(qa + (uint32_t)ks * 32u), idesc1, 1u);
            }
          } else {
            // BF16 / e4m3 values are exact in TF32: one MMA per 8-wide K step,
            // D[0,2N) += x . [q_hi ; q_lo]^T over the chunk's 64 values (two
            // 32-value chunks of the query operand)
#pragma unroll
            for (int ks = 0; ks < 8; ++ks) {
              const uint32_t qa = smem_u32(qop) + (uint32_t)((2 * c + (ks >> 2)) * 2 * N * 128) +
                                  (uint32_t)(ks & 3) * 32u;
              mma_tf32_tmem_a(d, ah + (uint32_t)(ks * 8), sw128_desc(qa), idesc2, (c | ks) != 0 ? 1u : 0u);
            }
            (void)al;
            (void)idesc1;
          }
          issued = true;
          mma_commit(&a_empty[l]);
          ++pr;
        }
        if (!ok) break;
        mma_commit(&acc_full[ab]);
        ++pa;
        ++pm;
      }
      if (issued) {  // every MMA has finished before the tensor memory is freed
        mma_commit(drain);
        if (!mbar_wait(drain, 0u)) ok = false;
      }
      if (!ok) atomicOr(a.err, kErrTimeout);
    }
    __syncwarp();
  } else if (warp < kEpiWarp0) {
    // ------------------------------------------------------------- converters
    const int quarter = warp & 3;
    const int r = quarter * 32 + lane;  // this thread's row of every tile
    uint64_t pm = 0, pr = 0;
    while (ok) {
      const int m = (int)(pm % kMetaDepth);
      if (!warp_wait(&meta_full[m], (uint32_t)((pm / kMetaDepth) & 1u), lane)) {
        ok = false;
        break;
      }
      if (meta[m].done) break;
      for (int c = 0; c < C; ++c) {
        const int s = (int)(pr % (uint64_t)S), l = (int)(pr % (uint64_t)kABufs);
        if (!warp_wait(&raw_full[s], (uint32_t)((pr / S) & 1u), lane)) {
          ok = false;
          break;
        }
        uint32_t hi[32], lo[32];  // FP32 rows: x_hi, x_lo; BF16/FP8 rows: values 0-31, 32-63
        const unsigned char *rowp = raw + (size_t)s * kChunkBytes + (size_t)r * tc_row_bytes(E);
        if constexpr (E == kElemF32) {
#pragma unroll
          for (int cc = 0; cc < 8; ++cc) {  // 16-byte chunk cc of the row sits at slot cc ^ (r % 8)
            const float4 v = *reinterpret_cast<const float4 *>(rowp + (((cc ^ (r & 7)) & 7) << 4));
            const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const uint32_t hb = __float_as_uint(e[u]) & 0xFFFFE000u;
              hi[cc * 4 + u] = hb;
              lo[cc * 4 + u] = __float_as_uint(e[u] - __uint_as_float(hb));
            }
          }
        } else if constexpr (E == kElemBF16) {
#pragma unroll
          for (int cc = 0; cc < 8; ++cc) {  // 128-byte swizzle: 8 values per 16-byte chunk
            const uint4 v = *reinterpret_cast<const uint4 *>(rowp + (((cc ^ (r & 7)) & 7) << 4));
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
            uint32_t *dst = cc < 4 ? hi : lo;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              dst[(cc & 3) * 8 + 2 * u] = w[u] << 16;
              dst[(cc & 3) * 8 + 2 * u + 1] = w[u] & 0xFFFF0000u;
            }
          }
        } else {
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {  // 64-byte swizzle: chunk cc of row r at slot cc ^ ((r / 2) % 4)
            const uint4 v = *reinterpret_cast<const uint4 *>(rowp + (((cc ^ (r >> 1)) & 3) << 4));
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
            uint32_t *dst = cc < 2 ? hi : lo;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const __half2_raw hr =
                    __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)((w[u] >> (16 * h)) & 0xFFFFu), __NV_E4M3);
                const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&hr));
                dst[(cc & 1) * 16 + 4 * u + 2 * h] = __float_as_uint(f.x);
                dst[(cc & 1) * 16 + 4 * u + 2 * h + 1] = __float_as_uint(f.y);
              }
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&raw_empty[s]);  // the row is in registers: the stage may refill
        if (!warp_wait(&a_empty[l], (uint32_t)((pr / kABufs) & 1u) ^ 1u, lane)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t ta = tmem_base + ((uint32_t)(quarter * 32) << 16) + acol0 + (uint32_t)(l * 64);
        tmem_st32(ta, hi);
        tmem_st32(ta + 32u, lo);
        tmem_st_wait();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&a_full[l]);
        ++pr;
      }
      if (!ok) break;
      ++pm;
    }
    if (!ok && lane == 0) atomicOr(a.err, kErrTimeout);
  } else {
    // ------------------------------------------------------------- epilogue
    const int quarter = warp & 3;
    const int ew = warp - kEpiWarp0;
    uint64_t pm = 0, pa = 0;
    // Candidates are recorded in a per-warp shared-memory list by the lanes that
    // find them (a shared-memory atomic each).  A flush tests them exactly,
    // counts them per query, reserves each query's range of its buffer with one
    // global atomic and scatters the keys, so a query with many candidates (a
    // broad filter in the threshold sample) does not serialise on its counter.
    // The flush stays inline: an out-of-line call in this loop, between the
    // warp-collective tensor-memory loads, has faulted.
    uint64_t *ckey = reinterpret_cast<uint64_t *>(smem + T.cand) + (size_t)ew * kWarpCand;
    uint8_t *cqry = reinterpret_cast<uint8_t *>(smem + T.cand + (size_t)4 * kWarpCand * 8) + (size_t)ew * kWarpCand;
    uint32_t *ccnt = reinterpret_cast<uint32_t *>(smem + T.ccnt) + ew;
    uint32_t *cq = reinterpret_cast<uint32_t *>(smem + T.cq) + (size_t)ew * 2 * N;
    uint32_t *cb = cq + N;
    if (lane == 0) *ccnt = 0u;
    __syncwarp();
    auto flush = [&]() {
      __syncwarp();
      const uint32_t n = *ccnt < (uint32_t)kWarpCand ? *ccnt : (uint32_t)kWarpCand;
      for (int i = lane; i < N; i += 32) cq[i] = 0u;
      __syncwarp();
      uint32_t rk[kWarpCand / 32];
#pragma unroll
      for (int u = 0; u < kWarpCand / 32; ++u) {
        const uint32_t e = (uint32_t)lane + 32u * (uint32_t)u;
        rk[u] = 0xFFFFFFFFu;
        if (e < n) {
          const int q = cqry[e];
          if (ckey[e] >= taus[q]) rk[u] = atomicAdd(&cq[q], 1u);
        }
      }
      __syncwarp();
      for (int i = lane; i < N; i += 32) {
        const uint32_t c = cq[i];
        cb[i] = c != 0u ? atomicAdd(&a.buf_cnt[a.q_base + i], c) : 0u;
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < kWarpCand / 32; ++u) {
        if (rk[u] == 0xFFFFFFFFu) continue;
        const uint32_t e = (uint32_t)lane + 32u * (uint32_t)u;
        const int q = cqry[e];
        const uint32_t pos = cb[q] + rk[u];
        if ((int64_t)pos < a.buf_cap)
          a.buf[(size_t)(a.q_base + q) * (size_t)a.buf_cap + pos] = ckey[e];
        else
          atomicOr(&a.overflow[a.q_base + q], 1u);
      }
      __syncwarp();
      if (lane == 0) *ccnt = 0u;
      __syncwarp();
    };
    while (ok) {
      const int m = (int)(pm % kMetaDepth);
      if (!warp_wait(&meta_full[m], (uint32_t)((pm / kMetaDepth) & 1u), lane)) {
        ok = false;
        break;
      }
      if (meta[m].done) break;
      const int ab = (int)(pa & 1u);
      if (!warp_wait(&acc_full[ab], (uint32_t)((pa >> 1) & 1u), lane)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ab * 2 * N);
      const uint64_t qmask = meta[m].qm[quarter * 32 + lane];
      const uint32_t grow = (uint32_t)(meta[m].row0 + quarter * 32 + lane);
      float xs = 1.f;  // FP8 rows: score = scale * <q, x8>
      if constexpr (E == kElemFP8) xs = (int64_t)grow < a.n ? __ldg(a.xscale + grow) : 0.f;
#pragma unroll 1
      for (int j = 0; j < N / 16; ++j) {
        const uint32_t bm = (uint32_t)(qmask >> (16 * j)) & 0xFFFFu;
        if (!__any_sync(0xFFFFFFFFu, bm != 0u)) continue;  // no lane needs this block of 16 queries
        __syncwarp();
        uint32_t rh[16], rl[16];
        tmem_ld16(taddr + (uint32_t)(16 * j), rh);      // x_hi.q_hi + x_lo.q_hi
        tmem_ld16(taddr + (uint32_t)(N + 16 * j), rl);  // x_hi.q_lo
        tmem_ld_wait();
        if (a.mode == kCollect) {
          // A key can reach the threshold only if its score word does, i.e. the
          // score reaches the float threshold: a branch-free test builds the
          // lane's hit mask, and only warps with a hit record candidates (the
          // exact key tests run at the flush).
          float sc[16];
          uint32_t hit = 0;
          const float4 *tv = reinterpret_cast<const float4 *>(thr + 16 * j);
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const float4 t = tv[v];
            const float tt[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int b = 4 * v + u;
              sc[b] = (__uint_as_float(rh[b]) + __uint_as_float(rl[b])) * xs;
              hit |= (sc[b] >= tt[u] ? 1u : 0u) << b;
            }
          }
          hit &= bm;
          if (__any_sync(0xFFFFFFFFu, hit != 0u)) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {  // at most 256 entries are added between two checks
              const uint32_t hh = (hit >> (8 * h)) & 0xFFu;
              if (!__any_sync(0xFFFFFFFFu, hh != 0u)) continue;
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                if ((hh >> u) & 1u) {
                  const int b = 8 * h + u;
                  const uint32_t e = atomicAdd(ccnt, 1u);
                  if (e < (uint32_t)kWarpCand) {
                    ckey[e] = make_key(sc[b], grow);
                    cqry[e] = (uint8_t)(16 * j + b);
                  }
                }
              }
              __syncwarp();
              if (*ccnt > (uint32_t)(kWarpCand / 2)) flush();
            }
          }
        } else {
#pragma unroll
          for (int b = 0; b < 16; ++b) {
            if (!((bm >> b) & 1u)) continue;
            const int q = 16 * j + b;
            const uint64_t key = make_key((__uint_as_float(rh[b]) + __uint_as_float(rl[b])) * xs, grow);
            if (top >= 64 || (key >> top) == (taus[q] >> top))
              atomicAdd(&a.hist[(size_t)(a.q_base + q) * kFbBins + (uint32_t)((key >> shift) & dmask)], 1u);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&acc_empty[ab]);
        mbar_arrive(&meta_empty[m]);
      }
      ++pa;
      ++pm;
    }
    flush();
    if (!ok && lane == 0) atomicOr(a.err, kErrTimeout);
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem_base, kTmemCols);

  // grid completion: the last CTA resets the work counter and, in kHist mode,
  // fixes this pass's digit for every participating query
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

template <int N, int E>
cudaError_t launch_tc(const ScanArgs &a, const CUtensorMap &tmap, int grid, cudaStream_t s) {
  static_assert(4 * N + 64 * kABufs <= (int)kTmemCols, "tensor memory budget");
  const size_t budget = 220u * 1024u;
  int S = 12;
  if (a.d_pad % tc_epc(E) != 0) return cudaErrorInvalidValue;
  while (S > 2 && tc_layout(a.d_pad, tc_epc(E), N, a.n_slots, S).total + 1024 > budget) --S;
  const TcLayout T = tc_layout(a.d_pad, tc_epc(E), N, a.n_slots, S);
  if (T.total + 1024 > budget) return cudaErrorInvalidValue;
  auto *fn = k_scan_tc<N, E>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(T.total + 1024));
  if (e != cudaSuccess) return e;
  fn<<<grid, kTcThreads, T.total + 1024, s>>>(a, tmap, S);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_scan_tc(const ScanArgs &a, const void *tmap_x, int grid, cudaStream_t s) {
  const CUtensorMap &tm = *static_cast<const CUtensorMap *>(tmap_x);
  const int n16 = (a.nq + 15) / 16 * 16;
  switch (a.elem * 4 + n16 / 16 - 1) {
    case kElemF32 * 4 + 0: return launch_tc<16, kElemF32>(a, tm, grid, s);
    case kElemF32 * 4 + 1: return launch_tc<32, kElemF32>(a, tm, grid, s);
    case kElemF32 * 4 + 2: return launch_tc<48, kElemF32>(a, tm, grid, s);
    case kElemF32 * 4 + 3: return launch_tc<64, kElemF32>(a, tm, grid, s);
    case kElemBF16 * 4 + 0: return launch_tc<16, kElemBF16>(a, tm, grid, s);
    case kElemBF16 * 4 + 1: return launch_tc<32, kElemBF16>(a, tm, grid, s);
    case kElemBF16 * 4 + 2: return launch_tc<48, kElemBF16>(a, tm, grid, s);
    case kElemBF16 * 4 + 3: return launch_tc<64, kElemBF16>(a, tm, grid, s);
    case kElemFP8 * 4 + 0: return launch_tc<16, kElemFP8>(a, tm, grid, s);
    case kElemFP8 * 4 + 1: return launch_tc<32, kElemFP8>(a, tm, grid, s);
    case kElemFP8 * 4 + 2: return launch_tc<48, kElemFP8>(a, tm, grid, s);
    case kElemFP8 * 4 + 3: return launch_tc<64, kElemFP8>(a, tm, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lr
