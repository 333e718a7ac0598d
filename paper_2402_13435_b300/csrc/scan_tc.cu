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
// The term predicate runs first, in the tile filter: it lists the 128-row
// tiles that some query passes, each with its per-row query masks; tiles nobody
// passes are never read ("skip rows").  CTA b of the scan takes list entries
// b, b + grid, b + 2 grid, ..., so every role knows the tile sequence without
// waiting for another.  One CTA per SM, 14 warps with fixed roles (18 for
// BF16/FP8 rows):
//   warp 0     loader: issues the 2-D TMA loads (128 rows x 32 floats, 128-byte
//              swizzle) of its tiles into a ring of raw stages.
//   warp 1     owns the tensor memory and issues the MMAs from one thread.  The
//              job operand comes from tensor memory: per 8-wide K step one MMA
//              of width 2N with x_hi against [q_hi ; q_lo] and one of width N
//              with x_lo against q_hi, so accumulator columns [0, N) and
//              [N, 2N) add up to the 3xTF32 product.  Four accumulator buffers
//              when N <= 32 (two above; always four for BF16 / FP8 rows, whose
//              accumulators are N columns wide), so the MMAs run ahead of the
//              epilogue.
//              BF16 and e4m3 rows skip the converters: the MMA reads the
//              landed stage from shared memory (BF16: kind::f16, 16-value K
//              steps, against the queries rounded to BF16; e4m3: kind::f8f6f4,
//              32-value K steps, against the queries rounded to e4m3 under one
//              power-of-two scale per launch; one accumulator column per
//              query: the low-precision scan only picks candidates for the
//              FP32 rescore) and its commit frees the stage.
//   warps 2-5, 10-13  converters (FP32 rows), two sets of one warp per
//              tensor-memory lane quarter, taking alternate chunks: each thread
//              reads its row of a landed chunk, releases the raw stage at once,
//              and writes x_hi and x_lo into tensor memory (tcgen05.st).  Raw
//              stages therefore never wait on the tensor core.
//   warps 6-9 (and 14-17)  epilogue: read the accumulator (warp w owns lanes
//              32*(w%4) ..), with the row masks of the tile read one tile
//              ahead, test every passing (row, query) against the query's
//              threshold without branches, and record the few candidates in a
//              per-warp shared-memory list flushed to the query buffers in
//              bulk; a second set takes alternate tiles for BF16/FP8 rows.
// All waits are bounded; on a timeout the error word gets LR_ERR_TIMEOUT, the
// loader lets issued copies land, the MMA warp waits for its MMAs, and the
// tensor memory is freed before the CTA exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <type_traits>

#include "lr_internal.h"
#include "ptx.h"
#include "scan_common.cuh"

namespace lr {
namespace {

// warp roles: 0 loader, 1 MMA issuer, 2-5 and 10-13 the two converter sets,
// 6-9 the epilogue set, and for BF16/FP8 rows 14-17 a second epilogue set (the
// narrow rows leave more tiles per microsecond to test; FP32 runs faster with
// one set and the shared memory it saves)
constexpr int kEpiWarp0 = 6;
constexpr int kConvWarp1 = 10;
constexpr int kEpiWarp1 = 14;
// BF16 and e4m3 rows need no converters (their MMAs read the loaded stage):
// warps 2-5 and 10-13 become epilogue sets 2 and 3 there, so four sets of four
// warps test alternate tiles
// FP32 rows: one set up to 32 queries (a second measured 1.5 % slower there:
// its shared memory comes out of the raw stages), two for wider blocks and for
// two-block launches (one set per block)
__host__ __device__ constexpr int tc_epi_sets(int e, int n, int nb) {
  return e != kElemF32 ? 4 : (nb > 1 || n > 32) ? 2 : 1;
}
__host__ __device__ constexpr int tc_threads(int e, int n, int nb) {
  return (tc_epi_sets(e, n, nb) == 1 ? kEpiWarp1 : kEpiWarp1 + 4) * 32;
}
__device__ __forceinline__ bool is_converter(int w) { return (w >= 2 && w < kEpiWarp0) || (w >= kConvWarp1 && w < kEpiWarp1); }
// epilogue set of an epilogue warp: 6-9 -> 0, 14-17 -> 1, 2-5 -> 2, 10-13 -> 3
__device__ __forceinline__ int epi_set(int w) { return w >= kEpiWarp1 ? 1 : w >= kConvWarp1 ? 3 : w >= kEpiWarp0 ? 0 : 2; }
constexpr int kLoadWarp = 0;
constexpr int kTileRows = 128;
constexpr int kChunkBytes = kTileRows * 128;  // one raw stage: a 128-row tile of 128-byte rows

// Row elements per raw chunk and the bytes of a chunk's row: FP32 rows come in
// 32-float (128-byte) column blocks; BF16 in 64-value (128-byte) blocks; FP8
// e4m3 in 64-value (64-byte) blocks.
__host__ __device__ constexpr int tc_epc(int e) { return e == kElemF32 ? 32 : 64; }
__host__ __device__ constexpr int tc_row_bytes(int e) { return e == kElemFP8 ? 64 : 128; }
// candidates staged per epilogue warp (half for FP32 two-block launches, whose
// query operands leave less shared memory)
__host__ __device__ constexpr int tc_warp_cand(int nb) { return nb == 2 ? 256 : 512; }
constexpr int kMaxABufs = 4;                  // x_hi/x_lo chunk buffers in tensor memory, at most
constexpr uint32_t kTmemCols = 512;           // the whole tensor memory: one CTA per SM
// Accumulator buffers (2N columns each): four when they fit beside the x_hi/x_lo
// buffers, so the MMAs can run up to four tiles ahead of the epilogue.
// accumulator buffers (even: each belongs to one epilogue set) and their
// columns: FP32 rows accumulate x.q_hi and x.q_lo side by side (2N columns);
// BF16 / FP8 rows, whose scan only picks candidates for the FP32 rescore,
// score against the queries rounded to BF16 (N columns), so four buffers fit
// up to N = 64
// (BF16 / e4m3 rows: eight N-column buffers, two per epilogue set, in the
// tensor memory the x_hi/x_lo buffers of FP32 rows would take)
__host__ __device__ constexpr int tc_acc_bufs(int e, int n) { return e != kElemF32 ? 8 : n <= 32 ? 4 : 2; }
__host__ __device__ constexpr int tc_acc_w(int e, int n) { return e == kElemF32 ? 2 * n : n; }
// FP32 rows: x_hi/x_lo buffers (64 columns each) in the tensor memory the
// accumulators leave, at most four (six for narrow blocks, with two
// accumulators instead of four, measured slower)
__host__ __device__ constexpr int tc_abufs(int e, int n) {
  return e != kElemF32 ? 0 : ((512 - tc_acc_bufs(e, n) * tc_acc_w(e, n)) / 64 & ~1) > kMaxABufs
                                 ? kMaxABufs
                                 : ((512 - tc_acc_bufs(e, n) * tc_acc_w(e, n)) / 64 & ~1);  // even: two converter sets
}

// Row mask word of the tile list: bit q = launch query q passes the row.
template <int N>
using RowMask = typename std::conditional<(N <= 32), uint32_t, uint64_t>::type;

struct TcLayout {
  int S, C, C32, N;
  size_t raw, q, taus, cand, ccnt, cq, bars, holder, total;
};

__host__ __device__ inline size_t tc_align(size_t v, size_t a) { return (v + a - 1) / a * a; }

__host__ __device__ inline TcLayout tc_layout(int d_pad, int e, int N, int S, int epi_warps, int NB = 1) {
  TcLayout T;
  const int epc = tc_epc(e);
  T.S = S;
  T.C = d_pad / epc;   // raw chunks per tile
  T.C32 = d_pad / 32;  // 32-value chunks of the query operand
  T.N = N;
  size_t off = 0;
  T.raw = off;
  off += (size_t)S * kChunkBytes;
  // the query operand: FP32 rows, per 32-value chunk 2N rows (q_hi, then q_lo)
  // of 128 bytes; BF16, per 64-value chunk a 2N-row block of 128-byte rows (N
  // used); e4m3, per 64-value chunk N rows of 64 bytes
  T.q = off;
  off += e == kElemF32    ? (size_t)NB * T.C32 * 2 * N * 128
         : e == kElemBF16 ? (size_t)T.C * (NB > 1 ? NB * N : 2 * N) * 128
                          : (size_t)NB * T.C * N * 64;
  T.taus = tc_align(off, 16);
  off = T.taus + (size_t)NB * N * 12;  // 64-bit thresholds, then their score words as floats
  T.cand = tc_align(off, 16);     // per epilogue warp: keys, then query indices (bytes)
  off = T.cand + (size_t)epi_warps * tc_warp_cand(NB) * 9;
  T.ccnt = tc_align(off, 16);
  off = T.ccnt + (size_t)epi_warps * 4;
  T.cq = off;  // per epilogue warp: per-query counts, then reserved bases, of one flush
  off = T.cq + (size_t)epi_warps * 2 * N * 4;
  T.bars = tc_align(off, 16);
  off = T.bars + (size_t)(2 * S + 2 * kMaxABufs + 2 * 8 + 1) * 8;  // at most eight accumulator buffers
  T.holder = tc_align(off, 16);
  T.total = T.holder + 16;
  return T;
}

// First row of list tile e: tile e & 1 of the (e >> 1)-th group the launch
// visits (groups g_begin + i g_step).
__device__ __forceinline__ int64_t tile_first_row(const ScanArgs &a, int32_t e) {
  return (a.g_begin + (int64_t)(e >> 1) * a.g_step) * kGroupRows + (int64_t)(e & 1) * kTileRows;
}

// Leader-lane wait broadcast to the warp.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, int lane) {
  bool got = true;
  if (lane == 0) got = mbar_wait(bar, parity);
  return __shfl_sync(0xFFFFFFFFu, got ? 1 : 0, 0) != 0;
}

// NB = 2: each converted tile is scored against two 64-query blocks, each into
// its own accumulator (FP32 rows only; 128 queries per launch).
template <int N, int E, int NB>
__global__ void __launch_bounds__(tc_threads(E, N, NB), 1)
    k_scan_tc(const ScanArgs a, const __grid_constant__ CUtensorMap tmap, int S) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
  static_assert(NB == 1 || (NB == 2 && E == kElemF32 && (N == kTc2BlockQ || N == 64)) ||
                    (NB == kBf16Blocks && E != kElemF32 && N == 64),
                "several query blocks: FP32 rows, two of 48 or 64 queries; BF16 / e4m3 rows, four of 64");
  static_assert(NB == 1 || NB == tc_epi_sets(E, N, NB), "with several query blocks each epilogue set takes one");
  if (a.any_active != nullptr && *reinterpret_cast<const volatile uint32_t *>(a.any_active) == 0u) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem =
      smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);  // 1024-byte aligned for the swizzle atoms
  constexpr int kSets = tc_epi_sets(E, N, NB), kThreads = tc_threads(E, N, NB);
  constexpr int kWarpCand = tc_warp_cand(NB), kLaneCand = kWarpCand / 32;
  static_assert(kLaneCand >= 8, "a lane records up to eight hits between two room checks");
  const TcLayout T = tc_layout(a.d_pad, E, N, S, 4 * kSets, NB);
  const int C = T.C;
  const int C32 = T.C32;
  unsigned char *raw = smem + T.raw;
  float *qop = reinterpret_cast<float *>(smem + T.q);
  uint64_t *taus = reinterpret_cast<uint64_t *>(smem + T.taus);
  float *thr = reinterpret_cast<float *>(taus + NB * N);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + T.bars);
  uint64_t *raw_full = bars, *raw_empty = bars + S;
  // several query blocks share each accumulator of 2 NB N columns (both
  // epilogue sets read it), as many as fit next to two x_hi/x_lo buffers:
  // two of 192 columns for 48-query blocks (the MMAs of a tile overlap the
  // tests of the one before), one of 256 for 64-query blocks
  constexpr int kAccW = NB > 1 ? (E == kElemF32 ? 2 : 1) * NB * N : tc_acc_w(E, N);
  constexpr int kAcc = NB > 1 ? (E == kElemF32 ? 512 - 2 * 64 : 512) / kAccW : tc_acc_bufs(E, N);
  constexpr int kABufs = E != kElemF32 ? 2 : NB > 1 ? (512 - kAcc * kAccW) / 64 : tc_abufs(E, N);  // (unused for BF16 / e4m3)
  static_assert(E != kElemF32 || (kAcc * kAccW + 64 * kABufs <= 512 && kABufs >= 2 && kABufs % 2 == 0),
                "tensor memory: accumulators and an even number of x_hi/x_lo buffers");
  uint64_t *a_full = bars + 2 * S, *a_empty = a_full + kABufs;
  uint64_t *acc_full = a_empty + kABufs, *acc_empty = acc_full + kAcc;
  uint64_t *drain = acc_empty + kAcc;
  uint32_t *holder = reinterpret_cast<uint32_t *>(smem + T.holder);
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const uint32_t acol0 = (uint32_t)(kAcc * kAccW);  // first tensor-memory column of the x_hi/x_lo buffers
  __shared__ bool s_last;
  __shared__ uint32_t s_nlist;
  __shared__ uint32_t s_live[2 * NB];  // bit q: query q takes part in this launch

  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&raw_full[i], 1);
      mbar_init(&raw_empty[i], E == kElemF32 ? 4 : 1);  // FP32: the converter warps; else the MMAs' commit
    }
    for (int i = 0; i < kABufs; ++i) {
      mbar_init(&a_full[i], 4);
      mbar_init(&a_empty[i], 1);
    }
    for (int i = 0; i < kAcc; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], NB > 1 ? 4 * kSets : 4);  // with several blocks every set releases it
    }
    mbar_init(drain, 1);
    fence_mbar_init();
    // tiles listed by the tile filter (never more than the list holds), or
    // with dense tile masks every tile of the visited groups, in order
    if (NB > 1 && a.dense_tiles) {
      const int64_t ng = a.g_begin < a.n_groups ? (a.n_groups - a.g_begin + a.g_step - 1) / a.g_step : 0;
      int64_t nt = 2 * ng;
      if (nt > 0 && tile_first_row(a, (int32_t)(nt - 1)) >= a.n) --nt;  // a last group of <= 128 rows
      s_nlist = (uint32_t)(nt < a.tile_cap ? nt : a.tile_cap);
    } else {
      const uint32_t nl = *reinterpret_cast<const volatile uint32_t *>(a.tile_cnt);
      s_nlist = (int64_t)nl < a.tile_cap ? nl : (uint32_t)a.tile_cap;
    }
  }
  // queries of the launch in the K-major 128-byte swizzle layout: a TF32
  // hi/lo pair for FP32 rows, the queries rounded to BF16 for BF16 and FP8
  // rows; each thread issues its loads of a round together, then stores
  constexpr int kQu = 8;
  __shared__ float s_qinv;  // FP8 rows: 1 / the launch's power-of-two query scale
  if constexpr (E == kElemFP8) {
    // e4m3 queries for kind::f8f6f4 MMAs against the e4m3 rows: one
    // power-of-two scale for the whole launch maps the largest |q| into the
    // e4m3 range (the scale is exact; the epilogue divides it out with the row
    // scale).  Per 64-value chunk c: rows 0..N-1 of 64 bytes, 64-byte swizzle
    // (16-byte unit j of row r at unit j ^ ((r / 2) % 4)).
    __shared__ float s_qmax[32];
    float mx = 0.f;
    for (int i = threadIdx.x; i < a.nq * a.d_pad; i += kThreads)
      mx = fmaxf(mx, fabsf(a.Q[(size_t)a.q_base * a.d_pad + i]));
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, off));
    if (lane == 0) s_qmax[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      float m = 0.f;
      for (int w = 0; w < kThreads / 32; ++w) m = fmaxf(m, s_qmax[w]);
      // 2^e with 2^e * m <= 256 (below the e4m3 maximum 448); m = 0: scale 1
      int e = 0;
      if (m > 0.f) {
        e = (int)floorf(log2f(256.f / m));
        while (ldexpf(m, e) > 256.f) --e;
        e = e > 100 ? 100 : (e < -100 ? -100 : e);
      }
      s_qinv = ldexpf(1.f, -e);
      s_qmax[0] = ldexpf(1.f, e);
    }
    __syncthreads();
    const float qs = s_qmax[0];
    unsigned char *q8 = reinterpret_cast<unsigned char *>(qop);
    constexpr int kQRows = NB * N;  // every block's queries
    for (int i = threadIdx.x; i < C * kQRows * 64; i += kThreads) {
      const int c = i / (kQRows * 64), rem = i % (kQRows * 64), r = rem / 64, k = rem % 64;
      const float v = r < a.nq ? a.Q[(size_t)(a.q_base + r) * a.d_pad + c * 64 + k] * qs : 0.f;
      q8[(size_t)c * kQRows * 64 + (size_t)r * 64 + ((((k >> 4) ^ (r >> 1)) & 3) << 4) + (k & 15)] =
          (unsigned char)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
    }
  } else if constexpr (E == kElemBF16) {
    // per 64-value chunk c: rows 0..NB N - 1 (every block's queries) of a
    // block of 128-byte rows (2N rows for one block), 16-byte unit j of row r
    // at unit j ^ (r % 8)
    constexpr int kQRows = NB * N;
    uint16_t *qb = reinterpret_cast<uint16_t *>(qop);
    for (int i0 = 0; i0 < C * kQRows * 64; i0 += kQu * kThreads) {
      float v[kQu];
#pragma unroll
      for (int u = 0; u < kQu; ++u) {
        const int i = i0 + u * kThreads + threadIdx.x;
        const int c = i / (kQRows * 64), rem = i % (kQRows * 64), r = rem / 64, k = rem % 64;
        v[u] = i < C * kQRows * 64 && r < a.nq ? a.Q[(size_t)(a.q_base + r) * a.d_pad + c * 64 + k] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kQu; ++u) {
        const int i = i0 + u * kThreads + threadIdx.x;
        if (i >= C * kQRows * 64) break;
        const int c = i / (kQRows * 64), rem = i % (kQRows * 64), r = rem / 64, k = rem % 64;
        const size_t base = (size_t)c * (NB > 1 ? kQRows : 2 * N) * 128;
        qb[(base + (size_t)r * 128 + ((((k >> 3) ^ (r & 7)) & 7) << 4) + (k & 7) * 2) / 2] =
            __bfloat16_as_ushort(__float2bfloat16_rn(v[u]));
      }
    }
  } else
  for (int i0 = 0; i0 < NB * C32 * N * 32; i0 += kQu * kThreads) {
    // block bq holds queries bq N .. bq N + N - 1 in its own operand region
    float v[kQu];
#pragma unroll
    for (int u = 0; u < kQu; ++u) {
      const int i = i0 + u * kThreads + threadIdx.x;
      const int bq = NB > 1 ? i / (C32 * N * 32) : 0, ii = NB > 1 ? i % (C32 * N * 32) : i;
      const int c = ii / (N * 32), rem = ii % (N * 32), r = rem / 32, k = rem % 32;
      const int qi = bq * N + r;
      v[u] = i < NB * C32 * N * 32 && qi < a.nq ? a.Q[(size_t)(a.q_base + qi) * a.d_pad + c * 32 + k] : 0.f;
      (void)qi;
    }
#pragma unroll
    for (int u = 0; u < kQu; ++u) {
      const int i = i0 + u * kThreads + threadIdx.x;
      if (i >= NB * C32 * N * 32) break;
      const int bq = NB > 1 ? i / (C32 * N * 32) : 0, ii = NB > 1 ? i % (C32 * N * 32) : i;
      const int c = ii / (N * 32), rem = ii % (N * 32), r = rem / 32, k = rem % 32;
      const float h = __uint_as_float(__float_as_uint(v[u]) & 0xFFFFE000u);
      const int rh = bq * N + r;  // rows of q_hi (all blocks), then of q_lo
      const int rl = NB * N + rh;
      const size_t base = (size_t)c * 2 * NB * N * 128;
      qop[(base + (size_t)rh * 128 + ((((k >> 2) ^ (rh & 7)) & 7) << 4) + (k & 3) * 4) / 4] = h;
      qop[(base + (size_t)rl * 128 + ((((k >> 2) ^ (rl & 7)) & 7) << 4) + (k & 3) * 4) / 4] = v[u] - h;
    }
  }
  {  // thread q < NB N: query q's threshold; warps 0 .. 2 NB - 1 record which queries take part
    const int q = threadIdx.x;
    bool live = false;
    if (q < NB * N) {
      const int g2 = a.q_base + q;
      live = q < a.nq && (a.active == nullptr || a.active[g2] != 0u);
      taus[q] = !live ? 0ull : (a.mode == kCollect ? (a.tau ? a.tau[g2] : 0ull) : a.prefix[g2]);
      // score_key(s) >= h  <=>  s >= thr[q] for every non-NaN score s
      const uint32_t h = (uint32_t)(taus[q] >> 32);
      thr[q] = h <= score_key(-INFINITY) ? -INFINITY
               : h > score_key(INFINITY) ? __uint_as_float(0x7FFFFFFFu)  // NaN: no score passes
                                         : key_score(h);
    }
    if (warp < 2 * NB) {
      const uint32_t b = __ballot_sync(0xFFFFFFFFu, live);
      if (lane == 0) s_live[warp] = b;
    }
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

  // this CTA's tiles: list entries blockIdx.x + k * gridDim.x, k < n_mine
  const int64_t n_list = (int64_t)s_nlist;
  const int64_t n_mine = n_list > (int64_t)blockIdx.x ? (n_list - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  auto entry = [&](int64_t k) -> int64_t { return (int64_t)blockIdx.x + k * (int64_t)gridDim.x; };
  // id of the CTA's k-th tile; an id outside the list's range or the index
  // (which the tile filter never writes) is reported and read as -1: its rows
  // are loaded from the first tile and no query tests them
  auto tile_id = [&](int64_t k) -> int32_t {
    // dense tile masks come with two-block launches only: a compile-time test
    // (a runtime one here, on every tile id, measured 6 % slower)
    const int32_t t = (NB > 1 && a.dense_tiles) ? (int32_t)entry(k) : a.tile_row[entry(k)];
    if ((int64_t)(uint32_t)t < a.tile_cap && tile_first_row(a, t) < a.n) return t;
    atomicOr(a.err, kErrTileList);
    return -1;
  };

  if (warp == kLoadWarp) {
    // ------------------------------------------------------------- loader
    // the warp reads the ids of 32 tiles at a time (the next 32 in flight
    // meanwhile); lane 0 issues the TMA loads into the raw ring
    auto ids_from = [&](int64_t k0) -> int32_t {
      const int64_t k = k0 + lane;
      return k < n_mine ? tile_id(k) : 0;
    };
    int32_t rcur = ids_from(0), rnext = ids_from(32);
    uint64_t pr = 0;
    for (int64_t k = 0; k < n_mine && ok; ++k) {
      if (k > 0 && (k & 31) == 0) {
        rcur = rnext;
        rnext = ids_from(k + 32);
      }
      const int row0 = (int)tile_first_row(a, max(__shfl_sync(0xFFFFFFFFu, rcur, (int)(k & 31)), 0));
      for (int c = 0; c < C; ++c) {
        const int s = (int)(pr % (uint64_t)S);
        if (!warp_wait(&raw_empty[s], (uint32_t)((pr / S) & 1u) ^ 1u, lane)) {
          ok = false;
          break;
        }
        if (lane == 0) {
          mbar_arrive_expect_tx(&raw_full[s], (uint32_t)(kTileRows * tc_row_bytes(E)));
          tma_load_2d(raw + (size_t)s * kChunkBytes, &tmap, c * tc_epc(E), row0, &raw_full[s]);
        }
        ++pr;
      }
    }
    if (!ok && lane == 0) {
      atomicOr(a.err, kErrTimeout);
      const uint64_t first = pr > (uint64_t)S ? pr - S : 0;  // let issued loads land
      for (uint64_t p = first; p < pr; ++p) mbar_wait(&raw_full[p % S], (uint32_t)((p / S) & 1u));
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      // every query block at once: x_hi against all 2 NB N operand rows, x_lo
      // against the NB N q_hi rows (one accumulator of 2 NB N columns)
      const uint32_t idesc2 = idesc_tf32(kTileRows, 2 * NB * N), idesc1 = idesc_tf32(kTileRows, NB * N);
      uint64_t pr = 0, pa = 0;
      bool issued = false;
      for (int64_t k = 0; k < n_mine && ok; ++k) {
        const int ab = (int)(pa % (uint64_t)kAcc);
        if (!mbar_wait(&acc_empty[ab], (uint32_t)((pa / kAcc) & 1u) ^ 1u)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(ab * kAccW);
        for (int c = 0; c < C && ok; ++c) {
          if constexpr (E == kElemFP8) {
            // e4m3 rows feed the tensor cores straight from the loaded stage:
            // D[0,N) += x8 . e4m3(q s)^T, two 32-value K steps per 64-value
            // chunk; the commit frees the stage once the MMAs have read it
            const int s = (int)(pr % (uint64_t)S);
            if (!mbar_wait(&raw_full[s], (uint32_t)((pr / S) & 1u))) {
              ok = false;
              break;
            }
            tc_fence_after();
            constexpr uint32_t idesc8 = idesc_e4m3(kTileRows, NB * N);  // every block's queries
            const uint32_t xa = smem_u32(raw + (size_t)s * kChunkBytes);
            const uint32_t qa = smem_u32(qop) + (uint32_t)(c * NB * N * 64);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks)
              mma_e4m3(d, sw64_desc(xa + (uint32_t)ks * 32u), sw64_desc(qa + (uint32_t)ks * 32u), idesc8,
                       (c | ks) != 0 ? 1u : 0u);
            issued = true;
            mma_commit(&raw_empty[s]);
            ++pr;
            continue;
          }
          if constexpr (E == kElemBF16) {
            // BF16 rows feed the tensor cores straight from the loaded stage:
            // D[0,N) += x . bf16(q)^T, four 16-value K steps per chunk; the
            // commit frees the stage once the MMAs have read it
            const int s = (int)(pr % (uint64_t)S);
            if (!mbar_wait(&raw_full[s], (uint32_t)((pr / S) & 1u))) {
              ok = false;
              break;
            }
            tc_fence_after();
            // every block's queries in one MMA (N = NB N: 256 columns with four blocks)
            constexpr uint32_t idesc_b = idesc_bf16(kTileRows, NB * N);
            const uint32_t xa = smem_u32(raw + (size_t)s * kChunkBytes);
            const uint32_t qa = smem_u32(qop) + (uint32_t)(c * (NB > 1 ? NB * N : 2 * N) * 128);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
              mma_bf16(d, sw128_desc(xa + (uint32_t)ks * 32u), sw128_desc(qa + (uint32_t)ks * 32u), idesc_b,
                       (c | ks) != 0 ? 1u : 0u);
            issued = true;
            mma_commit(&raw_empty[s]);
            ++pr;
            continue;
          }
          const int l = (int)(pr % (uint64_t)kABufs);
          if (!mbar_wait(&a_full[l], (uint32_t)((pr / kABufs) & 1u))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t ah = tmem_base + acol0 + (uint32_t)(l * 64), al = ah + 32u;
          const uint32_t qa = smem_u32(qop) + (uint32_t)(c * 2 * NB * N * 128);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            // D[0,2NB N) += x_hi . [q_hi ; q_lo]^T, then D[0,NB N) += x_lo . q_hi^T
            mma_tf32_tmem_a(d, ah + (uint32_t)(ks * 8), sw128_desc(qa + (uint32_t)ks * 32u), idesc2,
                            (c | ks) != 0 ? 1u : 0u);
            mma_tf32_tmem_a(d, al + (uint32_t)(ks * 8), sw128_desc(qa + (uint32_t)ks * 32u), idesc1, 1u);
          }
          issued = true;
          mma_commit(&a_empty[l]);
          ++pr;
        }
        if (!ok) break;
        mma_commit(&acc_full[ab]);
        ++pa;
      }
      if (issued) {  // every MMA has finished before the tensor memory is freed
        mma_commit(drain);
        if (!mbar_wait(drain, 0u)) ok = false;
      }
      if (!ok) atomicOr(a.err, kErrTimeout);
    }
    __syncwarp();
  } else if (E == kElemF32 && is_converter(warp)) {
    // ------------------------------------------------------------- converters
    // (FP32 rows only: the MMAs read BF16 and e4m3 rows from the loaded stage)
    // two sets of four warps take alternate chunks (set = chunk index & 1), so
    // two chunks per lane quarter are in flight; S and kABufs are even, so a
    // raw stage or an x_hi/x_lo buffer always belongs to the same set and its
    // barrier phases are met in order
    const int quarter = warp & 3;
    const uint64_t cset = warp >= kConvWarp1 ? 1u : 0u;
    const int r = quarter * 32 + lane;  // this thread's row of every tile
    uint64_t pr = 0;
    for (int64_t k = 0; E == kElemF32 && k < n_mine && ok; ++k) {
      for (int c = 0; c < C; ++c, ++pr) {
        if ((pr & 1u) != cset) continue;
        const int s = (int)(pr % (uint64_t)S), l = (int)(pr % (uint64_t)kABufs);
        if (!warp_wait(&raw_full[s], (uint32_t)((pr / S) & 1u), lane)) {
          ok = false;
          break;
        }
        uint32_t hi[32], lo[32];  // x_hi, x_lo of the row's 32 values
        const unsigned char *rowp = raw + (size_t)s * kChunkBytes + (size_t)r * tc_row_bytes(E);
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
      }
    }
    if (!ok && lane == 0) atomicOr(a.err, kErrTimeout);
  } else {
    // ------------------------------------------------------------- epilogue
    // with two sets, sets of four warps take alternate tiles (set = tile index
    // & 1); with an even number of accumulator buffers each buffer belongs to
    // one set
    const int quarter = warp & 3;
    const int eset = epi_set(warp);
    const int ew = eset * 4 + ((warp - 2) & 3);  // the warp's candidate list (each set's warps start at 2 mod 4)
    const int bq = NB > 1 ? eset : 0;  // the set's query block (one per set with several blocks)
    const int qoff = bq * N;           // its first query within the launch
    // Candidates are recorded in a per-warp shared-memory list by the lanes that
    // find them.  In the main scan, where hits are rare, each lane owns every
    // 32nd entry (entry 32 i + lane, i < kLaneCand) and counts its own in a
    // register: no shared atomic or cross-lane exchange sits on the hit path
    // (a shared-memory atomic per hit measured three times the cost of the
    // score tests).  In the threshold sample, where nearly every test hits, a
    // prefix sum over the lanes' hit counts packs the list.
    // A flush tests them exactly,
    // counts them per query, reserves each query's range of its buffer with one
    // global atomic and scatters the keys, so a query with many candidates (a
    // broad filter in the threshold sample) does not serialise on its counter.
    // The flush stays inline: an out-of-line call in this loop, between the
    // warp-collective tensor-memory loads, has faulted.
    uint64_t *ckey = reinterpret_cast<uint64_t *>(smem + T.cand) + (size_t)ew * kWarpCand;
    uint8_t *cqry = reinterpret_cast<uint8_t *>(smem + T.cand + (size_t)4 * kSets * kWarpCand * 8) + (size_t)ew * kWarpCand;
    uint32_t *ccnt = reinterpret_cast<uint32_t *>(smem + T.ccnt) + ew;
    uint32_t *cq = reinterpret_cast<uint32_t *>(smem + T.cq) + (size_t)ew * 2 * N;  // the set's block
    uint32_t *cb = cq + N;
    if (lane == 0) *ccnt = 0u;
    __syncwarp();
    const bool lane_slots = a.tau != nullptr;  // main scan: per-lane entries
    uint32_t lcnt = 0;                         // this lane's entries (lane_slots)
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
        if (lane_slots ? (uint32_t)u < lcnt : e < n) {
          const int q = cqry[e];
          if (ckey[e] >= taus[q]) rk[u] = atomicAdd(&cq[q - qoff], 1u);
        }
      }
      __syncwarp();
      for (int i = lane; i < N; i += 32) {
        const uint32_t c = cq[i];
        cb[i] = c != 0u ? atomicAdd(&a.buf_cnt[a.q_base + qoff + i], c) : 0u;
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < kWarpCand / 32; ++u) {
        if (rk[u] == 0xFFFFFFFFu) continue;
        const uint32_t e = (uint32_t)lane + 32u * (uint32_t)u;
        const int q = cqry[e];
        const uint32_t pos = cb[q - qoff] + rk[u];
        if ((int64_t)pos < a.buf_cap)
          a.buf[(size_t)(a.q_base + q) * (size_t)a.buf_cap + pos] = ckey[e];
        else
          atomicOr(&a.overflow[a.q_base + q], 1u);
      }
      __syncwarp();
      if (lane == 0) *ccnt = 0u;
      lcnt = 0u;
      __syncwarp();
    };
    // this lane's row mask (and FP8 row scale) read one tile ahead, the tile
    // ids two ahead, so no global load latency sits on the tile's path
    const int lr = quarter * 32 + lane;
    const RowMask<N> *msg = static_cast<const RowMask<N> *>(a.tile_msg) + lr;
    // blocks 1 .. NB - 1: their row masks in tile_msg2, msg_block_stride words apart
    const RowMask<N> *msg2 =
        NB > 1 ? static_cast<const RowMask<N> *>(a.tile_msg2) + (size_t)(bq > 0 ? bq - 1 : 0) * a.msg_block_stride + lr
               : msg;
    auto tile_of = [&](int64_t k) -> int32_t { return k < n_mine ? tile_id(k) : -1; };
    auto mask_of = [&](int32_t t, int64_t k, int bq) -> RowMask<N> {
      return k < n_mine && t >= 0 ? (bq == 0 ? msg : msg2)[(size_t)t * kTileRows] : (RowMask<N>)0;
    };
    auto scale_of = [&](int32_t t, int64_t k) -> float {  // FP8 rows: score = scale * <q, x8>
      if constexpr (E == kElemFP8) {
        const int64_t g = tile_first_row(a, max(t, 0)) + lr;
        return k < n_mine && t >= 0 && g < a.n ? __ldg(a.xscale + g) * s_qinv : 0.f;  // exact: 2^-e
      } else {
        return 1.f;
      }
    };
    // the list may be one written for a larger set of queries (the exact
    // fallback reuses the main pass's list): only this launch's queries count
    // Units of work: accumulator use pa = tile k x NB + query block; this set
    // takes pa = eset, eset + kSets, ..: alternate tiles with one block, block
    // eset of every tile with two (NB = kSets)
    uint64_t live_mask;  // bits of the launch's queries qoff .. qoff + N - 1
    {
      const int w = qoff >> 5, sh = qoff & 31;
      const uint64_t lo = (uint64_t)s_live[w] | ((uint64_t)(w + 1 < 2 * NB ? s_live[w + 1] : 0u) << 32);
      const uint64_t hi = w + 2 < 2 * NB ? s_live[w + 2] : 0u;
      live_mask = sh != 0 ? (lo >> sh) | (hi << (64 - sh)) : lo;
      if (N < 64) live_mask &= (1ull << N) - 1ull;
    }
    constexpr int kStep = NB > 1 ? 1 : kSets;  // tiles between two of the set's units
    const int64_t k0 = NB > 1 ? 0 : eset;
    int32_t t_next = tile_of(k0), t_after = tile_of(k0 + kStep);
    RowMask<N> qm_next = mask_of(t_next, k0, bq);
    float xs_next = scale_of(t_next, k0);
    for (int64_t k = k0; k < n_mine && ok; k += kStep) {  // this set's tiles
      const uint64_t qmask = (uint64_t)qm_next & live_mask;
      qm_next = mask_of(t_after, k + kStep, bq);
      const uint32_t grow = (uint32_t)(tile_first_row(a, max(t_next, 0)) + lr);
      const float xs = xs_next;
      xs_next = scale_of(t_after, k + kStep);
      t_next = t_after;
      t_after = tile_of(k + 2 * kStep);
      const uint64_t pa = (uint64_t)k;  // accumulator use = tile index
      const int ab = (int)(pa % (uint64_t)kAcc);
      if (!warp_wait(&acc_full[ab], (uint32_t)((pa / kAcc) & 1u), lane)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ab * kAccW);
      // queries 16j .. 16j+15 of the lane's row: rh = x_hi.q_hi + x_lo.q_hi, rl = x_hi.q_lo
      auto test_block = [&](int j, const uint32_t (&rh)[16], const uint32_t (&rl)[16]) {
        const uint32_t bm = (uint32_t)(qmask >> (16 * j)) & 0xFFFFu;
        if (a.mode == kCollect) {
          // A key can reach the threshold only if its score word does, i.e. the
          // score reaches the float threshold: a branch-free test builds the
          // lane's hit mask, and only warps with a hit record candidates (the
          // exact key tests run at the flush).
          float sc[16];
          uint32_t hit = 0;
          const float4 *tv = reinterpret_cast<const float4 *>(thr + qoff + 16 * j);
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const float4 t = tv[v];
            const float tt[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int b = 4 * v + u;
              sc[b] = (E == kElemF32 ? __uint_as_float(rh[b]) + __uint_as_float(rl[b]) : __uint_as_float(rh[b])) * xs;
              hit |= (sc[b] >= tt[u] ? 1u : 0u) << b;
            }
          }
          hit &= bm;
          if (NB == 1 && a.tau == nullptr) {
            // Threshold sample: every passing pair is a candidate, so nearly
            // every test hits; a prefix sum over the lanes' hit counts places
            // them in the warp's list without atomics (flushed when full).
            const uint32_t nh = (uint32_t)__popc(hit);
            uint32_t incl = nh;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
              const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, off);
              if (lane >= off) incl += t;
            }
            const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
            if (total != 0u) {
              uint32_t base = *ccnt;
              if (base + total > (uint32_t)kWarpCand) {
                flush();
                base = 0u;
              }
              uint32_t e = base + incl - nh;
#pragma unroll
              for (int b = 0; b < 16; ++b) {
                if ((hit >> b) & 1u) {
                  ckey[e] = make_key(sc[b], grow);
                  cqry[e] = (uint8_t)(qoff + 16 * j + b);
                  ++e;
                }
              }
              __syncwarp();
              if (lane == 0) *ccnt = base + total;
              __syncwarp();
            }
          } else if (__any_sync(0xFFFFFFFFu, hit != 0u)) {
            if constexpr (NB > 1) {
              // several-block launches (many candidates per tile): a lane
              // visits only its own hits (usually one or two), the score of
              // hit b picked by a branch-free select chain (measured 4-8 %
              // faster there, 0.7 % slower for one block)
              constexpr int kPart = kLaneCand >= 16 ? 16 : 8;  // queries per room check
#pragma unroll
              for (int h = 0; h < 16 / kPart; ++h) {
                uint32_t hh = kPart == 16 ? hit : (hit >> (8 * h)) & 0xFFu;
                if (__any_sync(0xFFFFFFFFu, lcnt + (uint32_t)__popc(hh) > (uint32_t)kLaneCand)) flush();
                while (hh != 0u) {
                  const int b = kPart * h + __ffs(hh) - 1;
                  hh &= hh - 1u;
                  float v = sc[0];
#pragma unroll
                  for (int u = 1; u < 16; ++u) v = b == u ? sc[u] : v;
                  const uint32_t e = lcnt * 32u + (uint32_t)lane;
                  ckey[e] = make_key(v, grow);
                  cqry[e] = (uint8_t)(qoff + 16 * j + b);
                  ++lcnt;
                }
              }
            } else {
#pragma unroll
              for (int h = 0; h < 2; ++h) {  // eight queries at a time: room for all of every lane's hits, else flush first
                const uint32_t hh = (hit >> (8 * h)) & 0xFFu;
                if (__any_sync(0xFFFFFFFFu, lcnt + (uint32_t)__popc(hh) > (uint32_t)kLaneCand)) flush();
                if (hh != 0u) {
#pragma unroll
                  for (int u = 0; u < 8; ++u) {
                    if ((hh >> u) & 1u) {
                      const int b = 8 * h + u;
                      const uint32_t e = lcnt * 32u + (uint32_t)lane;
                      ckey[e] = make_key(sc[b], grow);
                      cqry[e] = (uint8_t)(qoff + 16 * j + b);
                      ++lcnt;
                    }
                  }
                }
              }
            }
          }
        } else {
#pragma unroll
          for (int b = 0; b < 16; ++b) {
            if (!((bm >> b) & 1u)) continue;
            const int q = qoff + 16 * j + b;
            const uint64_t key =
                make_key((E == kElemF32 ? __uint_as_float(rh[b]) + __uint_as_float(rl[b]) : __uint_as_float(rh[b])) * xs,
                         grow);
            if (top >= 64 || (key >> top) == (taus[q] >> top))
              atomicAdd(&a.hist[(size_t)(a.q_base + q) * kFbBins + (uint32_t)((key >> shift) & dmask)], 1u);
          }
        }
      };
      // one block of 16 queries at a time (loading all blocks before one wait
      // was measured slower)
#pragma unroll 1
      for (int j = 0; j < N / 16; ++j) {
        if (!__any_sync(0xFFFFFFFFu, ((qmask >> (16 * j)) & 0xFFFFu) != 0u)) continue;  // no lane needs it
        __syncwarp();
        uint32_t rh[16], rl[16];
        tmem_ld16(taddr + (uint32_t)(qoff + 16 * j), rh);
        if constexpr (E == kElemF32) {
          tmem_ld16(taddr + (uint32_t)(NB * N + qoff + 16 * j), rl);
        } else {
#pragma unroll
          for (int z = 0; z < 16; ++z) rl[z] = 0u;  // one accumulator column per query (rl unused)
        }
        tmem_ld_wait();
        test_block(j, rh, rl);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[ab]);
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
      if (!a.keep_list) *a.tile_cnt = 0u;  // the next tile filter starts an empty list
      *a.done_ctr = 0u;
    }
  }
}

template <int N, int E, int NB = 1>
cudaError_t launch_tc(const ScanArgs &a, const CUtensorMap &tmap, int grid, cudaStream_t s) {
  static_assert(tc_acc_bufs(E, N) * tc_acc_w(E, N) + (E == kElemF32 ? 64 * tc_abufs(E, N) : 0) <= (int)kTmemCols,
                "tensor memory budget");
  static_assert(NB > 1 || tc_acc_bufs(E, N) % tc_epi_sets(E, N, NB) == 0,
                "each accumulator buffer belongs to one epilogue set");
  static_assert(E != kElemF32 || NB > 1 || (tc_abufs(E, N) % 2 == 0 && tc_abufs(E, N) >= 4),
                "each converter set owns every other x_hi/x_lo buffer");
  const size_t budget = 220u * 1024u;
  int S = 12;  // raw stages: even (each converter set owns every other stage)
  if (a.d_pad % tc_epc(E) != 0) return cudaErrorInvalidValue;
  while (S > 2 && tc_layout(a.d_pad, E, N, S, 4 * tc_epi_sets(E, N, NB), NB).total + 1024 > budget) S -= 2;
  const TcLayout T = tc_layout(a.d_pad, E, N, S, 4 * tc_epi_sets(E, N, NB), NB);
  if (T.total + 1024 > budget) return cudaErrorInvalidValue;
  auto *fn = k_scan_tc<N, E, NB>;
  cudaError_t e = allow_dynamic_smem((const void *)fn, (size_t)(T.total + 1024));
  if (e != cudaSuccess) return e;
  return launch_pdl(fn, dim3((unsigned)grid), dim3(tc_threads(E, N, NB)), (size_t)(T.total + 1024), s, a, tmap, S);
}

}  // namespace

cudaError_t launch_scan_tc(const ScanArgs &a, const void *tmap_x, int grid, cudaStream_t s) {
  if (a.dense_tiles) return cudaErrorInvalidValue;  // dense tile masks feed two-block launches only
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

cudaError_t launch_scan_tc2(const ScanArgs &a, const void *tmap_x, int grid, cudaStream_t s) {
  // the main scan only, d <= 128 (the query operand of every block in shared
  // memory): FP32 rows, block_q + 1 .. 2 block_q queries as two blocks of
  // block_q (48 or 64); BF16 and e4m3 rows, 65 .. 256 queries as four blocks of 64
  const int bq = a.block_q;
  const int nb = a.elem == kElemF32 ? 2 : kBf16Blocks;
  if (a.d_pad > 128 || a.nq <= bq || a.nq > nb * bq || (a.elem == kElemF32 && bq != kTc2BlockQ && bq != 64) ||
      (a.elem != kElemF32 && bq != 64) || !a.dense_tiles || a.tile_msg2 == nullptr || a.mode != kCollect ||
      a.tau == nullptr)
    return cudaErrorInvalidValue;
  const CUtensorMap &tm = *static_cast<const CUtensorMap *>(tmap_x);
  if (a.elem == kElemBF16) return launch_tc<64, kElemBF16, kBf16Blocks>(a, tm, grid, s);
  if (a.elem == kElemFP8) return launch_tc<64, kElemFP8, kBf16Blocks>(a, tm, grid, s);
  return bq == 64 ? launch_tc<64, kElemF32, 2>(a, tm, grid, s) : launch_tc<kTc2BlockQ, kElemF32, 2>(a, tm, grid, s);
}

}  // namespace lr
