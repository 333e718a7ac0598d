// Tile filter: the term predicate (F-TBR) of a tensor-core scan, evaluated
// ahead of the scan for all 256-row groups it visits.
//
// Sec. 5.2 restricts the candidates of each query to the jobs whose terms
// satisfy its CNF; Sec. 5.3 fuses that restriction with the embedding scan so
// that rows no query accepts are never read.  Here the restriction runs as its
// own wide kernel, one warp per group and one lane per two queries, and writes
// for every 128-row tile t (rows 128 t ..) that some query passes
//     tile_msg[t][r]     the mask of the launch's queries that pass row r
//                        (bit q; 32-bit words when the launch has at most 32
//                        queries, else 64-bit), stored at the tile's own slot,
// and appends t to the compact list tile_row[].  The scan then streams exactly
// the listed tiles, and its pipeline carries no predicate latency.  Each warp
// works alone on chunks of eight groups, with the next group's term words in
// flight while it evaluates the current one, and appends a chunk's tiles with
// one atomic, so the list order follows the warps' progress rather than the
// row order; the scan does not depend on it.  The per-query pass counts of the
// launch are accumulated here as well.
#include <algorithm>

#include "lr_internal.h"
#include "ptx.h"
#include "scan_common.cuh"

namespace lr {
namespace {

constexpr int kTfThreads = 256;
constexpr int kTfWarps = kTfThreads / 32;
constexpr int kTfMaxChunk = 8;  // groups per list append (16 tiles at most)

// 32x32 bit-matrix transpose across the warp: lane i holds row i on entry
// (bit c = column c) and column i on exit (bit r = row r).
template <int J, uint32_t M>
__device__ __forceinline__ uint32_t transpose_stage(uint32_t x, int lane) {
  const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, J);
  return (lane & J) ? (((y >> J) & M) | (x & ~M)) : ((x & M) | ((y & M) << J));
}

__device__ __forceinline__ uint32_t bit_transpose32(uint32_t x, int lane) {
  x = transpose_stage<16, 0x0000FFFFu>(x, lane);
  x = transpose_stage<8, 0x00FF00FFu>(x, lane);
  x = transpose_stage<4, 0x0F0F0F0Fu>(x, lane);
  x = transpose_stage<2, 0x33333333u>(x, lane);
  return transpose_stage<1, 0x55555555u>(x, lane);
}

template <typename W>
__global__ void __launch_bounds__(kTfThreads, 2) k_tile_filter(const ScanArgs a, int chunk) {
  if (a.any_active != nullptr && *reinterpret_cast<const volatile uint32_t *>(a.any_active) == 0u) return;
  extern __shared__ uint4 tf_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // per warp, two buffers of one group's term words, [slot][8] each
  uint32_t *tabs = reinterpret_cast<uint32_t *>(tf_smem) + (size_t)warp * 2 * a.n_slots * 8;
  __shared__ const uint32_t *s_bm[kGemvMaxSlots];
  __shared__ unsigned long long s_pass[64];
  for (int i = threadIdx.x; i < a.n_slots; i += blockDim.x) s_bm[i] = a.slot_bm[i];
  for (int i = threadIdx.x; i < 64; i += blockDim.x) s_pass[i] = 0ull;
  __syncthreads();

  const int q0 = lane, q1 = lane + 32;
  const bool live0 = q0 < a.nq && (a.active == nullptr || a.active[a.q_base + q0] != 0u);
  const bool live1 = q1 < a.nq && (a.active == nullptr || a.active[a.q_base + q1] != 0u);
  const PackedCnf pk0 = live0 ? pack_cnf(a, q0) : PackedCnf{};
  const PackedCnf pk1 = live1 ? pack_cnf(a, q1) : PackedCnf{};
  const int64_t n_items = a.g_begin < a.n_groups ? (a.n_groups - a.g_begin + a.g_step - 1) / a.g_step : 0;
  const int64_t n_chunks = (n_items + chunk - 1) / chunk;
  const int64_t gw = (int64_t)blockIdx.x * kTfWarps + warp, n_w = (int64_t)gridDim.x * kTfWarps;
  unsigned long long pass0 = 0, pass1 = 0;

  // the warp's items, in order: chunks gw, gw + n_w, ...; `chunk` items each
  auto item_at = [&](int64_t c, int j) -> int64_t {
    const int64_t it = c * chunk + j;
    return c < n_chunks && it < n_items ? it : -1;
  };
  auto prefetch = [&](int64_t it, int buf) {
    if (it >= 0) {
      const int64_t g = a.g_begin + it * a.g_step;
      uint32_t *dst = tabs + (size_t)buf * a.n_slots * 8;
      for (int i = lane; i < 2 * a.n_slots; i += 32) {
        const int s = i >> 1, h = i & 1;
        cp_async16(dst + s * 8 + h * 4, s_bm[s] + g * kGroupWords + h * 4);
      }
    }
    cp_async_commit();
  };
  int buf = 0;
  prefetch(item_at(gw, 0), 0);
  for (int64_t c = gw; c < n_chunks; c += n_w) {
    uint32_t my_tile = 0, n_tiles = 0;  // lane j: the chunk's j-th listed tile
    for (int j = 0; j < chunk; ++j) {
      const int64_t it = item_at(c, j);
      if (it < 0) break;
      // words of the next item in flight while this one is evaluated
      prefetch(j + 1 < chunk ? item_at(c, j + 1) : item_at(c + n_w, 0), buf ^ 1);
      cp_async_wait_group<1>();
      __syncwarp();
      const uint32_t *tab = tabs + (size_t)buf * a.n_slots * 8;
      const int64_t g = a.g_begin + it * a.g_step;
      uint32_t pw0[8], pw1[8];
#pragma unroll
      for (int w = 0; w < 8; ++w) pw0[w] = pw1[w] = 0u;
      if (live0) {
        if (pk0.ok) eval_packed(pk0, tab, pw0);
        else eval_cnf(a, q0, tab, pw0);
      }
      if (live1) {
        if (pk1.ok) eval_packed(pk1, tab, pw1);
        else eval_cnf(a, q1, tab, pw1);
      }
      __syncwarp();  // every lane has read this buffer before it is refilled
      buf ^= 1;
      const int64_t r0 = g * kGroupRows;
      uint32_t any0 = 0, any1 = 0;
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        const int64_t left = a.n - (r0 + w * 32);
        const uint32_t valid = left >= 32 ? 0xFFFFFFFFu : (left > 0 ? ((1u << left) - 1u) : 0u);
        pw0[w] &= valid;
        pw1[w] &= valid;
        pass0 += (unsigned long long)__popc(pw0[w]);
        pass1 += (unsigned long long)__popc(pw1[w]);
        if (w < 4) any0 |= pw0[w] | pw1[w];
        else any1 |= pw0[w] | pw1[w];
      }
      const uint32_t fl = (__reduce_or_sync(0xFFFFFFFFu, any0) != 0u ? 1u : 0u) |
                          (__reduce_or_sync(0xFFFFFFFFu, any1) != 0u ? 2u : 0u);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!((fl >> h) & 1u)) continue;
        const uint32_t tile = (uint32_t)(g * 2 + h);  // tile id: rows 128 * id ..
        W *msg = static_cast<W *>(a.tile_msg) + (size_t)tile * 128;
#pragma unroll
        for (int w = 0; w < 4; ++w) {  // lane r: the queries that pass row 32w + r of the tile
          const uint32_t lo32 = bit_transpose32(pw0[4 * h + w], lane);
          if constexpr (sizeof(W) == 8) {
            const uint32_t hi32 = bit_transpose32(pw1[4 * h + w], lane);
            msg[w * 32 + lane] = ((uint64_t)hi32 << 32) | lo32;
          } else {
            msg[w * 32 + lane] = lo32;
          }
        }
        if ((uint32_t)lane == n_tiles) my_tile = tile;
        ++n_tiles;
      }
    }
    // append the chunk's tiles to the list: one atomic per chunk
    uint32_t base = 0;
    if (lane == 0 && n_tiles != 0u) base = atomicAdd(a.tile_cnt, n_tiles);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if ((uint32_t)lane < n_tiles) {
      if ((int64_t)base + lane < a.tile_cap) a.tile_row[base + lane] = (int32_t)my_tile;
      else atomicOr(a.err, kErrTileList);
    }
  }
  cp_async_wait_all();
  if (a.pass_cnt != nullptr) {
    if (live0 && pass0) atomicAdd(&s_pass[q0], pass0);
    if (live1 && pass1) atomicAdd(&s_pass[q1], pass1);
    __syncthreads();
    for (int q = threadIdx.x; q < a.nq && q < 64; q += blockDim.x)
      if (s_pass[q] != 0ull) atomicAdd(&a.pass_cnt[a.q_base + q], s_pass[q]);
  }
}

}  // namespace

cudaError_t launch_tile_filter(const ScanArgs &a, int max_grid, cudaStream_t s) {
  if (a.nq < 1 || a.nq > 64 || a.n_slots > kGemvMaxSlots) return cudaErrorInvalidValue;
  const int64_t n_items = a.g_begin < a.n_groups ? (a.n_groups - a.g_begin + a.g_step - 1) / a.g_step : 0;
  // chunks of up to kTfMaxChunk groups, smaller when that leaves warps idle
  const int64_t warps = (int64_t)max_grid * kTfWarps;
  const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(kTfMaxChunk, n_items / std::max<int64_t>(warps, 1)));
  const int64_t want = ((n_items + chunk - 1) / chunk + kTfWarps - 1) / kTfWarps;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, max_grid));
  const size_t smem = (size_t)kTfWarps * 2 * (a.n_slots > 0 ? a.n_slots : 1) * 32;
  auto *fn = a.nq <= 32 ? k_tile_filter<uint32_t> : k_tile_filter<uint64_t>;
  // the static shared memory (slot pointers, pass counts) counts against the
  // 48 KB default too: opt in well before the dynamic part alone reaches it
  if (smem > 32u * 1024u) {
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  fn<<<grid, kTfThreads, smem, s>>>(a, chunk);
  return cudaGetLastError();
}

}  // namespace lr
