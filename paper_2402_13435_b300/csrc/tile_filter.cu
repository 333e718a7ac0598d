// Tile filter: the term predicate (F-TBR) of a tensor-core scan, evaluated
// ahead of the scan for all 256-row groups it visits.
//
// Sec. 5.2 restricts the candidates of each query to the jobs whose terms
// satisfy its CNF; Sec. 5.3 fuses that restriction with the embedding scan so
// that rows no query accepts are never read.  Here the restriction runs as its
// own wide kernel, one warp per group and one lane per two queries, and writes
// for every 128-row tile that some query passes one list entry:
//     tile_row[i]        the tile's first row,
//     tile_msg[i][r]     the mask of the launch's queries that pass row r
//                        (bit q; 32-bit words when the launch has at most 32
//                        queries, else 64-bit).
// The scan then streams exactly the listed tiles, and its pipeline carries no
// predicate latency.  Entries are appended with one atomic per block
// iteration (eight groups), so their order follows the blocks' progress and is
// not the row order; the scan does not depend on it.  The per-query pass
// counts of the launch are accumulated here as well.
#include <algorithm>

#include "lr_internal.h"
#include "ptx.h"
#include "scan_common.cuh"

namespace lr {
namespace {

constexpr int kTfThreads = 256;
constexpr int kTfWarps = kTfThreads / 32;

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
__global__ void __launch_bounds__(kTfThreads, 2) k_tile_filter(const ScanArgs a) {
  if (a.any_active != nullptr && *reinterpret_cast<const volatile uint32_t *>(a.any_active) == 0u) return;
  extern __shared__ uint4 tf_smem[];
  // per warp: the group's term words, [slot][8]
  uint32_t *tab = reinterpret_cast<uint32_t *>(tf_smem) + (size_t)(threadIdx.x >> 5) * a.n_slots * 8;
  __shared__ const uint32_t *s_bm[kGemvMaxSlots];
  __shared__ unsigned long long s_pass[64];
  __shared__ uint32_t s_flag[kTfWarps], s_off[kTfWarps], s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < a.n_slots; i += blockDim.x) s_bm[i] = a.slot_bm[i];
  for (int i = threadIdx.x; i < 64; i += blockDim.x) s_pass[i] = 0ull;
  __syncthreads();

  const int q0 = lane, q1 = lane + 32;
  const bool live0 = q0 < a.nq && (a.active == nullptr || a.active[a.q_base + q0] != 0u);
  const bool live1 = q1 < a.nq && (a.active == nullptr || a.active[a.q_base + q1] != 0u);
  const PackedCnf pk0 = live0 ? pack_cnf(a, q0) : PackedCnf{};
  const PackedCnf pk1 = live1 ? pack_cnf(a, q1) : PackedCnf{};
  const int64_t n_items = a.g_begin < a.n_groups ? (a.n_groups - a.g_begin + a.g_step - 1) / a.g_step : 0;
  unsigned long long pass0 = 0, pass1 = 0;

  for (int64_t it = blockIdx.x; it * kTfWarps < n_items; it += gridDim.x) {
    const int64_t item = it * kTfWarps + warp;
    const int64_t g = a.g_begin + item * a.g_step;
    uint32_t pw0[8], pw1[8];
#pragma unroll
    for (int w = 0; w < 8; ++w) pw0[w] = pw1[w] = 0u;
    if (item < n_items) {
      for (int i = lane; i < 2 * a.n_slots; i += 32) {
        const int s = i >> 1, h = i & 1;
        cp_async16(tab + s * 8 + h * 4, s_bm[s] + g * kGroupWords + h * 4);
      }
      cp_async_commit();
      cp_async_wait_all();
      __syncwarp();
      if (live0) {
        if (pk0.ok) eval_packed(pk0, tab, pw0);
        else eval_cnf(a, q0, tab, pw0);
      }
      if (live1) {
        if (pk1.ok) eval_packed(pk1, tab, pw1);
        else eval_cnf(a, q1, tab, pw1);
      }
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
      __syncwarp();  // every lane has read the word table before the next group overwrites it
    }
    // tiles of this group that some query passes
    uint32_t any0 = 0, any1 = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      any0 |= pw0[w] | pw1[w];
      any1 |= pw0[4 + w] | pw1[4 + w];
    }
    const uint32_t fl = (__reduce_or_sync(0xFFFFFFFFu, any0) != 0u ? 1u : 0u) |
                        (__reduce_or_sync(0xFFFFFFFFu, any1) != 0u ? 2u : 0u);
    if (lane == 0) s_flag[warp] = fl;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t tot = 0;
      for (int w = 0; w < kTfWarps; ++w) {
        s_off[w] = tot;
        tot += __popc(s_flag[w]);
      }
      s_base = tot != 0u ? atomicAdd(a.tile_cnt, tot) : 0u;
      if ((int64_t)s_base + tot > a.tile_cap) atomicOr(a.err, kErrTileList);
    }
    __syncthreads();
    uint32_t idx = s_base + s_off[warp];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (!((fl >> h) & 1u)) continue;
      const bool fits = (int64_t)idx < a.tile_cap;
      if (lane == 0 && fits) a.tile_row[idx] = (int32_t)(g * kGroupRows + h * 128);
      W *msg = static_cast<W *>(a.tile_msg) + (size_t)idx * 128;
#pragma unroll
      for (int w = 0; w < 4; ++w) {  // lane r: the queries that pass row 32w + r of the tile
        const uint32_t lo32 = bit_transpose32(pw0[4 * h + w], lane);
        if constexpr (sizeof(W) == 8) {
          const uint32_t hi32 = bit_transpose32(pw1[4 * h + w], lane);
          if (fits) msg[w * 32 + lane] = ((uint64_t)hi32 << 32) | lo32;
        } else {
          if (fits) msg[w * 32 + lane] = lo32;
        }
      }
      ++idx;
    }
  }
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
  const int64_t want = (n_items + kTfWarps - 1) / kTfWarps;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, max_grid));
  const size_t smem = (size_t)kTfWarps * (a.n_slots > 0 ? a.n_slots : 1) * 32;
  if (a.nq <= 32) {
    auto *fn = k_tile_filter<uint32_t>;
    if (smem > 48u * 1024u) {
      const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    fn<<<grid, kTfThreads, smem, s>>>(a);
  } else {
    auto *fn = k_tile_filter<uint64_t>;
    if (smem > 48u * 1024u) {
      const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    fn<<<grid, kTfThreads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace lr
