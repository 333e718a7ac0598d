// Tile filter: the term predicate (F-TBR) of a tensor-core scan, evaluated
// ahead of the scan for all 256-row groups it visits.
//
// Sec. 5.2 restricts the candidates of each query to the jobs whose terms
// satisfy its CNF; Sec. 5.3 fuses that restriction with the embedding scan so
// that rows no query accepts are never read.  Here the restriction runs as its
// own wide kernel, one warp per group and one lane per two queries, and writes
// for every 128-row tile t that some query passes
//     tile_msg[t][r]     the mask of the launch's queries that pass row r
//                        (bit q; 32-bit words when the launch has at most 32
//                        queries, else 64-bit), stored at the tile's own slot,
// and appends t to the compact list tile_row[]; t = 2 i + h for tile h of the
// i-th group the launch visits (groups g_begin + i g_step), so a full pass
// numbers tiles by their rows and a sampled pass uses a compact range.  The scan then streams exactly
// the listed tiles, and its pipeline carries no predicate latency.  Up to 32
// queries every warp streams its own groups (global warp index, stride = all
// warps of the grid) with the next group's term words (32 bytes per term) in
// flight while it evaluates the current one, in its own double buffer, so no
// block-wide barrier couples the warps; up to 64 queries a block loads runs of
// eight consecutive groups together (256 contiguous bytes per term), one group
// per warp.  A warp appends its tiles with one atomic per eight groups, so the
// list order follows the warps' progress rather than the row order; the scan
// does not depend on it.  The per-query pass
// counts of the launch are accumulated here as well.
#include <algorithm>

#include "bits.cuh"
#include "lr_internal.h"
#include "ptx.h"
#include "scan_common.cuh"

namespace lr {
namespace {

constexpr int kTfThreads = 256;
constexpr int kTfWarps = kTfThreads / 32;
constexpr int kTfRun = kTfWarps;  // groups a block has in flight (one per warp)
constexpr int kTfAppend = 8;      // groups between a warp's list appends (16 tiles at most)

// W = uint32_t: at most 32 queries, one per lane; uint64_t: up to 64, two per lane.
template <typename W>
__global__ void __launch_bounds__(kTfThreads, sizeof(W) == 8 ? 2 : 3) k_tile_filter(const ScanArgs a) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
  constexpr bool kTwo = sizeof(W) == 8;
  if (a.any_active != nullptr && *reinterpret_cast<const volatile uint32_t *>(a.any_active) == 0u) return;
  extern __shared__ uint4 tf_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // two buffers of term words per warp ([slot][8] each, up to 32 queries) or
  // per block ([group of the run][slot][8] each, up to 64): the same bytes;
  // then the launch's clause lists (qc, cl, cs), staged once per block
  const size_t run_words = (size_t)kTfRun * a.n_slots * 8;
  uint32_t *tabs = reinterpret_cast<uint32_t *>(tf_smem);
  int32_t *s_qc = reinterpret_cast<int32_t *>(tf_smem) + 2 * run_words;
  int32_t *s_cl = s_qc + a.nq + 1;
  int32_t *s_cs = s_cl + a.n_cl + 1;
  __shared__ const uint32_t *s_bm[kGemvMaxSlots];
  __shared__ unsigned long long s_pass[64];
  for (int i = threadIdx.x; i < a.n_slots; i += blockDim.x) s_bm[i] = a.slot_bm[i];
  for (int i = threadIdx.x; i < 64; i += blockDim.x) s_pass[i] = 0ull;
  for (int i = threadIdx.x; i <= a.nq; i += blockDim.x) s_qc[i] = a.qc_off[i];
  for (int i = threadIdx.x; i <= a.n_cl; i += blockDim.x) s_cl[i] = a.cl_off[i];
  for (int i = threadIdx.x; i < a.n_tm; i += blockDim.x) s_cs[i] = a.cl_slot[i];
  __syncthreads();

  const int64_t n_items = a.g_begin < a.n_groups ? (a.n_groups - a.g_begin + a.g_step - 1) / a.g_step : 0;
  // Up to 32 queries (three blocks per SM): every warp streams its own groups
  // (global warp index, stride = all warps), double buffering their term words
  // in its own part of shared memory, so no block-wide barrier separates one
  // group from the next.  Up to 64 queries (more terms, so fewer blocks per
  // SM): the block loads runs of kTfRun consecutive groups together (per slot
  // the run's words are 256 contiguous bytes), one group per warp, the next
  // run in flight while it evaluates the current one; with few warps per SM the
  // per-warp 32-byte copies measured slower there.
  const int64_t gw = (int64_t)blockIdx.x * kTfWarps + warp, nw = (int64_t)gridDim.x * kTfWarps;
  const int64_t n_runs = (n_items + kTfRun - 1) / kTfRun;
  uint32_t *wtab = tabs + (size_t)warp * 2 * a.n_slots * 8;
  auto prefetch = [&](int64_t it, int buf) {  // the group's 32 bytes of every slot
    uint32_t *dst = wtab + (size_t)buf * a.n_slots * 8;
    const size_t goff = (size_t)(a.g_begin + it * a.g_step) * kGroupWords;
    for (int i = lane; i < a.n_slots * 2; i += 32) {
      const int sl = i >> 1, h = i & 1;
      cp_async16(dst + sl * 8 + h * 4, s_bm[sl] + goff + h * 4);
    }
    cp_async_commit();
  };
  auto prefetch_run = [&](int64_t run, int buf) {  // [group of the run][slot][8]
    uint32_t *dst = tabs + (size_t)buf * run_words;
    for (int i = threadIdx.x; i < a.n_slots * kTfRun * 2; i += blockDim.x) {
      const int sl = i / (kTfRun * 2), p = i % (kTfRun * 2), gl = p >> 1, h = p & 1;
      const int64_t it = run * kTfRun + gl;
      if (it < n_items)
        cp_async16(dst + ((size_t)gl * a.n_slots + sl) * 8 + h * 4,
                   s_bm[sl] + (a.g_begin + it * a.g_step) * kGroupWords + h * 4);
    }
    cp_async_commit();
  };
  if constexpr (!kTwo) {  // in flight while the CNFs are packed
    if (gw < n_items) prefetch(gw, 0);
  } else {
    if ((int64_t)blockIdx.x < n_runs) prefetch_run(blockIdx.x, 0);
  }

  const int q0 = lane, q1 = lane + 32;
  const bool live0 = q0 < a.nq && (a.active == nullptr || a.active[a.q_base + q0] != 0u);
  const bool live1 = kTwo && q1 < a.nq && (a.active == nullptr || a.active[a.q_base + q1] != 0u);
  const PackedCnf pk0 = live0 ? pack_cnf_lists(s_qc, s_cl, s_cs, q0) : PackedCnf{};
  const PackedCnf pk1 = kTwo && live1 ? pack_cnf_lists(s_qc, s_cl, s_cs, q1) : PackedCnf{};
  unsigned long long pass0 = 0, pass1 = 0;
  uint32_t my_tile = 0, n_tiles = 0;  // lane j: the j-th tile this warp has not appended yet
  auto append = [&]() {  // one atomic for up to 2 * kTfAppend tiles
    uint32_t base = 0;
    if (lane == 0 && n_tiles != 0u) base = atomicAdd(a.tile_cnt, n_tiles);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if ((uint32_t)lane < n_tiles) {
      if ((int64_t)base + lane < a.tile_cap) a.tile_row[base + lane] = (int32_t)my_tile;
      else atomicOr(a.err, kErrTileList);
    }
    n_tiles = 0u;
  };

  // one group: CNFs of the launch's queries on its words (tab: [slot][8]),
  // pass counts, row masks and list entries of its passing tiles
  auto process = [&](int64_t it, const uint32_t *tab) {
    const int64_t g = a.g_begin + it * a.g_step;
    uint32_t pw0[8], pw1[8];
#pragma unroll
    for (int w = 0; w < 8; ++w) pw0[w] = pw1[w] = 0u;
    if (live0) {
      if (pk0.ok) eval_packed(pk0, tab, pw0);
      else eval_cnf_lists(s_qc, s_cl, s_cs, q0, tab, pw0);
    }
    if constexpr (kTwo) {
      if (live1) {
        if (pk1.ok) eval_packed(pk1, tab, pw1);
        else eval_cnf_lists(s_qc, s_cl, s_cs, q1, tab, pw1);
      }
    }
    const int64_t r0 = g * kGroupRows;
    if (r0 + kGroupRows > a.n) {  // the index's last group: rows past n do not exist
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        const int64_t left = a.n - (r0 + w * 32);
        const uint32_t valid = left >= 32 ? 0xFFFFFFFFu : (left > 0 ? ((1u << left) - 1u) : 0u);
        pw0[w] &= valid;
        pw1[w] &= valid;
      }
    }
    uint32_t any0 = 0, any1 = 0, c0 = 0, c1 = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      c0 += (uint32_t)__popc(pw0[w]);
      if constexpr (kTwo) c1 += (uint32_t)__popc(pw1[w]);
      if (w < 4) any0 |= pw0[w] | (kTwo ? pw1[w] : 0u);
      else any1 |= pw0[w] | (kTwo ? pw1[w] : 0u);
    }
    pass0 += c0;
    pass1 += c1;
    const uint32_t fl = (__reduce_or_sync(0xFFFFFFFFu, any0) != 0u ? 1u : 0u) |
                        (__reduce_or_sync(0xFFFFFFFFu, any1) != 0u ? 2u : 0u);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (!a.dense_tiles && !((fl >> h) & 1u)) continue;  // dense: every tile's masks, zero or not
      if ((int64_t)(it * 2 + h) >= a.tile_cap) {  // the list buffers are smaller than the visit
        if (lane == 0) atomicOr(a.err, kErrTileList);
        continue;
      }
      // tile id: tile h of the it-th visited group (for a full pass, rows
      // 128 id ..); ids stay below 2 x the groups visited <= tile_cap
      const uint32_t tile = (uint32_t)(it * 2 + h);
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
      if (a.dense_tiles) continue;  // no list: the scan visits every tile
      if ((uint32_t)lane == n_tiles) my_tile = tile;
      ++n_tiles;
    }
  };

  int buf = 0, since = 0;
  if constexpr (!kTwo) {
    for (int64_t it = gw; it < n_items; it += nw) {
      if (it + nw < n_items) {
        prefetch(it + nw, buf ^ 1);  // every lane finished reading that buffer last group
        cp_async_wait_group<1>();
      } else {
        cp_async_wait_group<0>();
      }
      __syncwarp();  // every lane's copies of this group have landed
      process(it, wtab + (size_t)buf * a.n_slots * 8);
      __syncwarp();  // every lane is done with this buffer before it is refilled
      buf ^= 1;
      if (++since == kTfAppend) {
        append();
        since = 0;
      }
    }
  } else {
    for (int64_t run = blockIdx.x; run < n_runs; run += gridDim.x) {
      cp_async_wait_all();
      __syncthreads();  // the run's words are visible, and every warp is done with the other buffer
      if (run + gridDim.x < n_runs) prefetch_run(run + gridDim.x, buf ^ 1);
      const int64_t it = run * kTfRun + warp;
      if (it < n_items) process(it, tabs + (size_t)buf * run_words + (size_t)warp * a.n_slots * 8);
      buf ^= 1;
      if (++since == kTfAppend) {
        append();
        since = 0;
      }
    }
  }
  append();
  cp_async_wait_all();
  if (a.pass_cnt != nullptr) {
    if (live0 && pass0) atomicAdd(&s_pass[q0], pass0);
    if (kTwo && live1 && pass1) atomicAdd(&s_pass[q1], pass1);
    __syncthreads();
    for (int q = threadIdx.x; q < a.nq && q < 64; q += blockDim.x)
      if (s_pass[q] != 0ull) atomicAdd(&a.pass_cnt[a.q_base + q], s_pass[q]);
  }
}

}  // namespace

cudaError_t launch_tile_filter(const ScanArgs &a, int num_sms, cudaStream_t s) {
  if (a.nq < 1 || a.nq > 64 || a.n_slots > kGemvMaxSlots) return cudaErrorInvalidValue;
  const int64_t n_items = a.g_begin < a.n_groups ? (a.n_groups - a.g_begin + a.g_step - 1) / a.g_step : 0;
  const int64_t runs = (n_items + kTfRun - 1) / kTfRun;
  const int per_sm = a.nq <= 32 ? 3 : 2;  // resident blocks per SM (registers)
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(runs, (int64_t)num_sms * per_sm));
  const size_t smem = (size_t)2 * kTfRun * (a.n_slots > 0 ? a.n_slots : 1) * 32 +
                      (size_t)(a.nq + 1 + a.n_cl + 1 + a.n_tm) * sizeof(int32_t);
  // dense masks feed a two-block scan, which reads 64-bit masks whatever the block's size
  auto *fn = a.nq <= 32 && !a.dense_tiles ? k_tile_filter<uint32_t> : k_tile_filter<uint64_t>;
  // the static shared memory (slot pointers, pass counts) counts against the
  // 48 KB default too: opt in well before the dynamic part alone reaches it
  if (smem > 32u * 1024u) {
    const cudaError_t e = allow_dynamic_smem((const void *)fn, (size_t)smem);
    if (e != cudaSuccess) return e;
  }
  return launch_pdl(fn, dim3((unsigned)grid), dim3(kTfThreads), smem, s, a);
}

}  // namespace lr
