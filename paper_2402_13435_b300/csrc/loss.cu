// Masked in-batch / sampled softmax loss of the retrieval towers and its
// gradients on the tensor cores (Sec. 5.1, Eq. 1 and Eq. 2).
//
//   z_ij = inv_tau <q_i, j_j>, over the columns j allowed for query i (the job
//          satisfies the query's term constraint, or j is the query's positive)
//   L    = (1/B) sum_i ( logsumexp_j z_ij - z_i,pos(i) )
//   dZ_ij = (dL/B) (softmax_ij - [j = pos(i)]) on allowed columns, 0 elsewhere
//   dQ = inv_tau dZ J,   dJ = inv_tau dZ^T Q
//
// The B x M logits are never stored: every pass recomputes its score tile on
// the tensor cores (BF16 operands, FP32 accumulation in tensor memory).  One
// kernel template serves three passes over tiles of a resident 128-row
// operand R against streamed 64-row tiles of an operand C:
//   kFwd: R = queries, C = jobs; online log-sum-exp per query row.
//   kDq:  R = queries, C = jobs; dZ tile -> acc[128 x d] += dZ C, with C's
//         transposed copy as the K-major B operand.
//   kDj:  R = jobs, C = queries; the same with dZ^T, acc[128 x d] += dZ^T Q.
//   kKeys: R = queries, C = jobs; the raw scores <q_i, j_j> of every allowed
//         negative (allowed column, not the positive) appended to the query's
//         key list as selection keys (ordered score, ~column) -- the in-batch
//         hard-negative mining of Sec. 5.1 ranks them.
// dZ enters the second product as two BF16 terms (hi + lo, near-FP32 accuracy).
// Warps 0-3: epilogue (TMEM lane quarters); warp 4: TMA; warp 5: MMA issue.
// Every wait is bounded; a timeout sets the status word.
#include <cuda.h>
#include <cuda_bf16.h>

#include "bits.cuh"
#include "lr_internal.h"
#include "ptx.h"

namespace lr {
namespace {

constexpr int kRRows = 128;     // rows of the resident tile
constexpr int kCRows = 64;      // rows of a streamed tile
constexpr int kLossThreads = 320;  // warps 0-3 and 6-9: two epilogue sets; 4: TMA; 5: MMA
constexpr int kLossFwdThreads = 192;  // the forward: one epilogue set
constexpr int kCBufs = 3;          // streamed-tile buffers: a tile loads while the two before it are in use
constexpr uint32_t kLossTmemCols = 256;  // 2 score tiles of 64 columns + accumulator (<= 128)
// backward passes at dp = 128: the second product runs transposed (the
// accumulator is [dp lanes][hi rows | lo rows], 256 columns), so 512 columns
constexpr uint32_t kLossTmemColsT = 512;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// 2^x on the special-function unit (ex2.approx: relative error ~2^-22; 2^-inf = 0).
// The epilogues work in log2 units -- z2 = s * inv_tau * log2(e) by one
// multiply(-add) -- so each exponential is this one instruction.
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

enum LossMode : int { kFwd = 0, kDq = 1, kDj = 2, kKeys = 3 };

struct LossSmem {
  size_t r, c, ct, dz, stage, bars, holder, total;
};

// kDj staging of one query tile for the epilogue: mask words of the CTA's 128
// job rows (4 per query), positives and log-sum-exps of the tile's 64 queries
struct DjStage {
  uint32_t mask[kCRows * 4];
  int32_t pos[kCRows];
  float lse[kCRows];
};

__host__ __device__ inline LossSmem loss_smem(int dp, int mode) {
  LossSmem L;
  size_t off = 0;
  L.r = off;
  off += (size_t)(dp / 64) * kRRows * 128;  // K-blocks of 128 rows x 128 bytes
  L.c = off;
  off += (size_t)kCBufs * (dp / 64) * kCRows * 128;
  L.ct = off;
  const bool one_product = mode == kFwd || mode == kKeys;
  off += one_product ? 0 : (size_t)kCBufs * dp * 128;  // transposed C tile: dp rows x 64 values
  L.dz = off;
  off += one_product ? 0 : (size_t)2 * 2 * kRRows * 128;  // [buffer][hi, lo] 128 rows x 64 values
  L.stage = off;
  off += mode == kDj ? 4 * sizeof(DjStage) : 0;  // two per epilogue set
  L.bars = off;
  off += 16 * 8;
  L.holder = off;
  L.total = off + 16;
  return L;
}

__device__ __forceinline__ bool wwait(uint64_t *bar, uint32_t parity, int lane) {
  bool got = true;
  if (lane == 0) got = mbar_wait(bar, parity);
  return __shfl_sync(0xFFFFFFFFu, got ? 1 : 0, 0) != 0;
}

template <int MODE>
__global__ void __launch_bounds__(kLossThreads, 1)
    k_loss(const LossArgs a, const __grid_constant__ CUtensorMap tm_r, const __grid_constant__ CUtensorMap tm_c,
           const __grid_constant__ CUtensorMap tm_ct) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  constexpr bool kOne = MODE == kFwd || MODE == kKeys;  // the score product only
  const int dp = a.dp;
  const LossSmem L = loss_smem(dp, MODE);
  const int KB = dp / 64;  // 64-value K-blocks of the score product
  unsigned char *sr = smem + L.r;
  unsigned char *sc = smem + L.c;
  unsigned char *sct = smem + L.ct;
  unsigned char *sdz = smem + L.dz;
  DjStage *stg = reinterpret_cast<DjStage *>(smem + L.stage);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.bars);
  uint64_t *bar_r = bars, *c_full = bars + 1, *c_empty = bars + 1 + kCBufs;  // [kCBufs] each
  uint64_t *s_full = bars + 1 + 2 * kCBufs, *s_empty = s_full + 2;               // [2]: one per epilogue set
  uint64_t *dz_full = s_empty + 2, *dz_empty = dz_full + 2, *acc_full = dz_empty + 2;
  uint32_t *holder = reinterpret_cast<uint32_t *>(smem + L.holder);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r0 = blockIdx.x * kRRows;
  const int t0 = blockIdx.y * a.c_per_split;
  const int T = min(a.c_per_split, a.n_ctiles - t0);  // streamed tiles of this CTA (>= 1 by construction)
  const size_t c_bytes = (size_t)KB * kCRows * 128;
  const size_t ct_bytes = (size_t)dp * 128;
  // Backward passes with dp = 128: acc^T[k][r | 128 + r] += C^T[k][c] .
  // [dZ_hi ; dZ_lo][r][c] as ONE MMA of N = 256 per 16-value K step (the
  // transposed C tile as A, the stacked hi / lo dZ rows as B) instead of two
  // MMAs of N = 128 with dZ_hi and dZ_lo as A: an MMA costs about the same
  // whatever its width up to 128 columns, so the product issues half the
  // instructions.  The write-out adds the two halves.
  const bool swap = !kOne && dp == 128;
  const uint32_t tmem_cols = swap ? kLossTmemColsT : kLossTmemCols;

  if (threadIdx.x == 0) {
    mbar_init(bar_r, 1);
    for (int i = 0; i < kCBufs; ++i) {
      mbar_init(&c_full[i], 1);
      mbar_init(&c_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&s_full[i], 1);
      mbar_init(&s_empty[i], 4);
      mbar_init(&dz_full[i], 4);
      mbar_init(&dz_empty[i], 1);
    }
    mbar_init(acc_full, 1);
    fence_mbar_init();
  }
  if (warp == 5) {
    tmem_alloc(holder, tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *holder;
  bool ok = true;

  if (warp == 4) {
    // ---------------------------------------------------------------- TMA
    if (lane == 0) {
      int issued = 0;
      mbar_arrive_expect_tx(bar_r, (uint32_t)(KB * kRRows * 128));
      for (int kb = 0; kb < KB; ++kb) tma_load_2d(sr + (size_t)kb * kRRows * 128, &tm_r, kb * 64, r0, bar_r);
      for (int t = 0; t < T && ok; ++t) {
        const int b = t % kCBufs;
        if (!mbar_wait(&c_empty[b], (uint32_t)((t / kCBufs) & 1) ^ 1u)) {
          ok = false;
          break;
        }
        const int c0 = (t0 + t) * kCRows;
        mbar_arrive_expect_tx(&c_full[b], (uint32_t)(c_bytes + (kOne ? 0 : ct_bytes)));
        for (int kb = 0; kb < KB; ++kb)
          tma_load_2d(sc + (size_t)b * c_bytes + (size_t)kb * kCRows * 128, &tm_c, kb * 64, c0, &c_full[b]);
        if (!kOne) tma_load_2d(sct + (size_t)b * ct_bytes, &tm_ct, c0, 0, &c_full[b]);
        issued = t + 1;
      }
      if (!ok) {
        atomicOr(a.status, kErrTimeout);
        mbar_wait(bar_r, 0u);  // let issued loads land
        for (int t = issued > kCBufs ? issued - kCBufs : 0; t < issued; ++t)
          mbar_wait(&c_full[t % kCBufs], (uint32_t)((t / kCBufs) & 1));
      }
    }
    __syncwarp();
  } else if (warp == 5) {
    // ---------------------------------------------------------------- MMA
    if (lane == 0) {
      const uint32_t id_s = idesc_bf16(kRRows, kCRows), id_g = idesc_bf16(kRRows, dp);
      const uint32_t id_t = idesc_bf16(128, 2 * kRRows);  // the transposed product: M = dp = 128, N = 256
      const uint32_t acc = tmem + 2u * kCRows;
      bool issued = false;
      auto issue_s = [&](int t) -> bool {
        const int b = t & 1, cb = t % kCBufs;  // score buffer (the epilogue set's), streamed-tile buffer
        if (!mbar_wait(&c_full[cb], (uint32_t)((t / kCBufs) & 1))) return false;
        if (!mbar_wait(&s_empty[b], (uint32_t)((t >> 1) & 1) ^ 1u)) return false;
        tc_fence_after();
        const uint32_t ra = smem_u32(sr), ca = smem_u32(sc + (size_t)cb * c_bytes);
        for (int k = 0; k < dp / 16; ++k) {
          const uint32_t koff = (uint32_t)(k & 3) * 32u;
          mma_bf16(tmem + (uint32_t)(b * kCRows), sw128_desc(ra + (uint32_t)(k >> 2) * (kRRows * 128) + koff),
                   sw128_desc(ca + (uint32_t)(k >> 2) * (kCRows * 128) + koff), id_s, k > 0 ? 1u : 0u);
        }
        issued = true;
        mma_commit(&s_full[b]);
        if (kOne) mma_commit(&c_empty[cb]);
        return true;
      };
      if (!mbar_wait(bar_r, 0u)) ok = false;
      if (ok && T > 0) ok = issue_s(0);
      for (int t = 0; t < T && ok; ++t) {
        if (t + 1 < T && !issue_s(t + 1)) {
          ok = false;
          break;
        }
        if (!kOne) {
          const int b = t & 1;
          if (!mbar_wait(&dz_full[b], (uint32_t)((t >> 1) & 1))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dh = smem_u32(sdz + (size_t)(2 * b) * kRRows * 128);
          const uint32_t dl = smem_u32(sdz + (size_t)(2 * b + 1) * kRRows * 128);
          const uint32_t ct = smem_u32(sct + (size_t)(t % kCBufs) * ct_bytes);
          if (swap) {  // dh and dl are adjacent: 256 rows of one K-major operand
#pragma unroll
            for (int k = 0; k < 4; ++k)  // K = the tile's 64 streamed rows
              mma_bf16(acc, sw128_desc(ct + (uint32_t)k * 32u), sw128_desc(dh + (uint32_t)k * 32u), id_t,
                       (t | k) != 0 ? 1u : 0u);
          } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {  // K = the tile's 64 streamed rows
              mma_bf16(acc, sw128_desc(dh + (uint32_t)k * 32u), sw128_desc(ct + (uint32_t)k * 32u), id_g,
                       (t | k) != 0 ? 1u : 0u);
              mma_bf16(acc, sw128_desc(dl + (uint32_t)k * 32u), sw128_desc(ct + (uint32_t)k * 32u), id_g, 1u);
            }
          }
          mma_commit(&dz_empty[b]);
          mma_commit(&c_empty[t % kCBufs]);
        }
      }
      if (issued) {  // every MMA has completed before the epilogue reads the accumulator / TMEM is freed
        mma_commit(acc_full);
        if (!mbar_wait(acc_full, 0u)) ok = false;
      } else {
        mbar_arrive(acc_full);
      }
      if (!ok) atomicOr(a.status, kErrTimeout);
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------------- epilogue
    // two sets of four warps (0-3 and 6-9) take alternate streamed tiles: set e
    // takes tiles e, e + 2, ..., so score buffer e and dZ buffer e are its own
    // and their barrier phases come in order; warp w reads tensor-memory lanes
    // 32 (w % 4) ..
    // the forward epilogue is issue-bound with one set, and two CTAs of 192
    // threads share an SM: it launches without warps 6-9
    constexpr int kSets = kOne ? 1 : 2;
    const int eset = warp >= 6 ? 1 : 0, quarter = warp & 3;
    const bool active = eset < kSets;
    const int r = quarter * 32 + lane;
    const int grow = r0 + r;
    const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
    // row identity: query (kFwd, kDq) or job (kDj)
    const bool rvalid = MODE == kDj ? grow < a.M : grow < a.B;
    int pos_row = -1;
    float lse_row = 0.f;
    if (MODE != kDj && rvalid) {
      pos_row = a.pos[grow];
      if (MODE == kDq) lse_row = a.lse[grow] * kLog2e;  // log2 units
    }
    float m = -INFINITY, ssum = 0.f, zpos = 0.f;
    bool have_pos = false;
    // Mask words (and for kDj the query tile's positives and lse) are fetched
    // one tile of the set ahead.  kFwd/kDq: this row's two words, in registers.
    // kDj: the set's 128 threads stage the query tile in shared memory (double
    // buffered per set; each iteration ends at the set's named barrier, which
    // every warp of the set reaches, also after a failed wait, so no warp
    // waits forever).
    uint32_t nw0 = ~0u, nw1 = ~0u;  // kFwd/kDq: next tile's mask words
    uint32_t sm0 = 0u, sm1 = 0u;    // kDj: this thread's share of the next stage
    int spos = -1;
    float slse = 0.f;
    auto fetch_row_words = [&](int tt) {
      const int cc0 = (t0 + tt) * kCRows;
      nw0 = nw1 = ~0u;
      if (rvalid && a.mask != nullptr && cc0 < a.M) {
        const uint32_t *mrow = a.mask + (size_t)grow * a.Mw + (cc0 >> 5);
        nw0 = __ldg(mrow);
        nw1 = (cc0 >> 5) + 1 < a.Mw ? __ldg(mrow + 1) : 0u;
      }
    };
    auto fetch_stage = [&](int tt) {
      const int cc0 = (t0 + tt) * kCRows;
      uint32_t v[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int i = r + k * kRRows;
        const int q = cc0 + (i >> 2), w = (r0 >> 5) + (i & 3);
        v[k] = q < a.B && w < a.Mw ? (a.mask != nullptr ? __ldg(a.mask + (size_t)q * a.Mw + w) : ~0u) : 0u;
      }
      sm0 = v[0];
      sm1 = v[1];
      const int q = cc0 + r;
      spos = (r < kCRows && q < a.B) ? __ldg(a.pos + q) : -1;
      slse = (r < kCRows && q < a.B) ? __ldg(a.lse + q) * kLog2e : 0.f;  // log2 units
    };
    auto store_stage = [&](int buf) {
      DjStage &st = stg[buf];
      st.mask[r] = sm0;
      st.mask[r + kRRows] = sm1;
      if (r < kCRows) {
        st.pos[r] = spos;
        st.lse[r] = slse;
      }
    };
    auto set_barrier = [&]() { asm volatile("bar.sync %0, 128;" ::"r"(1 + eset) : "memory"); };
    if (MODE == kDj) {
      if (eset < T) {
        fetch_stage(eset);
        store_stage(2 * eset);
      }
      set_barrier();
    } else if (active && eset < T) {
      fetch_row_words(eset);
    }
    for (int t = eset, it = 0; active && t < T; t += kSets, ++it) {
      const int b = t & 1;                 // two sets: == eset
      const int sb = 2 * eset + (it & 1);  // kDj: this tile's stage
      const int c0 = (t0 + t) * kCRows;
      const uint32_t cw0 = nw0, cw1 = nw1;
      if (t + kSets < T) {
        if (MODE == kDj) fetch_stage(t + kSets);
        else fetch_row_words(t + kSets);
      }
      do {
      if (!ok) break;
      if (!wwait(&s_full[b], (uint32_t)((t >> 1) & 1), lane)) {
        ok = false;
        break;
      }
      tc_fence_after();
      uint32_t sv[64];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t (&part)[16] = *reinterpret_cast<uint32_t (*)[16]>(&sv[16 * q]);
        tmem_ld16(trow + (uint32_t)(b * kCRows + 16 * q), part);
      }
      tmem_ld_wait();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&s_empty[b]);
      // allowed columns of this tile: bit c of al[c / 32]; kDj also the
      // columns whose positive is this row's job: bit c of pm[c / 32]
      uint32_t al[2] = {0u, 0u}, pm[2] = {0u, 0u};
      if (MODE == kDj) {
        // the tile's 64 queries x this warp's 32 jobs as two 32 x 32 bit
        // matrices, one query per lane (lane, lane + 32), transposed so that
        // lane r holds its job's column
        const DjStage &st = stg[sb];
        const int wj = (r0 >> 5) + quarter;
        uint32_t mw[2], pw[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int p = st.pos[lane + 32 * h];
          pw[h] = (p >= 0 && (p >> 5) == wj) ? 1u << (p & 31) : 0u;
          mw[h] = st.mask[(lane + 32 * h) * 4 + quarter] | pw[h];  // the positive is always allowed
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // every lane takes part in the transposes
          pm[h] = bit_transpose32(pw[h], lane);
          const uint32_t t = bit_transpose32(mw[h], lane);
          al[h] = rvalid ? t : 0u;
        }
      } else if (rvalid) {
        uint32_t w0 = cw0, w1 = cw1;
        const int lim = a.M - c0;  // columns past M do not exist
        w0 &= lim >= 32 ? ~0u : (lim > 0 ? ((1u << lim) - 1u) : 0u);
        w1 &= lim >= 64 ? ~0u : (lim > 32 ? ((1u << (lim - 32)) - 1u) : 0u);
        const int pc = pos_row - c0;
        if (pc >= 0 && pc < 32) w0 |= 1u << pc;
        if (pc >= 32 && pc < 64) w1 |= 1u << (pc - 32);
        al[0] = w0;
        al[1] = w1;
      }
      if (MODE == kFwd) {
        if (pos_row >= c0 && pos_row < c0 + 64) {
          const int pc = pos_row - c0;
#pragma unroll
          for (int c = 0; c < 64; ++c)
            if (c == pc) zpos = __uint_as_float(sv[c]) * a.inv_tau;
          have_pos = true;
        }
        // the running maximum m is in log2 units; failing columns become -inf,
        // whose exponential is 0
        const float c2 = a.inv_tau * kLog2e;
        float tmax = -INFINITY;
#pragma unroll
        for (int c = 0; c < 64; ++c) {
          const float z2 = ((al[c >> 5] >> (c & 31)) & 1u) ? __uint_as_float(sv[c]) * c2 : -INFINITY;
          sv[c] = __float_as_uint(z2);
          tmax = fmaxf(tmax, z2);
        }
        if (tmax > -INFINITY) {
          const float mn = fmaxf(m, tmax);
          float add = 0.f;
#pragma unroll
          for (int c = 0; c < 64; ++c) add += ex2_approx(__uint_as_float(sv[c]) - mn);
          ssum = ssum * ex2_approx(m - mn) + add;
          m = mn;
        }
      } else if (MODE == kKeys) {
        if (rvalid) {
          // allowed columns without the positive (al has no column past M),
          // appended to the row's key list in place of the tile's range
          uint32_t nb[2] = {al[0], al[1]};
          const int pc = pos_row - c0;
          if (pc >= 0 && pc < 32) nb[0] &= ~(1u << pc);
          if (pc >= 32 && pc < 64) nb[1] &= ~(1u << (pc - 32));
          const uint32_t cntk = (uint32_t)(__popc(nb[0]) + __popc(nb[1]));
          if (cntk) {
            uint32_t o = atomicAdd(&a.key_cnt[grow], cntk);
            uint64_t *krow = a.keys + (size_t)grow * (size_t)a.keys_ld;
#pragma unroll
            for (int c = 0; c < 64; ++c)
              if ((nb[c >> 5] >> (c & 31)) & 1u) krow[o++] = make_key(__uint_as_float(sv[c]), (uint32_t)(c0 + c));
          }
        }
      } else {
        // dZ of this tile as two BF16 terms, written in the 128-byte-swizzled K-major layout
        if (!wwait(&dz_empty[b], (uint32_t)((t >> 1) & 1) ^ 1u, lane)) {
          ok = false;
          break;
        }
        unsigned char *dh = sdz + (size_t)(2 * b) * kRRows * 128 + (size_t)r * 128;
        unsigned char *dl = sdz + (size_t)(2 * b + 1) * kRRows * 128 + (size_t)r * 128;
        const float g = (a.dloss != nullptr ? __ldg(a.dloss) : 1.f) * a.inv_b;
        const float c2 = a.inv_tau * kLog2e;
        const int pc = pos_row - c0;  // kDq: the positive's column in this tile
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
          uint32_t hw[4], lw[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            float dz2[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int c = ch * 8 + u * 2 + h;
              float lse, ispos;  // lse in log2 units
              if (MODE == kDq) {
                lse = lse_row;
                ispos = c == pc ? 1.f : 0.f;
              } else {
                lse = stg[sb].lse[c];
                ispos = ((pm[c >> 5] >> (c & 31)) & 1u) ? 1.f : 0.f;
              }
              const float dz = (ex2_approx(fmaf(__uint_as_float(sv[c]), c2, -lse)) - ispos) * g;
              dz2[h] = ((al[c >> 5] >> (c & 31)) & 1u) ? dz : 0.f;
            }
            const __nv_bfloat162 hv = __float22bfloat162_rn(make_float2(dz2[0], dz2[1]));
            const float2 hf = __bfloat1622float2(hv);
            const __nv_bfloat162 lv = __float22bfloat162_rn(make_float2(dz2[0] - hf.x, dz2[1] - hf.y));
            hw[u] = *reinterpret_cast<const uint32_t *>(&hv);
            lw[u] = *reinterpret_cast<const uint32_t *>(&lv);
          }
          const int slot = ((ch ^ (r & 7)) & 7) << 4;
          *reinterpret_cast<uint4 *>(dh + slot) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          *reinterpret_cast<uint4 *>(dl + slot) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&dz_full[b]);
      }
      } while (0);
      if (MODE == kDj) {  // the set's next stage, then this tile's barrier (every iteration, every warp of the set)
        if (t + 2 < T) store_stage(2 * eset + ((it + 1) & 1));
        set_barrier();
      }
    }
    if (MODE == kFwd) {  // one set: the row's log-sum-exp partial of this split
      if (rvalid) {
        a.part_m[(size_t)blockIdx.y * a.rows_p + grow] = m * kLn2;  // natural units for the combine
        a.part_s[(size_t)blockIdx.y * a.rows_p + grow] = ssum;
        if (have_pos) a.zpos[grow] = zpos;
      }
    } else if (MODE == kKeys) {
    } else if (eset == 0) {  // set 0 writes the accumulated rows
      if (!wwait(acc_full, 0u, lane)) ok = false;
      tc_fence_after();
      const uint32_t acc = trow + 2u * kCRows;
      if (swap) {
        // lane k (= this thread's TMEM lane) holds column k of every row: rows
        // r and 128 + r are the hi and lo halves; a warp's 32 lanes write 32
        // consecutive columns of a row
        const int k = quarter * 32 + lane;
        float *ocol = a.out + (size_t)blockIdx.y * a.out_split + k;
        const int rows_ok = MODE == kDq ? a.rows_p : a.M;
        for (int rr = 0; rr < kRRows; rr += 16) {
          uint32_t vh[16], vl[16];
          tmem_ld16(acc + (uint32_t)rr, vh);
          tmem_ld16(acc + (uint32_t)(kRRows + rr), vl);
          tmem_ld_wait();
          if (ok && k < a.out_cols)
#pragma unroll
            for (int i = 0; i < 16; ++i)
              if (r0 + rr + i < rows_ok)
                ocol[(size_t)(r0 + rr + i) * a.out_ld] = (__uint_as_float(vh[i]) + __uint_as_float(vl[i])) * a.inv_tau;
        }
      } else {
        float *orow = a.out + (size_t)blockIdx.y * a.out_split + (size_t)grow * a.out_ld;
        const bool wr = ok && (MODE == kDq ? grow < a.rows_p : grow < a.M);
        for (int c = 0; c < dp; c += 16) {
          uint32_t v[16];
          tmem_ld16(acc + (uint32_t)c, v);
          tmem_ld_wait();
          if (wr)
#pragma unroll
            for (int i = 0; i < 16; ++i)
              if (c + i < a.out_cols) orow[c + i] = __uint_as_float(v[i]) * a.inv_tau;
        }
      }
    }
    if (!ok && lane == 0) atomicOr(a.status, kErrTimeout);
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 5) tmem_dealloc(tmem, tmem_cols);
}

// X [rows][d] (BF16 or FP32) -> P [rows_p][dp] and PT [dp][rows_p], BF16, zero padded.
// A 32 x 32 tile per block goes through shared memory, so both copies are
// written along their rows.
constexpr int kPrepTile = 32;
__global__ void k_loss_prep(const void *X, int elem, int rows, int d, int rows_p, int dp, __nv_bfloat16 *P,
                            __nv_bfloat16 *PT) {
  __shared__ __nv_bfloat16 tile[kPrepTile][kPrepTile + 1];
  const int r0 = blockIdx.x * kPrepTile, k0 = blockIdx.y * kPrepTile;  // rows on x: no 65,535 limit
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8 threads
  for (int j = ty; j < kPrepTile; j += blockDim.y) {
    const int row = r0 + j, k = k0 + tx;
    __nv_bfloat16 v = __float2bfloat16_rn(0.f);
    if (row < rows && k < d) {
      v = elem == kElemBF16 ? reinterpret_cast<const __nv_bfloat16 *>(X)[(size_t)row * d + k]
                            : __float2bfloat16_rn(reinterpret_cast<const float *>(X)[(size_t)row * d + k]);
    }
    if (row < rows_p && k < dp) P[(size_t)row * dp + k] = v;
    tile[j][tx] = v;
  }
  __syncthreads();
  for (int j = ty; j < kPrepTile; j += blockDim.y) {
    const int k = k0 + j, row = r0 + tx;
    if (k < dp && row < rows_p) PT[(size_t)k * rows_p + row] = tile[tx][j];
  }
}

// Per query (one thread each): combine the split partials into its log-sum-exp.
__global__ void k_loss_lse(const LossArgs a, int splits, float *lse) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.B) return;
  float mx = -INFINITY;
  for (int s = 0; s < splits; ++s) mx = fmaxf(mx, a.part_m[(size_t)s * a.rows_p + q]);
  float sum = 0.f;
  for (int s = 0; s < splits; ++s) {
    const float ms = a.part_m[(size_t)s * a.rows_p + q];
    if (ms > -INFINITY) sum += a.part_s[(size_t)s * a.rows_p + q] * exp2f((ms - mx) * kLog2e);
  }
  lse[q] = mx + logf(sum);
}

// The loss: one CTA sums the queries' terms lse - z_pos in FP64 in a fixed
// order.  An out-of-range positive makes the loss NaN.
__global__ void k_loss_combine(const LossArgs a, const float *lse, float *loss) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int q = threadIdx.x; q < a.B; q += blockDim.x) {
    const int p = a.pos[q];
    acc += (p >= 0 && p < a.M) ? (double)lse[q] - (double)a.zpos[q] : (double)NAN;
  }
  // fixed reduction tree: lanes by shuffles, then the warps' sums in warp order
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (int)threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, off);
    if (threadIdx.x == 0) *loss = (float)(v / (double)a.B);
  }
}

__global__ void k_loss_dq_reduce(const float *part, int splits, size_t split_stride, int B, int d, int dp, float *dQ) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * d) return;
  const int q = (int)(i / d), k = (int)(i % d);
  float s = 0.f;
  for (int sp = 0; sp < splits; ++sp) s += part[(size_t)sp * split_stride + (size_t)q * dp + k];
  dQ[i] = s;
}

// Per query: the selection's K, and its pass count = the keys listed.
__global__ void k_hn_setup(int B, int n_neg, const uint32_t *key_cnt, int32_t *kq, unsigned long long *npass) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= B) return;
  kq[q] = n_neg;
  npass[q] = key_cnt[q];
}

// The mined negatives as loss mask bits (bit j of row q: job j is one of q's hard
// negatives); the rows were cleared before.
__global__ void k_hn_mask(const int32_t *ids, const int32_t *count, int B, int n_neg, int Mw, uint32_t *mask) {
  const int q = blockIdx.y;
  const int n = count[q];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n && i < n_neg; i += gridDim.x * blockDim.x) {
    const int j = ids[(size_t)q * n_neg + i];
    if (j >= 0 && (j >> 5) < Mw) atomicOr(&mask[(size_t)q * Mw + (j >> 5)], 1u << (j & 31));
  }
}

}  // namespace

cudaError_t launch_hn_setup(int B, int n_neg, const uint32_t *key_cnt, int32_t *kq, unsigned long long *npass,
                            cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  k_hn_setup<<<(B + 255) / 256, 256, 0, s>>>(B, n_neg, key_cnt, kq, npass);
  return cudaGetLastError();
}

cudaError_t launch_hn_mask(const int32_t *ids, const int32_t *count, int B, int n_neg, int Mw, uint32_t *mask,
                           cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  k_hn_mask<<<dim3((unsigned)((n_neg + 255) / 256), (unsigned)B), 256, 0, s>>>(ids, count, B, n_neg, Mw, mask);
  return cudaGetLastError();
}

cudaError_t launch_loss_prep(const void *X, int elem, int rows, int d, int rows_p, int dp, void *P, void *PT,
                             cudaStream_t s) {
  const dim3 grid((unsigned)((rows_p + kPrepTile - 1) / kPrepTile), (unsigned)((dp + kPrepTile - 1) / kPrepTile));
  k_loss_prep<<<grid, dim3(kPrepTile, 8), 0, s>>>(X, elem, rows, d, rows_p, dp, (__nv_bfloat16 *)P,
                                                  (__nv_bfloat16 *)PT);
  return cudaGetLastError();
}

cudaError_t launch_loss_pass(int mode, const LossArgs &a, int grid_x, int grid_y, const void *tm_r, const void *tm_c,
                             const void *tm_ct, cudaStream_t s) {
  const LossSmem L = loss_smem(a.dp, mode);
  const size_t smem = L.total + 1024;
  const CUtensorMap &r = *static_cast<const CUtensorMap *>(tm_r);
  const CUtensorMap &c = *static_cast<const CUtensorMap *>(tm_c);
  const CUtensorMap &ct = *static_cast<const CUtensorMap *>(tm_ct ? tm_ct : tm_c);
  dim3 grid(grid_x, grid_y);
  cudaError_t e;
  switch (mode) {
    case kFwd:
      e = allow_dynamic_smem((const void *)k_loss<kFwd>, (size_t)smem);
      if (e != cudaSuccess) return e;
      k_loss<kFwd><<<grid, kLossFwdThreads, smem, s>>>(a, r, c, ct);
      break;
    case kDq:
      e = allow_dynamic_smem((const void *)k_loss<kDq>, (size_t)smem);
      if (e != cudaSuccess) return e;
      k_loss<kDq><<<grid, kLossThreads, smem, s>>>(a, r, c, ct);
      break;
    case kDj:
      e = allow_dynamic_smem((const void *)k_loss<kDj>, (size_t)smem);
      if (e != cudaSuccess) return e;
      k_loss<kDj><<<grid, kLossThreads, smem, s>>>(a, r, c, ct);
      break;
    case kKeys:
      e = allow_dynamic_smem((const void *)k_loss<kKeys>, (size_t)smem);
      if (e != cudaSuccess) return e;
      k_loss<kKeys><<<grid, kLossFwdThreads, smem, s>>>(a, r, c, ct);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_loss_combine(const LossArgs &a, int splits, float *lse, float *loss, cudaStream_t s) {
  if (a.B > 0) k_loss_lse<<<(unsigned)((a.B + 255) / 256), 256, 0, s>>>(a, splits, lse);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_loss_combine<<<1, 1024, 0, s>>>(a, lse, loss);
  return cudaGetLastError();
}

cudaError_t launch_loss_dq_reduce(const float *part, int splits, size_t split_stride, int B, int d, int dp, float *dQ,
                                  cudaStream_t s) {
  const int64_t n = (int64_t)B * d;
  k_loss_dq_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(part, splits, split_stride, B, d, dp, dQ);
  return cudaGetLastError();
}

}  // namespace lr
