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
// Four epilogue sets of four warps (TMEM lane quarters) take the two tiles of
// a pair, two sets per tile with 32 columns each; warp 4 issues the TMA
// loads, warp 5 the MMAs.  The streamed
// tiles come in pairs: one N = 128 MMA per K step scores both tiles of a pair
// (an MMA costs about the same at N = 64 as at N = 128), into the two sets'
// score buffers.  Tensor memory holds the scores of two pairs (four in the
// score-only passes, which have no accumulator), so the MMAs of pair p + 2 are
// queued behind the second products of pair p and the sets find pair p + 1
// scored when they finish pair p.
// The streamed operand and its transposed copy (the second product's
// operand) sit in separate rings: a pair's stage is free once it is scored, a
// transposed tile's once its product is done.
// Every wait is bounded; a timeout sets the status word.
#include <cuda.h>
#include <cuda_bf16.h>

#include "bits.cuh"
#include "lr_internal.h"
#include "ptx.h"

namespace lr {
namespace {

constexpr int kRRows = 128;     // rows of the resident tile
constexpr int kCRows = 64;      // rows of a streamed tile (one epilogue set's score columns)
constexpr int kPairRows = 2 * kCRows;  // a pair of streamed tiles: the score MMAs' N
constexpr int kLossThreads = 576;  // warps 0-3, 6-9, 10-13, 14-17: four epilogue sets; 4: TMA; 5: MMA
constexpr int kPBufsOne = 6;       // pair stages of the score-only passes (TMA latency under load is ~2 us)
constexpr int kPBufs = 2;          // pair stages of the backward passes
constexpr int kTBufs = 3;          // transposed-tile stages of the backward passes
// tensor memory: two pair slots of 128 score columns, then (backward) the
// accumulator at column 256: [128 rows][dp], or at dp = 128 the transposed
// product's [dp lanes][hi rows | lo rows], 256 columns
constexpr uint32_t kLossTmemColsOne = 512;  // score-only passes: four pair slots
constexpr uint32_t kLossTmemCols = 512;
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

// kDj staging of one epilogue set's 32 queries of a tile: mask words of the
// CTA's 128 job rows (4 per query), positives and log-sum-exps
struct DjStage {
  uint32_t mask[32 * 4];
  int32_t pos[32];
  float lse[32];
};

__host__ __device__ inline LossSmem loss_smem(int dp, int mode) {
  LossSmem L;
  size_t off = 0;
  L.r = off;
  off += (size_t)(dp / 64) * kRRows * 128;  // K-blocks of 128 rows x 128 bytes
  L.c = off;
  const bool one_product = mode == kFwd || mode == kKeys;
  off += (size_t)(one_product ? kPBufsOne : kPBufs) * (dp / 64) * kPairRows * 128;  // [stage][K-block][128 rows]
  L.ct = off;
  off += one_product ? 0 : (size_t)kTBufs * dp * 128;  // transposed C tile: dp rows x 64 values
  L.dz = off;
  off += one_product ? 0 : (size_t)2 * 2 * kRRows * 128;  // [buffer][hi, lo] 128 rows x 64 values
  L.stage = off;
  off += mode == kDj ? 8 * sizeof(DjStage) : 0;  // two per epilogue set
  L.bars = off;
  off += 48 * 8;
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
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
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
  constexpr int nP = kOne ? kPBufsOne : kPBufs;  // pair stages
  uint64_t *bar_r = bars, *c_full = bars + 1, *c_empty = c_full + nP;  // [nP] each
  uint64_t *t_full = c_empty + nP, *t_empty = t_full + kTBufs;       // [kTBufs] each
  // pair slots of scores in tensor memory: four in the score-only passes (no
  // accumulator), two in the backward passes
  constexpr int kSlots = kOne ? 4 : 2;
  uint64_t *s_full = t_empty + kTBufs, *s_empty = s_full + 2 * kSlots;  // [pair slot][tile of the pair]
  uint64_t *dz_full = s_empty + 2 * kSlots, *dz_empty = dz_full + 2, *acc_full = dz_empty + 2;
  uint32_t *holder = reinterpret_cast<uint32_t *>(smem + L.holder);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r0 = blockIdx.x * kRRows;
  const int t0 = blockIdx.y * a.c_per_split;
  const int T = min(a.c_per_split, a.n_ctiles - t0);  // streamed tiles of this CTA (>= 1 by construction)
  const int NP = (T + 1) / 2;                          // pairs (the last one may hold one tile)
  const size_t p_bytes = (size_t)KB * kPairRows * 128;
  const size_t ct_bytes = (size_t)dp * 128;
  // Backward passes with dp = 128: acc^T[k][r | 128 + r] += C^T[k][c] .
  // [dZ_hi ; dZ_lo][r][c] as ONE MMA of N = 256 per 16-value K step (the
  // transposed C tile as A, the stacked hi / lo dZ rows as B) instead of two
  // MMAs of N = 128 with dZ_hi and dZ_lo as A: an MMA costs about the same
  // whatever its width up to 128 columns, so the product issues half the
  // instructions.  The write-out adds the two halves.
  const bool swap = !kOne && dp == 128;
  const uint32_t tmem_cols = kOne ? kLossTmemColsOne : kLossTmemCols;

  if (threadIdx.x == 0) {
    mbar_init(bar_r, 1);
    for (int i = 0; i < nP; ++i) {
      mbar_init(&c_full[i], 1);
      mbar_init(&c_empty[i], 1);
    }
    for (int i = 0; i < kTBufs; ++i) {
      mbar_init(&t_full[i], 1);
      mbar_init(&t_empty[i], 1);
    }
    for (int i = 0; i < 2 * kSlots; ++i) {
      mbar_init(&s_full[i], 1);
      mbar_init(&s_empty[i], 8);  // the two sets of the tile, four warps each
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&dz_full[i], 8);
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
      int np = 0, nc = 0;  // pairs and transposed tiles issued
      mbar_arrive_expect_tx(bar_r, (uint32_t)(KB * kRRows * 128));
      for (int kb = 0; kb < KB; ++kb) tma_load_2d(sr + (size_t)kb * kRRows * 128, &tm_r, kb * 64, r0, bar_r);
      auto load_pair = [&](int p) -> bool {
        const int st = p % nP, nt = min(2, T - 2 * p);
        if (!mbar_wait(&c_empty[st], (uint32_t)((p / nP) & 1) ^ 1u)) return false;
        mbar_arrive_expect_tx(&c_full[st], (uint32_t)(nt * KB * kCRows * 128));
        for (int h = 0; h < nt; ++h) {
          const int c0 = (t0 + 2 * p + h) * kCRows;
          for (int kb = 0; kb < KB; ++kb)
            tma_load_2d(sc + (size_t)st * p_bytes + (size_t)kb * kPairRows * 128 + (size_t)h * kCRows * 128, &tm_c,
                        kb * 64, c0, &c_full[st]);
        }
        return true;
      };
      auto load_ct = [&](int t) -> bool {
        const int st = t % kTBufs;
        if (!mbar_wait(&t_empty[st], (uint32_t)((t / kTBufs) & 1) ^ 1u)) return false;
        mbar_arrive_expect_tx(&t_full[st], (uint32_t)ct_bytes);
        tma_load_2d(sct + (size_t)st * ct_bytes, &tm_ct, (t0 + t) * kCRows, 0, &t_full[st]);
        return true;
      };
      // Issue order = the order in which the MMA thread frees stages: pair p
      // is scored before the products of tiles 2p - 2 and 2p - 1, so a pair
      // is loaded once the transposed tiles two pairs before it are queued.
      while (ok && (np < NP || (!kOne && nc < T))) {
        if (np < NP && (kOne || np <= nc / 2 + 2)) {
          ok = load_pair(np);
          np += ok ? 1 : 0;
        } else {
          ok = load_ct(nc);
          nc += ok ? 1 : 0;
        }
      }
      if (!ok) {
        atomicOr(a.status, kErrTimeout);
        mbar_wait(bar_r, 0u);  // let issued loads land
        for (int p = np > nP ? np - nP : 0; p < np; ++p) mbar_wait(&c_full[p % nP], (uint32_t)((p / nP) & 1));
        for (int t = nc > kTBufs ? nc - kTBufs : 0; t < nc; ++t)
          mbar_wait(&t_full[t % kTBufs], (uint32_t)((t / kTBufs) & 1));
      }
    }
    __syncwarp();
  } else if (warp == 5) {
    // ---------------------------------------------------------------- MMA
    if (lane == 0) {
      const uint32_t id_s2 = idesc_bf16(kRRows, kPairRows), id_s1 = idesc_bf16(kRRows, kCRows);
      const uint32_t id_g = idesc_bf16(kRRows, dp);
      const uint32_t id_t = idesc_bf16(128, 2 * kRRows);  // the transposed product: M = dp = 128, N = 256
      const uint32_t acc = tmem + 2u * kPairRows;
      bool issued = false;
      // scores of pair p into slot j = p % kSlots: tile 2p into columns
      // [128 j, 128 j + 64), tile 2p + 1 into the next 64, once the sets have
      // read pair p - kSlots's
      auto issue_pair = [&](int p) -> bool {
        const int st = p % nP, nt = min(2, T - 2 * p), j = p % kSlots;
        if (!mbar_wait(&c_full[st], (uint32_t)((p / nP) & 1))) return false;
        for (int h = 0; h < nt; ++h)
          if (!mbar_wait(&s_empty[2 * j + h], (uint32_t)((p / kSlots) & 1) ^ 1u)) return false;
        tc_fence_after();
        const uint32_t ra = smem_u32(sr), ca = smem_u32(sc + (size_t)st * p_bytes);
        for (int k = 0; k < dp / 16; ++k) {
          const uint32_t koff = (uint32_t)(k & 3) * 32u;
          mma_bf16(tmem + (uint32_t)(j * kPairRows), sw128_desc(ra + (uint32_t)(k >> 2) * (kRRows * 128) + koff),
                   sw128_desc(ca + (uint32_t)(k >> 2) * (kPairRows * 128) + koff), nt == 2 ? id_s2 : id_s1,
                   k > 0 ? 1u : 0u);
        }
        issued = true;
        mma_commit(&s_full[2 * j]);
        if (nt == 2) mma_commit(&s_full[2 * j + 1]);
        mma_commit(&c_empty[st]);
        return true;
      };
      if (!mbar_wait(bar_r, 0u)) ok = false;
      for (int p = 0; p < kSlots && p < NP && ok; ++p) ok = issue_pair(p);
      for (int p = 0; p < NP && ok; ++p) {
        for (int h = 0; h < 2 && 2 * p + h < T && !kOne; ++h) {
          const int t = 2 * p + h, st = t % kTBufs;
          if (!mbar_wait(&dz_full[h], (uint32_t)(p & 1)) || !mbar_wait(&t_full[st], (uint32_t)((t / kTBufs) & 1))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dh = smem_u32(sdz + (size_t)(2 * h) * kRRows * 128);
          const uint32_t dl = smem_u32(sdz + (size_t)(2 * h + 1) * kRRows * 128);
          const uint32_t ct = smem_u32(sct + (size_t)st * ct_bytes);
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
          mma_commit(&dz_empty[h]);
          mma_commit(&t_empty[st]);
        }
        if (ok && p + kSlots < NP && !issue_pair(p + kSlots)) ok = false;
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
    // four sets of four warps (0-3, 6-9, 10-13, 14-17): set e takes column
    // half e >> 1 of the pair's tile e & 1 (tiles e & 1, e & 1 + 2, ...), so
    // score buffer b = e & 1 and dZ buffer b are shared by two sets, each with
    // its own 32 columns, and their barrier phases come in order; warp w reads
    // tensor-memory lanes 32 (w % 4) ..
    constexpr int kSets = 4;
    const int eset = warp < 4 ? 0 : (warp - 2) >> 2, quarter = warp & 3;
    const int b = eset & 1, half = eset >> 1;
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
    // Mask words (and for kDj the set's 32 queries' positives and lse) are
    // fetched one tile of the set ahead.  kFwd/kDq: this row's word of the
    // set's 32 columns, in a register.  kDj: the set's 128 threads stage its
    // queries in shared memory (double buffered per set; each iteration ends
    // at the set's named barrier, which every warp of the set reaches, also
    // after a failed wait, so no warp waits forever).
    uint32_t nw = ~0u;  // kFwd/kDq: next tile's mask word
    uint32_t smw = 0u;  // kDj: this thread's share of the next stage
    int spos = -1;
    float slse = 0.f;
    auto fetch_row_word = [&](int tt) {
      const int cc0 = (t0 + tt) * kCRows + 32 * half;
      nw = ~0u;
      if (rvalid && a.mask != nullptr && cc0 < a.M) nw = __ldg(a.mask + (size_t)grow * a.Mw + (cc0 >> 5));
    };
    auto fetch_stage = [&](int tt) {
      const int cq0 = (t0 + tt) * kCRows + 32 * half;
      const int q = cq0 + (r >> 2), w = (r0 >> 5) + (r & 3);
      smw = q < a.B && w < a.Mw ? (a.mask != nullptr ? __ldg(a.mask + (size_t)q * a.Mw + w) : ~0u) : 0u;
      const int qq = cq0 + r;
      spos = (r < 32 && qq < a.B) ? __ldg(a.pos + qq) : -1;
      slse = (r < 32 && qq < a.B) ? __ldg(a.lse + qq) * kLog2e : 0.f;  // log2 units
    };
    auto store_stage = [&](int buf) {
      DjStage &st = stg[buf];
      st.mask[r] = smw;
      if (r < 32) {
        st.pos[r] = spos;
        st.lse[r] = slse;
      }
    };
    auto set_barrier = [&]() { asm volatile("bar.sync %0, 128;" ::"r"(1 + eset) : "memory"); };
    if (MODE == kDj) {
      if (b < T) {
        fetch_stage(b);
        store_stage(2 * eset);
      }
      set_barrier();
    } else if (b < T) {
      fetch_row_word(b);
    }
    for (int t = b, it = 0; t < T; t += 2, ++it) {
      const int sb = 2 * eset + (it & 1);  // kDj: this tile's stage
      const int c0 = (t0 + t) * kCRows + 32 * half;  // first column of the set's 32
      const uint32_t cw = nw;
      if (t + 2 < T) {
        if (MODE == kDj) fetch_stage(t + 2);
        else fetch_row_word(t + 2);
      }
      do {
      if (!ok) break;
      const int slot = (t >> 1) % kSlots;  // pair slot of this tile's scores
      if (!wwait(&s_full[2 * slot + b], (uint32_t)(((t >> 1) / kSlots) & 1), lane)) {
        ok = false;
        break;
      }
      tc_fence_after();
      uint32_t sv[32];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        uint32_t (&part)[16] = *reinterpret_cast<uint32_t (*)[16]>(&sv[16 * q]);
        tmem_ld16(trow + (uint32_t)(slot * kPairRows + b * kCRows + 32 * half + 16 * q), part);
      }
      tmem_ld_wait();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&s_empty[2 * slot + b]);
      // allowed columns of the set's 32: bit c of al; kDj also the columns
      // whose positive is this row's job: bit c of pm
      uint32_t al = 0u, pm = 0u;
      if (MODE == kDj) {
        // the set's 32 queries x this warp's 32 jobs as a 32 x 32 bit matrix,
        // one query per lane, transposed so that lane r holds its job's row
        const DjStage &st = stg[sb];
        const int wj = (r0 >> 5) + quarter;
        const int p = st.pos[lane];
        const uint32_t pw = (p >= 0 && (p >> 5) == wj) ? 1u << (p & 31) : 0u;
        const uint32_t mw = st.mask[lane * 4 + quarter] | pw;  // the positive is always allowed
        pm = bit_transpose32(pw, lane);  // every lane takes part in the transposes
        const uint32_t tr = bit_transpose32(mw, lane);
        al = rvalid ? tr : 0u;
      } else if (rvalid) {
        uint32_t w0 = cw;
        const int lim = a.M - c0;  // columns past M do not exist
        w0 &= lim >= 32 ? ~0u : (lim > 0 ? ((1u << lim) - 1u) : 0u);
        const int pc = pos_row - c0;
        if (pc >= 0 && pc < 32) w0 |= 1u << pc;
        al = w0;
      }
      if (MODE == kFwd) {
        if (pos_row >= c0 && pos_row < c0 + 32) {
          const int pc = pos_row - c0;
#pragma unroll
          for (int c = 0; c < 32; ++c)
            if (c == pc) zpos = __uint_as_float(sv[c]) * a.inv_tau;
          have_pos = true;
        }
        // ssum = sum of 2^(z2 - m) over the allowed columns seen, z2 = s inv_tau
        // log2(e) (log2 units; failing columns add 0).  The offset m is the
        // maximum of the set's first tile of the row with an allowed column
        // and stays fixed (one FMA, one exponential per column) unless a
        // later tile's terms would overflow: that tile is redone with its own
        // maximum as the new offset.
        const float c2 = a.inv_tau * kLog2e;
        auto tile_max = [&]() {
          float tmax = -INFINITY;
#pragma unroll
          for (int c = 0; c < 32; ++c)
            if ((al >> c) & 1u) tmax = fmaxf(tmax, __uint_as_float(sv[c]) * c2);
          return tmax;
        };
        if (m == -INFINITY) m = tile_max();
        if (m > -INFINITY) {
          float add = 0.f;
#pragma unroll
          for (int c = 0; c < 32; ++c)
            add += ((al >> c) & 1u) ? ex2_approx(fmaf(__uint_as_float(sv[c]), c2, -m)) : 0.f;
          if (add < 0x1p100f) {
            ssum += add;
          } else {  // overflow or near it: rescale to this tile's maximum
            const float mn = fmaxf(m, tile_max());
            add = 0.f;
#pragma unroll
            for (int c = 0; c < 32; ++c)
              add += ((al >> c) & 1u) ? ex2_approx(fmaf(__uint_as_float(sv[c]), c2, -mn)) : 0.f;
            ssum = ssum * ex2_approx(m - mn) + add;
            m = mn;
          }
        }
      } else if (MODE == kKeys) {
        if (rvalid) {
          // allowed columns without the positive (al has no column past M),
          // appended to the row's key list in place of the tile's range
          uint32_t nb = al;
          const int pc = pos_row - c0;
          if (pc >= 0 && pc < 32) nb &= ~(1u << pc);
          const uint32_t cntk = (uint32_t)__popc(nb);
          if (cntk) {
            uint32_t o = atomicAdd(&a.key_cnt[grow], cntk);
            uint64_t *krow = a.keys + (size_t)grow * (size_t)a.keys_ld;
#pragma unroll
            for (int c = 0; c < 32; ++c)
              if ((nb >> c) & 1u) krow[o++] = make_key(__uint_as_float(sv[c]), (uint32_t)(c0 + c));
          }
        }
      } else {
        // dZ of the set's 32 columns as two BF16 terms, written in the
        // 128-byte-swizzled K-major layout of the tile (chunks 4 half .. 4 half + 3)
        if (!wwait(&dz_empty[b], (uint32_t)((t >> 1) & 1) ^ 1u, lane)) {
          ok = false;
          break;
        }
        unsigned char *dh = sdz + (size_t)(2 * b) * kRRows * 128 + (size_t)r * 128;
        unsigned char *dl = sdz + (size_t)(2 * b + 1) * kRRows * 128 + (size_t)r * 128;
        const float c2 = a.inv_tau * kLog2e;
        // dZ / g = softmax - [positive] on allowed columns (the factor g =
        // dL / B is applied to the accumulated product); here the softmax
        // term, the positives' -1 after the tile is written
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {
          uint32_t hw[4], lw[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int c = ch * 8 + u * 2;  // columns c, c + 1 of the set's 32
            const float l0 = MODE == kDq ? lse_row : stg[sb].lse[c];  // log2 units
            const float l1 = MODE == kDq ? lse_row : stg[sb].lse[c + 1];
            const float p0 = ((al >> c) & 1u) ? ex2_approx(fmaf(__uint_as_float(sv[c]), c2, -l0)) : 0.f;
            const float p1 = ((al >> (c + 1)) & 1u) ? ex2_approx(fmaf(__uint_as_float(sv[c + 1]), c2, -l1)) : 0.f;
            // hi = p truncated to BF16 (its upper 16 bits), lo = p - hi (exact)
            // rounded to nearest: p = hi + lo within 2^-15 p
            const uint32_t u0 = __float_as_uint(p0), u1 = __float_as_uint(p1);
            const __nv_bfloat162 lv =
                __floats2bfloat162_rn(p0 - __uint_as_float(u0 & 0xFFFF0000u), p1 - __uint_as_float(u1 & 0xFFFF0000u));
            hw[u] = __byte_perm(u0, u1, 0x7632);
            lw[u] = *reinterpret_cast<const uint32_t *>(&lv);
          }
          const int so = (((4 * half + ch) ^ (r & 7)) & 7) << 4;
          *reinterpret_cast<uint4 *>(dh + so) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          *reinterpret_cast<uint4 *>(dl + so) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        // column c of this row is a positive (an allowed column: the positive
        // always is): its entry becomes p - 1, computed in FP32 from the
        // column's score so that it keeps its relative accuracy when p is near 1
        auto patch = [&](int c, float lse2) {
          float sc = 0.f;
#pragma unroll
          for (int k = 0; k < 32; ++k) sc = k == c ? __uint_as_float(sv[k]) : sc;
          const float v = ex2_approx(fmaf(sc, c2, -lse2)) - 1.f;
          const __nv_bfloat16 nh = __float2bfloat16_rn(v);
          const int gc = 32 * half + c;
          const int so = ((((gc >> 3) ^ (r & 7)) & 7) << 4) | ((gc & 7) << 1);
          *reinterpret_cast<__nv_bfloat16 *>(dh + so) = nh;
          *reinterpret_cast<__nv_bfloat16 *>(dl + so) = __float2bfloat16_rn(v - __bfloat162float(nh));
        };
        if (MODE == kDq) {
          const int pc = pos_row - c0;
          if (pc >= 0 && pc < 32) patch(pc, lse_row);
        } else {
          for (uint32_t w = pm & al; w != 0u; w &= w - 1u) {
            const int c = __ffs(w) - 1;
            patch(c, stg[sb].lse[c]);
          }
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
    if (MODE == kFwd) {  // the row's log-sum-exp partial of this split and set
      if (rvalid) {
        const size_t part = (size_t)(kSets * blockIdx.y + eset) * a.rows_p + grow;
        a.part_m[part] = m * kLn2;  // natural units for the combine
        a.part_s[part] = ssum;
        if (have_pos) a.zpos[grow] = zpos;
      }
    } else if (MODE == kKeys) {
    } else {  // the four sets write the accumulated rows, set e its quarter
      if (!wwait(acc_full, 0u, lane)) ok = false;
      tc_fence_after();
      const uint32_t acc = trow + 2u * kPairRows;
      const float scale = a.inv_tau * (a.dloss != nullptr ? __ldg(a.dloss) : 1.f) * a.inv_b;  // inv_tau g
      if (swap) {
        // lane k (= this thread's TMEM lane) holds column k of every row: rows
        // r and 128 + r are the hi and lo halves; a warp's 32 lanes write 32
        // consecutive columns of a row.  Set e takes rows [32 e, 32 e + 32)
        // (four loads in flight per wait).
        const int k = quarter * 32 + lane;
        float *ocol = a.out + (size_t)blockIdx.y * a.out_split + k;
        const int rows_ok = MODE == kDq ? a.rows_p : a.M;
        const int rr = 32 * eset;
        uint32_t vh[32], vl[32];
        tmem_ld16(acc + (uint32_t)rr, *reinterpret_cast<uint32_t (*)[16]>(&vh[0]));
        tmem_ld16(acc + (uint32_t)(rr + 16), *reinterpret_cast<uint32_t (*)[16]>(&vh[16]));
        tmem_ld16(acc + (uint32_t)(kRRows + rr), *reinterpret_cast<uint32_t (*)[16]>(&vl[0]));
        tmem_ld16(acc + (uint32_t)(kRRows + rr + 16), *reinterpret_cast<uint32_t (*)[16]>(&vl[16]));
        tmem_ld_wait();
        if (ok && k < a.out_cols)
#pragma unroll
          for (int i = 0; i < 32; ++i)
            if (r0 + rr + i < rows_ok)
              ocol[(size_t)(r0 + rr + i) * a.out_ld] = (__uint_as_float(vh[i]) + __uint_as_float(vl[i])) * scale;
      } else {
        // thread r holds row r: set e writes columns [e dp / 4, (e + 1) dp / 4)
        float *orow = a.out + (size_t)blockIdx.y * a.out_split + (size_t)grow * a.out_ld;
        const bool wr = ok && (MODE == kDq ? grow < a.rows_p : grow < a.M);
        for (int c = eset * (dp / 4); c < (eset + 1) * (dp / 4); c += 16) {
          uint32_t v[16];
          tmem_ld16(acc + (uint32_t)c, v);
          tmem_ld_wait();
          if (wr)
#pragma unroll
            for (int i = 0; i < 16; i += 4)
              *reinterpret_cast<float4 *>(orow + c + i) =
                  make_float4(__uint_as_float(v[i]) * scale, __uint_as_float(v[i + 1]) * scale,
                              __uint_as_float(v[i + 2]) * scale, __uint_as_float(v[i + 3]) * scale);
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

// X [rows][d] (BF16 or FP32) -> P [rows_p][dp] and/or PT [dp][rows_p], BF16,
// zero padded (either output may be null), for two operands in one launch
// (blocks [0, nb0) take job 0).  A 64 x 64 tile per block goes through shared
// memory; a thread moves two adjacent values, so both copies are written
// along their rows in 4-byte words.
constexpr int kPrepTile = 64;

struct PrepJob {
  const void *X;
  int rows, rows_p;
  __nv_bfloat16 *P, *PT;
};

__global__ void __launch_bounds__(256) k_loss_prep(const PrepJob j0, const PrepJob j1, int nb0, int elem, int d,
                                                   int dp) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
  __shared__ __nv_bfloat16 tile[kPrepTile][kPrepTile + 2];
  const bool second = (int)blockIdx.x >= nb0;
  const PrepJob &J = second ? j1 : j0;
  const void *X = J.X;
  const int rows = J.rows, rows_p = J.rows_p;
  __nv_bfloat16 *P = J.P, *PT = J.PT;
  const int r0 = ((int)blockIdx.x - (second ? nb0 : 0)) * kPrepTile, k0 = blockIdx.y * kPrepTile;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;              // 32 x 8 threads
  const int k = k0 + 2 * tx;
  for (int j = ty; j < kPrepTile; j += 8) {
    const int row = r0 + j;
    float v0 = 0.f, v1 = 0.f;
    if (row < rows) {
      if (elem == kElemBF16) {
        const __nv_bfloat16 *x = reinterpret_cast<const __nv_bfloat16 *>(X) + (size_t)row * d;
        if (k < d) v0 = __bfloat162float(x[k]);
        if (k + 1 < d) v1 = __bfloat162float(x[k + 1]);
      } else {
        const float *x = reinterpret_cast<const float *>(X) + (size_t)row * d;
        if (k < d) v0 = x[k];
        if (k + 1 < d) v1 = x[k + 1];
      }
    }
    const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
    if (P != nullptr && row < rows_p && k < dp) *reinterpret_cast<__nv_bfloat162 *>(P + (size_t)row * dp + k) = h;
    tile[j][2 * tx] = h.x;
    tile[j][2 * tx + 1] = h.y;
  }
  if (PT == nullptr) return;
  __syncthreads();
  const int row = r0 + 2 * tx;  // PT columns (rows of X) of this thread
  for (int j = ty; j < kPrepTile; j += 8) {
    const int kk = k0 + j;
    if (kk < dp && row < rows_p) {
      __nv_bfloat162 h;
      h.x = tile[2 * tx][j];
      h.y = tile[2 * tx + 1][j];
      *reinterpret_cast<__nv_bfloat162 *>(PT + (size_t)kk * rows_p + row) = h;
    }
  }
}

// Per query (one warp each, lane s reads partials s and s + 32, so the
// partials load in one round): combine the split partials into its log-sum-exp; each block
// sums its queries' terms lse - z_pos in FP64 in a fixed order, and the last
// block to finish adds the blocks' sums in block order (the loss does not
// depend on the blocks' timing).  An out-of-range positive makes the loss
// NaN.  done[0] counts finished blocks (zero before the launch; the last block
// resets it).  At most 64 partials per query.
constexpr int kLseThreads = 256;
constexpr int kLseQueries = kLseThreads / 32;

__global__ void __launch_bounds__(kLseThreads) k_loss_lse(const LossArgs a, int splits, float *lse, double *bsum,
                                                          uint32_t *done, float *loss) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
  __shared__ double red[kLseQueries];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int q = blockIdx.x * kLseQueries + w;
  double term = 0.0;
  if (q < a.B) {
    const int s1 = lane + 32;
    const float ms = lane < splits ? a.part_m[(size_t)lane * a.rows_p + q] : -INFINITY;
    const float ss = lane < splits ? a.part_s[(size_t)lane * a.rows_p + q] : 0.f;
    const float ms1 = s1 < splits ? a.part_m[(size_t)s1 * a.rows_p + q] : -INFINITY;
    const float ss1 = s1 < splits ? a.part_s[(size_t)s1 * a.rows_p + q] : 0.f;
    float mx = fmaxf(ms, ms1);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, off));
    float sum = (ms > -INFINITY ? ss * exp2f((ms - mx) * kLog2e) : 0.f) +
                (ms1 > -INFINITY ? ss1 * exp2f((ms1 - mx) * kLog2e) : 0.f);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, off);
    const float l = mx + logf(sum);
    if (lane == 0) {
      lse[q] = l;
      const int p = a.pos[q];
      term = (p >= 0 && p < a.M) ? (double)l - (double)a.zpos[q] : (double)NAN;
    }
  }
  if (lane == 0) red[w] = term;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int i = 0; i < kLseQueries; ++i) v += red[i];
    bsum[blockIdx.x] = v;
    __threadfence();
    last = atomicAdd(done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (w == 0) {  // the blocks' sums in block order: lane-strided partials, then a fixed shuffle tree
    double v = 0.0;
    for (int i = lane; i < (int)gridDim.x; i += 32) v += __ldcg(bsum + i);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, off);
    if (lane == 0) {
      *loss = (float)(v / (double)a.B);
      *done = 0u;
    }
  }
}

// dQ / dJ = the sum of the split partials; four values of a row per thread.
__global__ void k_loss_dq_reduce(const float *part, int splits, size_t split_stride, int B, int d, int dp, float *dQ) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
  const int dq4 = (d + 3) / 4;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * dq4) return;
  const int q = (int)(i / dq4), k = 4 * (int)(i % dq4);
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int sp = 0; sp < splits; ++sp) {
    const float4 v = __ldcs(reinterpret_cast<const float4 *>(part + (size_t)sp * split_stride + (size_t)q * dp + k));
    s.x += v.x;
    s.y += v.y;
    s.z += v.z;
    s.w += v.w;
  }
  float *o = dQ + (size_t)q * d + k;
  if ((d & 3) == 0) {
    *reinterpret_cast<float4 *>(o) = s;
  } else {
    o[0] = s.x;
    if (k + 1 < d) o[1] = s.y;
    if (k + 2 < d) o[2] = s.z;
    if (k + 3 < d) o[3] = s.w;
  }
}

// Per query: the selection's K, and its pass count = the keys listed.
__global__ void k_hn_setup(int B, int n_neg, const uint32_t *key_cnt, int32_t *kq, unsigned long long *npass) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= B) return;
  kq[q] = n_neg;
  npass[q] = key_cnt[q];
}

// The mined negatives as loss mask bits (bit j of row q: job j is one of q's hard
// negatives); the rows were cleared before.
__global__ void k_hn_mask(const int32_t *ids, const int32_t *count, int B, int n_neg, int Mw, uint32_t *mask) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
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
  return launch_pdl(k_hn_setup, dim3((unsigned)((B + 255) / 256)), dim3(256), 0, s, B, n_neg, key_cnt, kq, npass);
}

cudaError_t launch_hn_mask(const int32_t *ids, const int32_t *count, int B, int n_neg, int Mw, uint32_t *mask,
                           cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  return launch_pdl(k_hn_mask, dim3((unsigned)((n_neg + 255) / 256), (unsigned)B), dim3(256), 0, s, ids, count, B, n_neg,
                    Mw, mask);
}

cudaError_t launch_loss_prep(int elem, int d, int dp, const void *X0, int rows0, int rows_p0, void *P0, void *PT0,
                             const void *X1, int rows1, int rows_p1, void *P1, void *PT1, cudaStream_t s) {
  const PrepJob j0{X0, rows0, rows_p0, (__nv_bfloat16 *)P0, (__nv_bfloat16 *)PT0};
  const PrepJob j1{X1, rows1, rows_p1, (__nv_bfloat16 *)P1, (__nv_bfloat16 *)PT1};
  const int nb0 = (rows_p0 + kPrepTile - 1) / kPrepTile, nb1 = (rows_p1 + kPrepTile - 1) / kPrepTile;
  const dim3 grid((unsigned)(nb0 + nb1), (unsigned)((dp + kPrepTile - 1) / kPrepTile));
  return launch_pdl(k_loss_prep, grid, dim3(256), 0, s, j0, j1, nb0, elem, d, dp);
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
      return launch_pdl(k_loss<kFwd>, grid, dim3(kLossThreads), smem, s, a, r, c, ct);
    case kDq:
      e = allow_dynamic_smem((const void *)k_loss<kDq>, (size_t)smem);
      if (e != cudaSuccess) return e;
      return launch_pdl(k_loss<kDq>, grid, dim3(kLossThreads), smem, s, a, r, c, ct);
    case kDj:
      e = allow_dynamic_smem((const void *)k_loss<kDj>, (size_t)smem);
      if (e != cudaSuccess) return e;
      return launch_pdl(k_loss<kDj>, grid, dim3(kLossThreads), smem, s, a, r, c, ct);
    case kKeys:
      e = allow_dynamic_smem((const void *)k_loss<kKeys>, (size_t)smem);
      if (e != cudaSuccess) return e;
      return launch_pdl(k_loss<kKeys>, grid, dim3(kLossThreads), smem, s, a, r, c, ct);
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_loss_combine(const LossArgs &a, int splits, float *lse, double *bsum, uint32_t *done, float *loss,
                                cudaStream_t s) {
  if (splits > 64) return cudaErrorInvalidValue;
  return launch_pdl(k_loss_lse, dim3((unsigned)loss_combine_blocks(a.B)), dim3(kLseThreads), 0, s, a, splits, lse, bsum,
                    done, loss);
}

int loss_combine_blocks(int B) { return (B + kLseQueries - 1) / kLseQueries; }

cudaError_t launch_loss_dq_reduce(const float *part, int splits, size_t split_stride, int B, int d, int dp, float *dQ,
                                  cudaStream_t s) {
  const int64_t n = (int64_t)B * ((d + 3) / 4);
  return launch_pdl(k_loss_dq_reduce, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, s, part, splits, split_stride, B,
                    d, dp, dQ);
}

}  // namespace lr
