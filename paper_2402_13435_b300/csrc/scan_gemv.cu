// SIMT scan for small query batches: fused term predicate (F-TBR) + FP32 scoring
// (F-EBR) + candidate gathering, one pass over the job embeddings.
//
// Sec. 5.3 ("F-TBR and F-EBR are integrated in the same program") and the
// appendix paragraphs "TBR", "EBR" ("skip rows") and "Batch Inference" describe
// the method; this kernel is a B300 design of it:
//
//   * The index is cut into groups of 256 rows.  A warp owns one group at a time.
//     For each distinct term of the launch it loads the group's 8 bitmap words
//     (32 contiguous bytes of a term-major bitmap) into shared memory, and lane q
//     evaluates query q's CNF (AND over clauses of OR over terms) word-wise,
//     giving 8 pass words per query.
//   * Rows no query of the launch passes are never read from HBM ("skip rows").
//   * A passing row is read once (lane L holds dims [L*VEC, L*VEC+VEC), 16-byte
//     vector loads, one 512-byte coalesced request per row at d = 128), and its
//     dot products with all NQ queries (held in registers) are reduced across
//     the warp by a transpose butterfly: NQ-1 + 5-log2(NQ) shuffles for NQ sums.
//     The butterfly visits lane pairs in the same order for every query, so a
//     score does not depend on which other queries share the launch.
//   * Candidate handling (mode kCollect): the 64-bit key (score, ~id) of each
//     passing pair is compared with the query's threshold and appended to the
//     query's buffer when it is not below it.  Mode kHist instead histograms one
//     11-bit digit of the keys that match the query's prefix (exact radix
//     selection); the last CTA to finish fixes the digit for every query.
#include "lr_internal.h"

namespace lr {
namespace {

__device__ __forceinline__ uint4 ld_nc_v4(const void *p) {
  uint4 r;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p));
  return r;
}

__device__ __forceinline__ float4 ld_stream_f4(const float *p) {
  float4 r;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
               : "l"(p));
  return r;
}

__device__ __forceinline__ float2 ld_stream_f2(const float *p) {
  float2 r;
  asm volatile("ld.global.nc.L1::no_allocate.v2.f32 {%0,%1}, [%2];" : "=f"(r.x), "=f"(r.y) : "l"(p));
  return r;
}

template <int VEC>
__device__ __forceinline__ void load_row(const float *p, float (&x)[VEC]) {
  if constexpr (VEC % 4 == 0) {
#pragma unroll
    for (int v = 0; v < VEC; v += 4) {
      float4 t = ld_stream_f4(p + v);
      x[v] = t.x; x[v + 1] = t.y; x[v + 2] = t.z; x[v + 3] = t.w;
    }
  } else if constexpr (VEC == 2) {
    float2 t = ld_stream_f2(p);
    x[0] = t.x; x[1] = t.y;
  } else {
#pragma unroll
    for (int v = 0; v < VEC; ++v) x[v] = __ldcs(p + v);
  }
}

// CNF of launch-local query q over the current group's words (sw: [slot][8]).
__device__ __forceinline__ void eval_cnf(const ScanArgs &a, int q, const uint32_t *sw, uint32_t (&pw)[8]) {
#pragma unroll
  for (int w = 0; w < 8; ++w) pw[w] = 0xFFFFFFFFu;
  const int c0 = a.qc_off[q], c1 = a.qc_off[q + 1];
  for (int c = c0; c < c1; ++c) {
    uint32_t cw[8];
#pragma unroll
    for (int w = 0; w < 8; ++w) cw[w] = 0u;
    const int t0 = a.cl_off[c], t1 = a.cl_off[c + 1];
    for (int t = t0; t < t1; ++t) {
      const uint4 *s = reinterpret_cast<const uint4 *>(sw + a.cl_slot[t] * 8);
      const uint4 lo = s[0], hi = s[1];
      cw[0] |= lo.x; cw[1] |= lo.y; cw[2] |= lo.z; cw[3] |= lo.w;
      cw[4] |= hi.x; cw[5] |= hi.y; cw[6] |= hi.z; cw[7] |= hi.w;
    }
#pragma unroll
    for (int w = 0; w < 8; ++w) pw[w] &= cw[w];
  }
}

template <int NQ>
struct Log2 { static constexpr int v = (NQ <= 1) ? 0 : 1 + Log2<NQ / 2>::v; };
template <>
struct Log2<1> { static constexpr int v = 0; };

// Per-row work: NQ dot products, butterfly, owner lanes test and record.
template <int VEC, int NQ>
__device__ __forceinline__ void score_row(const ScanArgs &a, const float (&x)[VEC], const float (&qv)[NQ][VEC],
                                          uint32_t my_pw, int bit, uint32_t row, uint64_t my_tau,
                                          uint64_t my_pre, int lane, int top, int shift, uint32_t dmask) {
  constexpr int M = Log2<NQ>::v;
  float p[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    float acc = x[0] * qv[q][0];
#pragma unroll
    for (int v = 1; v < VEC; ++v) acc = fmaf(x[v], qv[q][v], acc);
    p[q] = acc;
  }
  // transpose stages: offsets 16, 8, ... keep half of the values each time
#pragma unroll
  for (int st = 0; st < M; ++st) {
    const int off = 16 >> st;
    const int half = NQ >> (st + 1);
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = up ? p[i] : p[i + half];
      const float keep = up ? p[i + half] : p[i];
      p[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, off);
    }
  }
  float z = p[0];
#pragma unroll
  for (int off = (16 >> M); off >= 1; off >>= 1) z += __shfl_xor_sync(0xFFFFFFFFu, z, off);

  const int qidx = (lane >> (5 - M)) & (NQ - 1);
  const uint32_t pwq = __shfl_sync(0xFFFFFFFFu, my_pw, qidx);
  const bool owner = (lane & ((1 << (5 - M)) - 1)) == 0;
  if (a.mode == kCollect) {
    const uint64_t tq = __shfl_sync(0xFFFFFFFFu, my_tau, qidx);
    if (owner && ((pwq >> bit) & 1u)) {
      const uint64_t key = make_key(z, row);
      if (key >= tq) {
        const int gq = a.q_base + qidx;
        const uint32_t pos = atomicAdd(&a.buf_cnt[gq], 1u);
        if ((int64_t)pos < a.buf_cap)
          a.buf[(size_t)gq * (size_t)a.buf_cap + pos] = key;
        else
          atomicOr(&a.overflow[gq], 1u);
      }
    }
  } else {
    const uint64_t pq = __shfl_sync(0xFFFFFFFFu, my_pre, qidx);
    if (owner && ((pwq >> bit) & 1u)) {
      const uint64_t key = make_key(z, row);
      if (top >= 64 || (key >> top) == (pq >> top)) {
        const int gq = a.q_base + qidx;
        atomicAdd(&a.hist[(size_t)gq * kFbBins + (uint32_t)((key >> shift) & dmask)], 1u);
      }
    }
  }
}

// Digit step of the exact fallback: for every participating query find the
// digit whose bin holds the krem-th largest key, fix it in the prefix and clear
// the histogram.  Runs in the last CTA of a kHist launch.
__device__ void hist_step(const ScanArgs &a, int top, int shift) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  const int nb = 1 << (top - shift);
  const int per = nb / 32;
  for (int q = warp; q < a.nq; q += wpc) {
    const int gq = a.q_base + q;
    if (a.active && a.active[gq] == 0) continue;
    uint32_t *h = a.hist + (size_t)gq * kFbBins;
    const uint32_t krem = (uint32_t)a.krem[gq];
    if (krem == 0u) {  // nothing passes this filter: no rank to find
      for (int i = lane; i < nb; i += 32) h[i] = 0u;
      continue;
    }
    const int hi_bin = nb - 1 - lane * per;  // this lane's chunk: [hi_bin-per+1, hi_bin]
    uint32_t csum = 0;
    for (int i = 0; i < per; ++i) csum += __ldcg(h + hi_bin - i);
    uint32_t incl = csum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, off);
      if (lane >= off) incl += t;
    }
    const uint32_t excl = incl - csum;
    const unsigned hit = __ballot_sync(0xFFFFFFFFu, excl < krem && krem <= incl);
    if (hit == 0u) {
      if (lane == 0) atomicOr(a.err, 2u);  // rank beyond the histogram total: inconsistent state
    } else if (lane == __ffs(hit) - 1) {
      uint32_t cum = excl;
      int digit = hi_bin;
      for (int i = 0; i < per; ++i) {
        const uint32_t c = __ldcg(h + hi_bin - i);
        if (cum + c >= krem) { digit = hi_bin - i; break; }
        cum += c;
      }
      a.prefix[gq] |= (uint64_t)digit << shift;
      a.krem[gq] = (int32_t)(krem - cum);
    }
    __syncwarp();
    for (int i = lane; i < nb; i += 32) h[i] = 0u;
  }
}

template <int VEC, int NQ>
__global__ void __launch_bounds__(kScanThreads) k_scan_gemv(const ScanArgs a) {
  if (a.any_active != nullptr && *reinterpret_cast<const volatile uint32_t *>(a.any_active) == 0u) return;
  extern __shared__ __align__(16) uint32_t smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpc = blockDim.x >> 5;
  uint32_t *sw = smem + (size_t)warp * (size_t)a.n_slots * 8;

  const int gq = a.q_base + lane;
  const bool qlive = lane < a.nq && (a.active == nullptr || a.active[gq] != 0u);
  uint64_t my_tau = 0, my_pre = 0;
  if (qlive) {
    if (a.mode == kCollect) my_tau = a.tau ? a.tau[gq] : 0ull;
    else my_pre = a.prefix[gq];
  }
  const int top = 64 - kFbBits * a.hist_pass;
  const int shift = top - kFbBits > 0 ? top - kFbBits : 0;
  const uint32_t dmask = (1u << (top - shift)) - 1u;

  float qv[NQ][VEC];
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int v = 0; v < VEC; ++v)
      qv[q][v] = (q < a.nq) ? a.Q[(size_t)(a.q_base + q) * (size_t)a.d_pad + (size_t)lane * VEC + v] : 0.f;

  unsigned long long my_pass = 0;
  const int64_t gw = (int64_t)blockIdx.x * wpc + warp;
  const int64_t nw = (int64_t)gridDim.x * wpc;
  for (int64_t it = gw;; it += nw) {
    const int64_t g = a.g_begin + it * a.g_step;
    if (g >= a.n_groups) break;
    for (int s = lane; s < a.n_slots; s += 32) {
      const uint32_t *src = a.slot_bm[s] + g * kGroupWords;
      const uint4 w0 = ld_nc_v4(src), w1 = ld_nc_v4(src + 4);
      uint4 *dst = reinterpret_cast<uint4 *>(sw + s * 8);
      dst[0] = w0;
      dst[1] = w1;
    }
    __syncwarp();
    uint32_t pw[8];
    if (qlive) {
      eval_cnf(a, lane, sw, pw);
    } else {
#pragma unroll
      for (int w = 0; w < 8; ++w) pw[w] = 0u;
    }
    const int64_t r0 = g * kGroupRows;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const int64_t left = a.n - (r0 + w * 32);
      const uint32_t valid = left >= 32 ? 0xFFFFFFFFu : (left > 0 ? ((1u << left) - 1u) : 0u);
      pw[w] &= valid;
      my_pass += (unsigned long long)__popc(pw[w]);
    }
    __syncwarp();
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      uint32_t u = __reduce_or_sync(0xFFFFFFFFu, pw[w]);
      while (u != 0u) {
        int rb[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          rb[r] = -1;
          if (u != 0u) { rb[r] = __ffs(u) - 1; u &= u - 1u; }
        }
        float xv[4][VEC];
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (rb[r] >= 0)
            load_row<VEC>(a.X + (size_t)(r0 + w * 32 + rb[r]) * (size_t)a.d_pad + (size_t)lane * VEC, xv[r]);
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (rb[r] >= 0)
            score_row<VEC, NQ>(a, xv[r], qv, pw[w], rb[r], (uint32_t)(r0 + w * 32 + rb[r]), my_tau, my_pre, lane,
                               top, shift, dmask);
      }
    }
  }
  if (qlive && a.pass_cnt != nullptr) atomicAdd(&a.pass_cnt[gq], my_pass);

  if (a.mode == kHist) {
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      s_last = atomicAdd(a.done_ctr, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      hist_step(a, top, shift);
      __syncthreads();
      if (threadIdx.x == 0) *a.done_ctr = 0u;
    }
  }
}

template <int VEC, int NQ>
cudaError_t launch_one(const ScanArgs &a, int grid, cudaStream_t s) {
  const size_t smem = (size_t)(kScanThreads / 32) * (size_t)a.n_slots * 8 * sizeof(uint32_t);
  auto *fn = k_scan_gemv<VEC, NQ>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  fn<<<grid, kScanThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int VEC>
cudaError_t dispatch_nq(const ScanArgs &a, int nq_tmpl, int grid, cudaStream_t s) {
  switch (nq_tmpl) {
    case 1: return launch_one<VEC, 1>(a, grid, s);
    case 2: return launch_one<VEC, 2>(a, grid, s);
    case 4: return launch_one<VEC, 4>(a, grid, s);
    case 8: return launch_one<VEC, 8>(a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_scan_gemv(const ScanArgs &a, int nq_tmpl, int vec, int grid, cudaStream_t s) {
  switch (vec) {
    case 1: return dispatch_nq<1>(a, nq_tmpl, grid, s);
    case 2: return dispatch_nq<2>(a, nq_tmpl, grid, s);
    case 4: return dispatch_nq<4>(a, nq_tmpl, grid, s);
    case 8: return dispatch_nq<8>(a, nq_tmpl, grid, s);
    case 16: return dispatch_nq<16>(a, nq_tmpl, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lr
