// Device helpers shared by the scan kernels (included by each kernel file).
#pragma once

#include "lr_internal.h"

namespace lr {
namespace {

// CNF of launch-local query q over the current group's words (sw: [slot][8]),
// from the launch's clause lists qc (clause ranges per query), cl (slot ranges
// per clause) and cs (slot ids), which may sit in shared or global memory.
__device__ __forceinline__ void eval_cnf_lists(const int32_t *qc, const int32_t *cl, const int32_t *cs, int q,
                                               const uint32_t *sw, uint32_t (&pw)[8]) {
#pragma unroll
  for (int w = 0; w < 8; ++w) pw[w] = 0xFFFFFFFFu;
  const int c0 = qc[q], c1 = qc[q + 1];
  int t0 = cl[c0];
  for (int c = c0; c < c1; ++c) {
    uint32_t cw[8];
#pragma unroll
    for (int w = 0; w < 8; ++w) cw[w] = 0u;
    const int t1 = cl[c + 1];
    for (int t = t0; t < t1; ++t) {
      const uint4 *s = reinterpret_cast<const uint4 *>(sw + cs[t] * 8);
      const uint4 lo = s[0], hi = s[1];
      cw[0] |= lo.x; cw[1] |= lo.y; cw[2] |= lo.z; cw[3] |= lo.w;
      cw[4] |= hi.x; cw[5] |= hi.y; cw[6] |= hi.z; cw[7] |= hi.w;
    }
#pragma unroll
    for (int w = 0; w < 8; ++w) pw[w] &= cw[w];
    t0 = t1;
  }
}

__device__ __forceinline__ void eval_cnf(const ScanArgs &a, int q, const uint32_t *sw, uint32_t (&pw)[8]) {
  eval_cnf_lists(a.qc_off, a.cl_off, a.cl_slot, q, sw, pw);
}

// A query's CNF held in registers: up to 16 slot ids (one byte each, in clause
// order) and a mask of the terms that open a clause.  Evaluating it issues only
// independent shared-memory loads, no dependent global ones.
struct PackedCnf {
  uint32_t slot[4];
  uint32_t start;  // bit t: term t opens a new clause
  int nt;          // terms
  bool ok;         // false: the query does not fit (more than 16 terms)
};

// From clause lists qc (clause ranges per query), cl (slot ranges per clause)
// and cs (slot ids), in shared or global memory.
__device__ __forceinline__ PackedCnf pack_cnf_lists(const int32_t *qc, const int32_t *cl, const int32_t *cs, int q) {
  PackedCnf p;
  p.slot[0] = p.slot[1] = p.slot[2] = p.slot[3] = 0u;
  p.start = 0u;
  p.nt = 0;
  p.ok = true;
  const int c0 = qc[q], c1 = qc[q + 1];
  for (int c = c0; c < c1; ++c) {
    const int t0 = cl[c], t1 = cl[c + 1];
    for (int t = t0; t < t1; ++t) {
      const int s = cs[t];
      if (p.nt >= 16 || s > 255) {
        p.ok = false;
        return p;
      }
      if (t == t0) p.start |= 1u << p.nt;
      p.slot[p.nt >> 2] |= (uint32_t)s << ((p.nt & 3) * 8);
      ++p.nt;
    }
  }
  return p;
}

__device__ __forceinline__ PackedCnf pack_cnf(const ScanArgs &a, int q) {
  return pack_cnf_lists(a.qc_off, a.cl_off, a.cl_slot, q);
}

__device__ __forceinline__ void eval_packed(const PackedCnf &p, const uint32_t *sw, uint32_t (&pw)[8]) {
  uint32_t cw[8];
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    pw[w] = 0xFFFFFFFFu;
    cw[w] = 0u;
  }
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    if (t < p.nt) {
      if (t > 0 && ((p.start >> t) & 1u)) {
#pragma unroll
        for (int w = 0; w < 8; ++w) {
          pw[w] &= cw[w];
          cw[w] = 0u;
        }
      }
      const uint32_t s = (p.slot[t >> 2] >> ((t & 3) * 8)) & 0xFFu;
      const uint4 *src = reinterpret_cast<const uint4 *>(sw + s * 8);
      const uint4 lo = src[0], hi = src[1];
      cw[0] |= lo.x; cw[1] |= lo.y; cw[2] |= lo.z; cw[3] |= lo.w;
      cw[4] |= hi.x; cw[5] |= hi.y; cw[6] |= hi.z; cw[7] |= hi.w;
    }
  }
  if (p.nt > 0)
#pragma unroll
    for (int w = 0; w < 8; ++w) pw[w] &= cw[w];
}

// Digit step of the exact fallback: for every participating query find the
// digit whose bin holds the krem-th largest key, fix it in the prefix and clear
// the histogram.  Runs in the last CTA of a kHist launch; after the last digit
// (shift 0) the prefix is the selected key itself and becomes the query's tau.
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
      if (shift == 0 && a.tau_out && lane == 0) a.tau_out[gq] = a.prefix[gq];
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
      if (shift == 0 && a.tau_out) a.tau_out[gq] = a.prefix[gq];
    }
    __syncwarp();
    for (int i = lane; i < nb; i += 32) h[i] = 0u;
  }
}

}  // namespace
}  // namespace lr
