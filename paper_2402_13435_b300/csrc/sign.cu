// Sign-bit pre-selection (appendix "Quantization"; Sec. 5.3, a quantisation
// akin to OP+ORP): every job row carries a code of nbits sign bits, each the
// sign of a randomly signed sum over a bin of permuted coordinates; a query is
// compared with every passing job by Eq. 4 -- the number of bit positions
// where the two codes agree, popcount(~(x XOR y)) over 64-bit words -- and only
// the jobs of the highest agreement levels go on to the exact FP32 scoring.
//
// Kernels:
//   k_sign_encode     codes of rows (index build) or of queries (per search):
//                     one warp per row, the row and the projection in shared
//                     memory, FP32 sums in bin order, 32 bits per ballot;
//   k_sign_scan       per job row (one thread) and query: the pass bit (from
//                     the batch's pass bitmaps), Eq. 4 against the query code
//                     held in shared memory, then either a histogram of the
//                     agreement levels (shared memory, added to the query's
//                     histogram) or, given the level t of the query, the job id
//                     appended to the query's candidate list when its level is
//                     at least t;
//   k_sign_levels     per query: the level t (highest level with at least
//                     min(quantK, #passing) jobs at or above it, one higher when
//                     that set would pass the list's capacity);
//   k_sign_rescore    the kept jobs' FP32 scores (one warp per job), written in
//                     place as selection keys for the library's exact top-K.
#include "lr_internal.h"

namespace lr {
namespace {

constexpr int kSgThreads = 256;

__global__ void __launch_bounds__(kSgThreads) k_sign_encode(const float *x, int64_t n, int dim, int64_t ld,
                                                            int nbits, int bin, const int32_t *idx, const int8_t *sgn,
                                                            uint64_t *codes) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int total = nbits * bin;
  int32_t *s_idx = reinterpret_cast<int32_t *>(sm);
  int8_t *s_sgn = reinterpret_cast<int8_t *>(s_idx + total);
  float *s_row = reinterpret_cast<float *>(sm + (((size_t)total * 5 + 15) / 16) * 16);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const int32_t v = idx[i];
    s_idx[i] = (v >= 0 && v < dim) ? v : 0;  // keeps every read inside the staged row
    s_sgn[i] = sgn[i];
  }
  __syncthreads();
  float *row = s_row + (size_t)warp * dim;
  const int W = nbits / 64;
  for (int64_t r = (int64_t)blockIdx.x * nw + warp; r < n; r += (int64_t)gridDim.x * nw) {
    const float *src = x + (size_t)r * (size_t)ld;
    for (int k = lane; k < dim; k += 32) row[k] = src[k];
    __syncwarp();
    for (int w = 0; w < W; ++w) {
      uint32_t half[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int b = w * 64 + h * 32 + lane;
        float s = 0.0f;
        for (int m = 0; m < bin; ++m) {
          const float v = row[s_idx[b * bin + m]];
          s = __fadd_rn(s, s_sgn[b * bin + m] > 0 ? v : -v);
        }
        half[h] = __ballot_sync(0xFFFFFFFFu, s > 0.0f);
      }
      if (lane == 0) codes[(size_t)r * W + w] = (uint64_t)half[0] | ((uint64_t)half[1] << 32);
    }
    __syncwarp();
  }
}

template <int W>
__global__ void __launch_bounds__(kSgThreads) k_sign_scan(const SignScanArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  uint64_t *qc = reinterpret_cast<uint64_t *>(sm);                     // [nq][W]
  uint32_t *hist = reinterpret_cast<uint32_t *>(qc + (size_t)a.nq * W);  // [nq][nbits + 1] (mode 0)
  const int L = a.nbits + 1;
  for (int i = threadIdx.x; i < a.nq * W; i += blockDim.x) qc[i] = a.qcodes[(size_t)a.q_base * W + i];
  if (a.mode == 0)
    for (int i = threadIdx.x; i < a.nq * L; i += blockDim.x) hist[i] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  // whole warps walk consecutive rows, so the lanes share each pass word
  for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x; r0 < a.n; r0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = r0 + threadIdx.x;
    const bool live = r < a.n;
    uint64_t c[W];
    if (live) {
      const uint4 *src = reinterpret_cast<const uint4 *>(a.codes + (size_t)r * W);
#pragma unroll
      for (int i = 0; i < W / 2; ++i) {
        const uint4 v = __ldg(src + i);
        c[2 * i] = (uint64_t)v.x | ((uint64_t)v.y << 32);
        c[2 * i + 1] = (uint64_t)v.z | ((uint64_t)v.w << 32);
      }
    }
    for (int q = 0; q < a.nq; ++q) {
      const int gq = a.q_base + q;
      bool pass = false;
      if (live) pass = (__ldg(a.pass + (size_t)gq * a.pass_words + (r >> 5)) >> (r & 31)) & 1u;
      int s = 0;
      if (pass) {
#pragma unroll
        for (int w = 0; w < W; ++w) s += __popcll(~(c[w] ^ qc[q * W + w]));
      }
      if (a.mode == 0) {
        if (pass) atomicAdd(&hist[q * L + s], 1u);
      } else {
        const bool take = pass && s >= a.level[gq];
        const unsigned m = __ballot_sync(0xFFFFFFFFu, take);
        if (m != 0u) {
          const int lead = __ffs(m) - 1;
          uint32_t base = 0;
          if (lane == lead) base = atomicAdd(&a.cnt[gq], (uint32_t)__popc(m));
          base = __shfl_sync(0xFFFFFFFFu, base, lead);
          const uint32_t pos = base + (uint32_t)__popc(m & ((1u << lane) - 1u));
          if (take && pos < (uint32_t)a.cap) a.buf[(size_t)gq * a.cap + pos] = (uint64_t)r;
        }
      }
    }
  }
  if (a.mode == 0) {
    __syncthreads();
    for (int i = threadIdx.x; i < a.nq * L; i += blockDim.x)
      if (hist[i]) atomicAdd(&a.hist[(size_t)(a.q_base + i / L) * a.hist_stride + i % L], hist[i]);
  }
}

// One warp per query: the level t from the agreement histogram.
__global__ void k_sign_levels(const uint32_t *hist, int hist_stride, int nbits, int B, const int64_t *quant_k,
                              const unsigned long long *pass_cnt, int64_t cap, int32_t *level,
                              unsigned long long *ncand) {
  const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= B) return;
  const uint32_t *h = hist + (size_t)q * hist_stride;
  const unsigned long long P = pass_cnt[q];
  const unsigned long long want = (unsigned long long)quant_k[q] < P ? (unsigned long long)quant_k[q] : P;
  if (want == 0ull) {
    if (lane == 0) {
      level[q] = nbits + 1;
      ncand[q] = 0ull;
    }
    return;
  }
  // runs of levels per lane from the top; prefix sums over lanes find the run
  const int L = nbits + 1, per = (L + 31) / 32, top0 = nbits - lane * per;
  unsigned long long sum = 0;
  for (int j = 0; j < per; ++j)
    if (top0 - j >= 0) sum += h[top0 - j];
  unsigned long long incl = sum;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long t = __shfl_up_sync(0xFFFFFFFFu, incl, off);
    if (lane >= off) incl += t;
  }
  const unsigned long long excl = incl - sum;
  const unsigned hit = __ballot_sync(0xFFFFFFFFu, excl < want && want <= incl);
  if (hit != 0u && lane == __ffs(hit) - 1) {
    unsigned long long cum = excl;
    int t = 0;
    for (int j = 0; j < per; ++j) {
      const int lv = top0 - j;
      if (lv < 0) break;
      cum += h[lv];
      if (cum >= want) {
        t = lv;
        break;
      }
    }
    if (cum > (unsigned long long)cap) {  // the level itself would pass the list's capacity
      cum -= h[t];
      t += 1;
    }
    level[q] = t;
    ncand[q] = cum;
  }
}

// FP32 score of every kept job (one warp per job, float4 loads of the row),
// stored over the job id as the selection key.
__global__ void __launch_bounds__(kSgThreads) k_sign_rescore(const float *X, int d_pad, const float *Q,
                                                             uint64_t *buf, int64_t cap, const uint32_t *cnt) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
  const int q = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int64_t nc = (int64_t)cnt[q] < cap ? (int64_t)cnt[q] : cap;
  const float *qv = Q + (size_t)q * d_pad;
  uint64_t *b = buf + (size_t)q * cap;
  const int nv = d_pad / 4;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nc;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const uint32_t id = (uint32_t)b[i];
    const float4 *xr = reinterpret_cast<const float4 *>(X + (size_t)id * d_pad);
    const float4 *qr = reinterpret_cast<const float4 *>(qv);
    float p = 0.f;
    for (int v = lane; v < nv; v += 32) {
      const float4 x = __ldg(xr + v), y = __ldg(qr + v);
      p = fmaf(x.x, y.x, p);
      p = fmaf(x.y, y.y, p);
      p = fmaf(x.z, y.z, p);
      p = fmaf(x.w, y.w, p);
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) p += __shfl_xor_sync(0xFFFFFFFFu, p, off);
    __syncwarp();
    if (lane == 0) b[i] = make_key(p, id);
  }
}

}  // namespace

size_t sign_encode_smem(int nbits, int bin, int dim) {
  return (((size_t)nbits * bin * 5 + 15) / 16) * 16 + (size_t)(kSgThreads / 32) * dim * sizeof(float);
}

cudaError_t launch_sign_encode(const float *x, int64_t n, int dim, int64_t ld, int nbits, int bin, const int32_t *idx,
                               const int8_t *sgn, uint64_t *codes, int num_sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t smem = sign_encode_smem(nbits, bin, dim);
  if (smem > 48 * 1024) {
    const cudaError_t e = allow_dynamic_smem((const void *)k_sign_encode, smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t want = (n + 7) / 8;
  const int grid = (int)(want < (int64_t)num_sms * 8 ? want : (int64_t)num_sms * 8);
  k_sign_encode<<<grid, kSgThreads, smem, s>>>(x, n, dim, ld, nbits, bin, idx, sgn, codes);
  return cudaGetLastError();
}

cudaError_t launch_sign_scan(const SignScanArgs &a, int num_sms, cudaStream_t s) {
  const int W = a.nbits / 64;
  const size_t smem = (size_t)a.nq * W * 8 + (a.mode == 0 ? (size_t)a.nq * (a.nbits + 1) * 4 : 0);
  const void *fn = nullptr;
  switch (W) {
    case 2: fn = (const void *)k_sign_scan<2>; break;
    case 4: fn = (const void *)k_sign_scan<4>; break;
    case 8: fn = (const void *)k_sign_scan<8>; break;
    case 16: fn = (const void *)k_sign_scan<16>; break;
    default: return cudaErrorInvalidValue;
  }
  if (smem > 48 * 1024) {
    const cudaError_t e = allow_dynamic_smem(fn, smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t want = (a.n + kSgThreads - 1) / kSgThreads;
  const int per_sm = smem > 100 * 1024 ? 2 : 4;
  const int grid = (int)(want < (int64_t)num_sms * per_sm ? want : (int64_t)num_sms * per_sm);
  switch (W) {
    case 2: k_sign_scan<2><<<grid, kSgThreads, smem, s>>>(a); break;
    case 4: k_sign_scan<4><<<grid, kSgThreads, smem, s>>>(a); break;
    case 8: k_sign_scan<8><<<grid, kSgThreads, smem, s>>>(a); break;
    default: k_sign_scan<16><<<grid, kSgThreads, smem, s>>>(a); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_sign_levels(const uint32_t *hist, int hist_stride, int nbits, int B, const int64_t *quant_k,
                               const unsigned long long *pass_cnt, int64_t cap, int32_t *level,
                               unsigned long long *ncand, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  k_sign_levels<<<(B + 7) / 8, 256, 0, s>>>(hist, hist_stride, nbits, B, quant_k, pass_cnt, cap, level, ncand);
  return cudaGetLastError();
}

cudaError_t launch_sign_rescore(const float *X, int d_pad, const float *Q, uint64_t *buf, int64_t cap,
                                const uint32_t *cnt, int B, int num_sms, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  int gx = (4 * num_sms + B - 1) / B;
  if (gx < 1) gx = 1;
  return launch_pdl(k_sign_rescore, dim3((unsigned)gx, (unsigned)B), dim3(kSgThreads), 0, s, X, d_pad, Q, buf, cap, cnt);
}

}  // namespace lr

using namespace lr;

namespace {
bool sign_dev_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}
}  // namespace

extern "C" lr_status lr_sign_encode(const float *x, int64_t n, int32_t dim, int32_t nbits, int32_t bin,
                                    const int32_t *idx, const int8_t *sgn, uint64_t *codes, void *stream) {
  if (!x || !idx || !sgn || !codes) return fail(LR_ERR_INVALID, "lr_sign_encode: null pointer");
  if (n < 1 || dim < 1 || dim > 256) return fail(LR_ERR_INVALID, "lr_sign_encode: need n >= 1 and dim in [1, 256]");
  if (nbits != 128 && nbits != 256 && nbits != 512 && nbits != 1024)
    return fail(LR_ERR_INVALID, "lr_sign_encode: nbits must be 128, 256, 512 or 1024");
  if (bin < 1 || (int64_t)nbits * bin > 32768) return fail(LR_ERR_INVALID, "lr_sign_encode: nbits * bin <= 32768");
  if (reinterpret_cast<uintptr_t>(codes) % 16 != 0) return fail(LR_ERR_INVALID, "lr_sign_encode: codes 16-byte aligned");
  if (!sign_dev_ptr(x) || !sign_dev_ptr(idx) || !sign_dev_ptr(sgn) || !sign_dev_ptr(codes))
    return fail(LR_ERR_INVALID, "lr_sign_encode: every array must be device memory");
  int dev = 0, sms = 148;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = launch_sign_encode(x, n, dim, dim, nbits, bin, idx, sgn, codes, sms, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "lr_sign_encode");
  return LR_OK;
}
