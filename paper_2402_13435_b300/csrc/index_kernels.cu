// Index construction and per-batch preparation kernels.
//
// Term storage (appendix "TBR", "Storing Dense Matrix"): the paper keeps a
// fixed-width attribute matrix per document and intersects sorted vectors.  On
// B300 the predicate becomes word-wise bit logic, so terms are stored
// term-major: term t owns a bitmap with bit j set iff job j holds t, padded to
// whole 256-row groups.  Frequent terms keep a resident bitmap; rare terms keep
// their posting list and are expanded into a workspace bitmap only when a batch
// uses them.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "lr_internal.h"

namespace lr {
namespace {

// One warp per row: copy a job row into the index layout [n][d_pad] (zero
// padded), normalised in FP32 for the cosine metric; non-finite values set err.
__global__ void k_rows_to_index(const float *in, float *out, int64_t n, int dim, int d_pad, int cosine,
                                uint32_t *err) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  const float *src = in + (size_t)row * (size_t)dim;
  float *dst = out + (size_t)row * (size_t)d_pad;
  float ss = 0.f;
  bool bad = false;
  for (int k = lane; k < dim; k += 32) {
    const float v = src[k];
    bad |= !isfinite(v);
    ss = fmaf(v, v, ss);
  }
  for (int off = 16; off >= 1; off >>= 1) ss += __shfl_xor_sync(0xFFFFFFFFu, ss, off);
  if (__any_sync(0xFFFFFFFFu, bad)) {
    if (lane == 0) atomicOr(err, 1u);
  }
  float scale = 1.f;
  if (cosine) scale = ss > 0.f ? 1.0f / sqrtf(ss) : 0.f;
  for (int k = lane; k < d_pad; k += 32) dst[k] = k < dim ? src[k] * scale : 0.f;
}

// Low-precision copy of the index rows (precision form).  BF16: each value
// rounded to nearest even.  FP8 e4m3: per-row scale = max_k |x_k| / 448 (1 for
// an all-zero row) and x8_k = e4m3(x_k / scale), round to nearest even with
// saturation to the finite range, so that scale * x8 approximates x with the
// row's largest magnitude mapped onto e4m3's largest finite value.  One warp
// per row.
__global__ void k_quantize_rows(const float *X, int64_t n, int d_pad, int elem, void *Xq, float *scale) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  const float *x = X + (size_t)row * d_pad;
  if (elem == kElemBF16) {
    __nv_bfloat16 *o = reinterpret_cast<__nv_bfloat16 *>(Xq) + (size_t)row * d_pad;
    for (int k = lane; k < d_pad; k += 32) o[k] = __float2bfloat16_rn(x[k]);
    return;
  }
  float amax = 0.f;
  for (int k = lane; k < d_pad; k += 32) amax = fmaxf(amax, fabsf(x[k]));
  for (int off = 16; off >= 1; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xFFFFFFFFu, amax, off));
  const float sc = amax > 0.f ? amax / kFp8Max : 1.f;
  __nv_fp8_storage_t *o = reinterpret_cast<__nv_fp8_storage_t *>(Xq) + (size_t)row * d_pad;
  for (int k = lane; k < d_pad; k += 32) o[k] = __nv_cvt_float_to_fp8(x[k] / sc, __NV_SATFINITE, __NV_E4M3);
  if (lane == 0) scale[row] = sc;
}

// Job-major 64-bit bitsets -> term-major 32-bit bitmap words.  Thread (jw, tw)
// reads the 32 jobs of word jw for terms [64*tw, 64*tw+64) and writes one word
// for each of those 64 terms.
__global__ void k_bitsets_to_termmajor(const uint64_t *bits, int64_t n, int vocab, uint32_t *out, int64_t n_words) {
  const int64_t jw = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int tw = blockIdx.y;
  const int64_t W = (vocab + 63) / 64;
  if (jw >= n_words) return;
  uint64_t v[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const int64_t row = jw * 32 + j;
    v[j] = row < n ? bits[(size_t)row * (size_t)W + tw] : 0ull;
  }
  for (int t = 0; t < 64; ++t) {
    const int term = tw * 64 + t;
    if (term >= vocab) break;
    uint32_t w = 0;
#pragma unroll
    for (int j = 0; j < 32; ++j) w |= (uint32_t)((v[j] >> t) & 1ull) << j;
    out[(size_t)term * (size_t)n_words + jw] = w;
  }
}

// Expand posting lists into bitmaps: bitmap i receives the postings of
// terms[i].  Lanes that hit the same word combine their bits before one atomic.
__global__ void k_scatter_postings(const int64_t *post_off, const uint32_t *post_ids, const int32_t *terms,
                                   int n_terms, uint32_t *bitmaps, int64_t n_words, int64_t n, uint32_t *err) {
  const int i = blockIdx.y;
  if (i >= n_terms) return;
  const int32_t t = terms[i];
  const int64_t b = post_off[t], e = post_off[t + 1];
  uint32_t *bm = bitmaps + (size_t)i * (size_t)n_words;
  const int lane = threadIdx.x & 31;
  for (int64_t p0 = b + ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)); p0 < e;
       p0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = p0 + lane;
    const bool valid = p < e;
    uint32_t id = valid ? post_ids[p] : 0u;
    if (valid && (int64_t)id >= n) {
      atomicOr(err, 4u);
      id = 0u;
    }
    const bool ok = valid && (int64_t)id < n;
    const unsigned act = __ballot_sync(0xFFFFFFFFu, ok);
    if (ok) {
      const uint32_t word = id >> 5;
      const unsigned peers = __match_any_sync(act, word);
      const uint32_t bits = __reduce_or_sync(peers, 1u << (id & 31u));
      if (lane == __ffs(peers) - 1) atomicOr(bm + word, bits);
    }
    __syncwarp();
  }
}

// Dense expansion of sorted posting lists into term-major bitmaps (one block
// per span of 2^span_log2 words of one term): the block ORs the span's
// postings into shared memory and writes every word of the span once, so the
// bitmaps need no clearing and no global atomics.  spans[t][j] is the offset
// of term t's first posting at or after row 32 * 2^span_log2 * j.
__global__ void k_expand_postings(const int64_t *post_off, const uint32_t *post_ids, const int32_t *spans,
                                  int n_spans, int span_log2, const int32_t *terms, uint32_t *bitmaps,
                                  int64_t n_words, int64_t n) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
  extern __shared__ __align__(16) uint32_t span_words[];
  const int j = blockIdx.x;
  const int32_t t = terms[blockIdx.y];
  const int sw = 1 << span_log2;
  const int64_t w0 = (int64_t)j << span_log2;
  const int64_t base = post_off[t];
  const int32_t *sp = spans + (size_t)t * (size_t)(n_spans + 1);
  const int64_t lo = base + sp[j], hi = base + sp[j + 1];
  uint4 *span4 = reinterpret_cast<uint4 *>(span_words);  // spans are whole multiples of 4 words
  for (int v = threadIdx.x; v < (sw >> 2); v += blockDim.x) span4[v] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  for (int64_t p = lo + threadIdx.x; p < hi; p += blockDim.x) {
    const uint32_t id = post_ids[p];
    const int64_t local = (int64_t)(id >> 5) - w0;
    if ((int64_t)id < n && local >= 0 && local < sw) atomicOr(&span_words[local], 1u << (id & 31u));
  }
  __syncthreads();
  // n_words and w0 are multiples of 8 words: 16-byte stores stay aligned and
  // a vector lies entirely inside or entirely past the bitmap
  uint4 *bm4 = reinterpret_cast<uint4 *>(bitmaps + (size_t)blockIdx.y * (size_t)n_words + w0);
  for (int v = threadIdx.x; v < (sw >> 2) && w0 + 4 * v < n_words; v += blockDim.x) bm4[v] = span4[v];
}

// Jobs holding each term (popcount of its term-major bitmap): one block per term.
__global__ void k_term_counts(const uint32_t *bitmaps, int64_t n_words, int64_t *out) {
  const uint32_t *bm = bitmaps + (size_t)blockIdx.x * (size_t)n_words;
  unsigned long long c = 0;
  for (int64_t w = threadIdx.x; w < n_words; w += blockDim.x) c += (unsigned long long)__popc(bm[w]);
  for (int off = 16; off >= 1; off >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, off);
  __shared__ unsigned long long s_c[32];
  if ((threadIdx.x & 31) == 0) s_c[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += s_c[i];
    out[blockIdx.x] = (int64_t)t;
  }
}

// One warp per query: copy into [B][d_pad] (zero padded), FP32-normalised for cosine.
__global__ void k_prep_queries(const float *in, float *out, int B, int dim, int d_pad, int cosine, uint32_t *err) {
  pdl_wait();  // launched by launch_pdl: the previous kernel's writes are visible from here on
  const int lane = threadIdx.x & 31;
  const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (q >= B) return;
  const float *src = in + (size_t)q * (size_t)dim;
  float ss = 0.f;
  bool bad = false;
  for (int k = lane; k < dim; k += 32) {
    const float v = src[k];
    bad |= !isfinite(v);
    ss = fmaf(v, v, ss);
  }
  for (int off = 16; off >= 1; off >>= 1) ss += __shfl_xor_sync(0xFFFFFFFFu, ss, off);
  if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) atomicOr(err, 8u);
  float scale = 1.f;
  if (cosine) scale = ss > 0.f ? 1.0f / sqrtf(ss) : 0.f;
  for (int k = lane; k < d_pad; k += 32) out[(size_t)q * (size_t)d_pad + k] = k < dim ? src[k] * scale : 0.f;
}

// Exact filter export (lr_filter_count): per 256-row group and query, the 8
// pass words; counts per query and optional bitmap rows (query q's row at
// out_bitmap + (q - out_row0) * out_words).
__global__ void __launch_bounds__(kScanThreads) k_filter_eval(const ScanArgs a, unsigned long long *pass_cnt,
                                                              uint32_t *out_bitmap, int64_t out_words,
                                                              int out_row0) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  uint32_t *sw = smem + (size_t)warp * (size_t)a.n_slots * 8;
  const bool qlive = lane < a.nq;
  unsigned long long my = 0;
  for (int64_t g = (int64_t)blockIdx.x * wpc + warp; g < a.n_groups; g += (int64_t)gridDim.x * wpc) {
    for (int s = lane; s < a.n_slots; s += 32) {
      const uint4 *src = reinterpret_cast<const uint4 *>(a.slot_bm[s] + g * kGroupWords);
      uint4 *dst = reinterpret_cast<uint4 *>(sw + s * 8);
      dst[0] = __ldg(src);
      dst[1] = __ldg(src + 1);
    }
    __syncwarp();
    if (qlive) {
      uint32_t pw[8];
#pragma unroll
      for (int w = 0; w < 8; ++w) pw[w] = 0xFFFFFFFFu;
      for (int c = a.qc_off[lane]; c < a.qc_off[lane + 1]; ++c) {
        uint32_t cw[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int t = a.cl_off[c]; t < a.cl_off[c + 1]; ++t) {
          const uint32_t *s = sw + a.cl_slot[t] * 8;
#pragma unroll
          for (int w = 0; w < 8; ++w) cw[w] |= s[w];
        }
#pragma unroll
        for (int w = 0; w < 8; ++w) pw[w] &= cw[w];
      }
      const int64_t r0 = g * kGroupRows;
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        const int64_t left = a.n - (r0 + w * 32);
        const uint32_t valid = left >= 32 ? 0xFFFFFFFFu : (left > 0 ? ((1u << left) - 1u) : 0u);
        pw[w] &= valid;
        my += (unsigned long long)__popc(pw[w]);
        const int64_t word = g * kGroupWords + w;
        if (out_bitmap != nullptr && word < out_words)
          out_bitmap[(size_t)(a.q_base + lane - out_row0) * (size_t)out_words + word] = pw[w];
      }
    }
    __syncwarp();
  }
  if (qlive) atomicAdd(&pass_cnt[a.q_base + lane], my);
}

}  // namespace

cudaError_t launch_rows_to_index(const float *in, float *out, int64_t n, int dim, int d_pad, int cosine,
                                 uint32_t *err, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int wpb = 8;
  k_rows_to_index<<<(unsigned)((n + wpb - 1) / wpb), wpb * 32, 0, s>>>(in, out, n, dim, d_pad, cosine, err);
  return cudaGetLastError();
}

cudaError_t launch_quantize_rows(const float *X, int64_t n, int d_pad, int elem, void *Xq, float *scale,
                                 cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int wpb = 8;
  k_quantize_rows<<<(unsigned)((n + wpb - 1) / wpb), wpb * 32, 0, s>>>(X, n, d_pad, elem, Xq, scale);
  return cudaGetLastError();
}

cudaError_t launch_bitsets_to_termmajor(const uint64_t *bits, int64_t n, int vocab, uint32_t *out, int64_t n_words,
                                        cudaStream_t s) {
  if (n_words <= 0 || vocab <= 0) return cudaSuccess;
  dim3 grid((unsigned)((n_words + 127) / 128), (unsigned)((vocab + 63) / 64));
  k_bitsets_to_termmajor<<<grid, 128, 0, s>>>(bits, n, vocab, out, n_words);
  return cudaGetLastError();
}

cudaError_t launch_scatter_postings(const int64_t *post_off, const uint32_t *post_ids, const int32_t *terms,
                                    int n_terms, uint32_t *bitmaps, int64_t n_words, int64_t n, uint32_t *err,
                                    cudaStream_t s) {
  for (int t0 = 0; t0 < n_terms; t0 += 65535) {  // grid.y is limited to 65535
    const int nt = n_terms - t0 < 65535 ? n_terms - t0 : 65535;
    dim3 grid(64, (unsigned)nt);
    k_scatter_postings<<<grid, 256, 0, s>>>(post_off, post_ids, terms + t0, nt, bitmaps + (size_t)t0 * n_words,
                                            n_words, n, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_expand_postings(const int64_t *post_off, const uint32_t *post_ids, const int32_t *spans,
                                   int n_spans, int span_log2, const int32_t *terms, int n_terms, uint32_t *bitmaps,
                                   int64_t n_words, int64_t n, cudaStream_t s) {
  const size_t smem = (size_t)4 << span_log2;
  if (smem > 48u * 1024u) return cudaErrorInvalidValue;
  for (int t0 = 0; t0 < n_terms; t0 += 65535) {  // grid.y is limited to 65535
    const int nt = n_terms - t0 < 65535 ? n_terms - t0 : 65535;
    const cudaError_t e =
        launch_pdl(k_expand_postings, dim3((unsigned)n_spans, (unsigned)nt), dim3(256), smem, s, post_off, post_ids,
                   spans, n_spans, span_log2, terms + t0, bitmaps + (size_t)t0 * n_words, n_words, n);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_term_counts(const uint32_t *bitmaps, int n_terms, int64_t n_words, int64_t *out, cudaStream_t s) {
  if (n_terms <= 0) return cudaSuccess;
  k_term_counts<<<n_terms, 256, 0, s>>>(bitmaps, n_words, out);
  return cudaGetLastError();
}

cudaError_t launch_prep_queries(const float *q_in, float *q_out, int B, int dim, int d_pad, int cosine,
                                uint32_t *err, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const int wpb = 8;
  return launch_pdl(k_prep_queries, dim3((unsigned)((B + wpb - 1) / wpb)), dim3(wpb * 32), 0, s, q_in, q_out, B, dim,
                    d_pad, cosine, err);
}

cudaError_t launch_filter_eval(const ScanArgs &a, unsigned long long *pass_cnt, uint32_t *out_bitmap,
                               int64_t out_words, int out_row0, int grid, cudaStream_t s) {
  const size_t smem = (size_t)(kScanThreads / 32) * (size_t)a.n_slots * 8 * sizeof(uint32_t);
  if (smem > 48 * 1024) {
    cudaError_t e = allow_dynamic_smem((const void *)k_filter_eval, (size_t)smem);
    if (e != cudaSuccess) return e;
  }
  k_filter_eval<<<grid, kScanThreads, smem, s>>>(a, pass_cnt, out_bitmap, out_words, out_row0);
  return cudaGetLastError();
}

}  // namespace lr
