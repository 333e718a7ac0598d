// Warp-wide bit-matrix helpers shared by the kernels.
#pragma once

#include <stdint.h>

namespace lr {

// One exchange stage of the 32x32 transpose: lanes J apart swap the bit blocks
// selected by M.
template <int J, uint32_t M>
__device__ __forceinline__ uint32_t transpose_stage(uint32_t x, int lane) {
  const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, J);
  return (lane & J) ? (((y >> J) & M) | (x & ~M)) : ((x & M) | ((y & M) << J));
}

// 32x32 bit-matrix transpose across a full warp: lane i holds row i on entry
// (bit c = column c) and column i on exit (bit r = row r).
__device__ __forceinline__ uint32_t bit_transpose32(uint32_t x, int lane) {
  x = transpose_stage<16, 0x0000FFFFu>(x, lane);
  x = transpose_stage<8, 0x00FF00FFu>(x, lane);
  x = transpose_stage<4, 0x0F0F0F0Fu>(x, lane);
  x = transpose_stage<2, 0x33333333u>(x, lane);
  return transpose_stage<1, 0x55555555u>(x, lane);
}

}  // namespace lr
