// Deterministic block reductions (fixed shuffle tree, fixed warp order).
// Every caller launches a multiple of 32 threads.
#pragma once

#include <cuda_runtime.h>
#include <algorithm>

namespace jfft {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[32];
  __syncthreads();
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) ws[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    r = lane < nw ? ws[lane] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

}  // namespace jfft
