// Deterministic block reductions (fixed shuffle tree, fixed warp order). Blocks of
// any size are supported: the last warp may be partial, and only its existing
// lanes take part in the shuffles.
#pragma once

#include <cuda_runtime.h>
#include <algorithm>

namespace jfft {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the existing lanes of a possibly partial warp (nl lanes, mask of them).
__device__ __forceinline__ double warp_sum_partial(double v, int nl) {
  const unsigned mask = nl >= 32 ? 0xffffffffu : ((1u << nl) - 1u);
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double t = __shfl_down_sync(mask, v, o);
    if (lane + o < nl) v += t;
  }
  return v;
}

// Sum over the block; the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[32];
  __syncthreads();
  const int w0 = threadIdx.x >> 5;
  const int nl = min(32, (int)blockDim.x - 32 * w0);
  v = nl == 32 ? warp_sum(v) : warp_sum_partial(v, nl);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) ws[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    r = lane < nw ? ws[lane] : 0.0;
    r = nl == 32 ? warp_sum(r) : warp_sum_partial(r, nl);
  }
  return r;
}

}  // namespace jfft
