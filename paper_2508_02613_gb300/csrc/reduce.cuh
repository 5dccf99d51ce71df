// Deterministic block reductions (fixed shuffle tree, fixed warp order). Blocks of
// any size are supported: the last warp may be partial, and only its existing
// lanes take part in the shuffles.
#pragma once

#include <cuda_runtime.h>
#include <algorithm>

#include "jfft_internal.cuh"

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

// Update one right-hand side's CG scalars with the reduced value v of a stage
// (see ScalarStage): ||f||^2 and the stop threshold, gamma = r.z, alpha = gamma / p.q,
// the residual test and iteration count, beta and the new gamma.
__device__ __forceinline__ void apply_stage(CgState& s, int stage, double v, double tol, int stop_mode, int max_iter) {
  switch (stage) {
    case kStageInitFF:
    case kStageInitFFKeep: {
      // a continued recurrence keeps gamma (the last r.z) unless its previous run broke down
      const bool keep = stage == kStageInitFFKeep && s.done != kBreakdown && s.gamma > 0.0 && isfinite(s.gamma);
      s.ff = v;
      s.rr = v;
      s.rr_stop = stop_mode == 0 ? tol * tol * v : tol;
      s.iters = 0;
      s.max_iter = max_iter;
      s.alpha = 0.0;
      s.beta = 0.0;
      if (!keep) s.gamma = 0.0;
      s.done = (v == 0.0 || v <= s.rr_stop) ? kConverged : kRunning;
      if (!isfinite(v)) s.done = kBreakdown;
      break;
    }
    case kStageReplace:
      // beta = 0 (a fresh start, p = z) where no gamma was kept
      s.beta = s.gamma > 0.0 ? v / s.gamma : 0.0;
      s.gamma = v;
      if (!(v > 0.0) || !isfinite(v)) s.done = kBreakdown;
      break;
    case kStageInitGamma:
      s.gamma = v;
      s.beta = 0.0;
      if (!(v > 0.0) || !isfinite(v)) s.done = kBreakdown;
      break;
    case kStageAlpha:
      if (!(v > 0.0) || !isfinite(v)) s.done = kBreakdown;
      else s.alpha = s.gamma / v;
      break;
    case kStageRR:
      s.rr = v;
      s.iters += 1;
      if (!isfinite(v)) s.done = kBreakdown;
      else if (v <= s.rr_stop) s.done = kConverged;
      else if (s.iters >= s.max_iter) s.done = kNoConv;
      break;
    case kStageBeta:
      if (!isfinite(v)) {
        s.done = kBreakdown;
      } else {
        s.beta = v / s.gamma;
        s.gamma = v;
      }
      break;
    default:
      break;
  }
}

// Sum of p[0..n) in an order fixed by n alone (not by the block size): 256 strided
// sequential sums, then a pairwise tree. Every thread of the block must call it;
// the result is valid in every thread.
__device__ __forceinline__ double canonical_sum(const double* p, int n) {
  __shared__ double sh[256];
  __syncthreads();
  for (int v = threadIdx.x; v < 256; v += blockDim.x) {
    double a = 0.0;
    for (int i = v; i < n; i += 256) a += __ldcg(&p[i]);
    sh[v] = a;
  }
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    for (int i = threadIdx.x; i < s; i += blockDim.x) sh[i] += sh[i + s];
    __syncthreads();
  }
  return sh[0];
}

// Tail of a kernel that produces the partial sums of a scalar stage: thread 0 of
// every block has stored the block's partial at partial_row[slot]. The block that
// arrives last for right-hand side b (atomic counter) sums partial_row[0..nblocks)
// with canonical_sum and applies the stage to cg[b] (skipped for a right-hand side
// that is done, except at the two InitFF stages), then re-arms the counter. Every thread
// of the block must call it.
__device__ __forceinline__ void fused_stage_tail(const StageCtl& sc, CgState* cg, int b, const double* partial_row,
                                                 int nblocks) {
  if (sc.stage < 0) return;
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&sc.cnt[b], 1u);
    s_last = prev == (unsigned)(nblocks - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const double v = canonical_sum(partial_row, nblocks);
  if (threadIdx.x == 0) {
    if (sc.stage == kStageInitFF || sc.stage == kStageInitFFKeep || !cg[b].done)
      apply_stage(cg[b], sc.stage, v, sc.tol, sc.stop_mode, sc.max_iter);
    sc.cnt[b] = 0u;
  }
}

}  // namespace jfft
