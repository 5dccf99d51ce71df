// FP64 fused multiply-add throughput probe (measurement support for the FP64 roofline
// peak; not part of the solver). Every thread runs kChains independent FMA chains of
// `iters` steps; the sum of the chains is written only if it takes one impossible value,
// which keeps the compiler from removing the work without adding memory traffic.
//
//   int jfft_probe_fp64_fma(int blocks, int threads, int iters, float* ms)
//     blocks x threads threads (threads <= 1024, a multiple of 32), each doing
//     kChains * iters FMAs; ms receives the kernel time (CUDA events, after one warm-up
//     launch). Returns 0 or the cudaError_t of the first failing call.
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;

__global__ void k_fp64_fma(double* sink, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = 1e-3 * threadIdx.x + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == -1.2345678e300) sink[0] = s;
}

}  // namespace

extern "C" int jfft_probe_fp64_fma(int blocks, int threads, int iters, float* ms) {
  if (blocks <= 0 || threads <= 0 || threads > 1024 || threads % 32 || iters <= 0 || !ms) return cudaErrorInvalidValue;
  double* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&sink, sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // a slightly below one and b small keep every chain bounded
  const double a = 0.999999999, b = 1e-9;
  if (e == cudaSuccess) {
    k_fp64_fma<<<blocks, threads>>>(sink, iters, a, b);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0);
  if (e == cudaSuccess) {
    k_fp64_fma<<<blocks, threads>>>(sink, iters, a, b);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (e1) cudaEventDestroy(e1);
  if (e0) cudaEventDestroy(e0);
  if (sink) cudaFree(sink);
  return (int)e;
}
