// FP64 instances of the Green / Green-Jacobi preconditioner passes (fft_passes.cuh)
// and the twiddle tables.
#include "fft_passes.cuh"

namespace jfft {

__global__ void k_twiddles(double2* tw, int n) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(-2.0 * (double)m / (double)n, &s, &c);
    tw[m] = make_double2(c, s);
  }
}

cudaError_t launch_twiddles(double2* tw, int n, cudaStream_t st) {
  JFFT_K("twiddles", st, k_twiddles<<<(n + 255) / 256, 256, 0, st>>>(tw, n));
  return cudaGetLastError();
}

cudaError_t launch_green_precond(const Grid& g, const FftPlan& p, const double* r, double* z, int nb,
                                 int64_t /*field_stride*/, const double* js, bool jacobi, double* partial, int* nparts,
                                 CgState* done, cudaStream_t st, StageCtl sc, int64_t jcs) {
  return green_precond_t<double>(g, p, r, z, nb, js, jacobi, partial, nparts, done, st, sc, jcs);
}

template <>
cudaError_t launch_green_precond_xr<double>(const Grid& g, const FftPlanT<double>& p, double* x, double* r, const double* pv, const double* q,
                                        double* z, int nb, const double* js, bool jacobi, double* partial, int* nparts,
                                        CgState* cg, cudaStream_t st, StageCtl sc_rr, StageCtl sc, int64_t jcs) {
  return green_precond_xr_t<double>(g, p, x, r, pv, q, z, nb, js, jacobi, partial, nparts, cg, st, sc_rr, sc, jcs);
}

}  // namespace jfft
