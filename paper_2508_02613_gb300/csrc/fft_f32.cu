// FP32 instances of the Green / Green-Jacobi preconditioner passes (fft_passes.cuh)
// for the mixed-precision inner solve.
#include "fft_passes.cuh"

namespace jfft {

cudaError_t launch_green_precond_f32(const Grid& g, const FftPlanT<float>& p, const float* r, float* z, int nb,
                                     const float* js, bool jacobi, double* partial, int* nparts, CgState* done,
                                     cudaStream_t st, StageCtl sc, int64_t jcs) {
  return green_precond_t<float>(g, p, r, z, nb, js, jacobi, partial, nparts, done, st, sc, jcs);
}

template <>
cudaError_t launch_green_precond_xr<float>(const Grid& g, const FftPlanT<float>& p, float* x, float* r, const float* pv, const float* q,
                                        float* z, int nb, const float* js, bool jacobi, double* partial, int* nparts,
                                        CgState* cg, cudaStream_t st, StageCtl sc_rr, StageCtl sc, int64_t jcs) {
  return green_precond_xr_t<float>(g, p, x, r, pv, q, z, nb, js, jacobi, partial, nparts, cg, st, sc_rr, sc, jcs);
}

}  // namespace jfft
