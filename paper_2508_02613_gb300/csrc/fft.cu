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

// Stage tables of the FP64 fused-multiply-add engine for line length L (first stage of
// radix RM, later ones as StageRadix): slot NS - RM + e NS + k holds (c, t) of W_{R NS}^q,
// q = lf_exponent(R, NS, e, k), for every stage of span NS >= RM, R = min(RM, L / NS);
// c = cos(2 pi q / (R NS)), t = Im / c; where the cosine is zero (w = +-i), c = 2^-60 and
// c t = +-1 exactly, the cosine's share then below 2^-60 |b|.
static_assert(radix_max<double>() == kFftRadix64, "stage-table size of the plan");
__global__ void k_lf_table(double2* dst, int L) {
  constexpr int RM = radix_max<double>();
  for (int NS = RM; NS < L;) {
    const int R = L / NS >= RM ? RM : L / NS;
    for (int i = threadIdx.x; i < (R - 1) * NS; i += blockDim.x) {
      const int e = i / NS, k = i % NS;
      const int q = lf_exponent(R, NS, e, k);
      double s, c;
      sincospi(-2.0 * (double)q / (double)(R * NS), &s, &c);
      if (c == 0.0) c = 0x1p-60;
      dst[NS - RM + i] = make_double2(c, s / c);
    }
    NS *= R;
  }
}

cudaError_t launch_lf_table(double2* dst, int L, cudaStream_t st) {
  if (L <= radix_max<double>()) return cudaErrorInvalidValue;
  JFFT_K("lf_table", st, k_lf_table<<<1, 256, 0, st>>>(dst, L));
  return cudaGetLastError();
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
