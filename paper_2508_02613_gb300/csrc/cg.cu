// PCG vector updates, inner-product partials and the device-resident scalar
// recurrences (S4, S7; textbook PCG, Saad Alg. 9.1, as cited in paper Sec. 3).
// Scalars never leave the device during the iteration: each stage kernel reduces
// the per-block partials of one right-hand side in a fixed order and updates its
// CgState; the vector kernels read alpha / beta from there and skip right-hand
// sides that are done.
#include "jfft_internal.cuh"
#include "reduce.cuh"

namespace jfft {

static int vec_blocks(int64_t n2) {  // n2 = number of double2 elements per rhs
  return (int)std::max<int64_t>(1, std::min<int64_t>((n2 + 255) / 256, 152 * 4));
}

// x += alpha p ; r -= alpha q ; partial ||r||^2
__global__ void __launch_bounds__(256) k_cg_xr(double2* __restrict__ x, double2* __restrict__ r,
                                               const double2* __restrict__ p, const double2* __restrict__ q,
                                               int64_t n2, int64_t stride2, const CgState* __restrict__ cg,
                                               double* __restrict__ partial) {
  const int b = blockIdx.y;
  if (cg[b].done) return;
  const double al = cg[b].alpha;
  const int64_t off = (int64_t)b * stride2;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
    double2 xv = x[off + i], rv = r[off + i];
    const double2 pv = p[off + i], qv = q[off + i];
    xv.x = fma(al, pv.x, xv.x);
    xv.y = fma(al, pv.y, xv.y);
    rv.x = fma(-al, qv.x, rv.x);
    rv.y = fma(-al, qv.y, rv.y);
    x[off + i] = xv;
    r[off + i] = rv;
    acc = fma(rv.x, rv.x, acc);
    acc = fma(rv.y, rv.y, acc);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) partial[(int64_t)b * kMaxPartials + blockIdx.x] = s;
}

cudaError_t launch_cg_xr(const Grid& g, double* x, double* r, const double* p, const double* q, int nb, int64_t stride,
                         CgState* cg, double* partial, int* nparts, cudaStream_t st) {
  const int64_t n2 = g.d * g.N / 2;
  const int bl = vec_blocks(n2);
  JFFT_K("cg_xr", st, k_cg_xr<<<dim3(bl, nb), 256, 0, st>>>((double2*)x, (double2*)r, (const double2*)p, (const double2*)q, n2, stride / 2,
                                       cg, partial));
  *nparts = bl;
  return cudaGetLastError();
}

// p = z + beta p
__global__ void __launch_bounds__(256) k_cg_p(double2* __restrict__ p, const double2* __restrict__ z, int64_t n2,
                                              int64_t stride2, const CgState* __restrict__ cg) {
  const int b = blockIdx.y;
  if (cg[b].done) return;
  const double be = cg[b].beta;
  const int64_t off = (int64_t)b * stride2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
    double2 pv = p[off + i];
    const double2 zv = z[off + i];
    pv.x = fma(be, pv.x, zv.x);
    pv.y = fma(be, pv.y, zv.y);
    p[off + i] = pv;
  }
}

cudaError_t launch_cg_p(const Grid& g, double* p, const double* z, int nb, int64_t stride, CgState* cg, cudaStream_t st) {
  const int64_t n2 = g.d * g.N / 2;
  JFFT_K("cg_p", st, k_cg_p<<<dim3(vec_blocks(n2), nb), 256, 0, st>>>((double2*)p, (const double2*)z, n2, stride / 2, cg));
  return cudaGetLastError();
}

// z = J r (J = (J^1/2)^2 per component; identity: z = r), partial r.z
__global__ void __launch_bounds__(256) k_jacobi_pc(Grid g, const double* __restrict__ r, double* __restrict__ z,
                                                   int64_t stride, const double* __restrict__ js, double3 jscale,
                                                   double void_js, int identity, const CgState* __restrict__ cg,
                                                   double* __restrict__ partial) {
  const int b = blockIdx.y;
  if (cg && cg[b].done) return;
  const int64_t off = (int64_t)b * stride;
  const int64_t n = g.d * g.N;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double rv = r[off + i];
    double zv = rv;
    if (!identity) {
      const int a = (int)(i / g.N);
      const double s = js[i - a * g.N];
      const double ka = a == 0 ? jscale.x : (a == 1 ? jscale.y : jscale.z);
      const double jh = s > 0.0 ? s * ka : void_js;
      zv = jh * jh * rv;
    }
    z[off + i] = zv;
    acc = fma(rv, zv, acc);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) partial[(int64_t)b * kMaxPartials + blockIdx.x] = s;
}

cudaError_t launch_jacobi_precond(const Grid& g, const double* r, double* z, int nb, int64_t stride, const double* js,
                                  const double* jscale, double void_js, bool identity, double* partial, int* nparts,
                                  const CgState* done, cudaStream_t st) {
  const int bl = vec_blocks(g.d * g.N / 2);
  JFFT_K("jacobi_pc", st, k_jacobi_pc<<<dim3(bl, nb), 256, 0, st>>>(g, r, z, stride, js, make_double3(jscale[0], jscale[1], jscale[2]), void_js,
                                           identity ? 1 : 0, done, partial));
  *nparts = bl;
  return cudaGetLastError();
}

// partial[b][blk] = sum a_b . c_b
__global__ void __launch_bounds__(256) k_dot(const double* __restrict__ a, const double* __restrict__ c, int64_t n,
                                             int64_t stride, double* __restrict__ partial) {
  const int b = blockIdx.y;
  const int64_t off = (int64_t)b * stride;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc = fma(a[off + i], c[off + i], acc);
  const double s = block_sum(acc);
  if (threadIdx.x == 0) partial[(int64_t)b * kMaxPartials + blockIdx.x] = s;
}

cudaError_t launch_dot(const Grid& g, const double* a, const double* c, int nb, int64_t stride, double* partial,
                       int* nparts, cudaStream_t st) {
  const int bl = vec_blocks(g.d * g.N / 2);
  JFFT_K("dot", st, k_dot<<<dim3(bl, nb), 256, 0, st>>>(a, c, g.d * g.N, stride, partial));
  *nparts = bl;
  return cudaGetLastError();
}

// Scalar stages; one block per rhs.
__global__ void __launch_bounds__(1024) k_scalars(int stage, CgState* __restrict__ cg, const double* __restrict__ partial,
                                                  int nparts, double tol, int stop_mode, int max_iter) {
  const int b = blockIdx.x;
  CgState& s = cg[b];
  if (stage != kStageInitFF && s.done) return;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += partial[(int64_t)b * kMaxPartials + i];
  const double v = block_sum(acc);
  if (threadIdx.x != 0) return;
  switch (stage) {
    case kStageInitFF: {
      s.ff = v;
      s.rr = v;
      s.rr_stop = stop_mode == 0 ? tol * tol * v : tol;
      s.iters = 0;
      s.max_iter = max_iter;
      s.alpha = 0.0;
      s.beta = 0.0;
      s.gamma = 0.0;
      s.done = (v == 0.0 || v <= s.rr_stop) ? kConverged : kRunning;
      if (!isfinite(v)) s.done = kBreakdown;
      break;
    }
    case kStageInitGamma:
      s.gamma = v;
      s.beta = 0.0;
      if (!(v > 0.0) || !isfinite(v)) s.done = kBreakdown;
      break;
    case kStageAlpha:
      if (!(v > 0.0) || !isfinite(v)) {
        s.done = kBreakdown;
      } else {
        s.alpha = s.gamma / v;
      }
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
  }
}

cudaError_t launch_cg_scalars(int stage, CgState* cg, const double* partial, int nparts, int nb, double tol,
                              int stop_mode, int max_iter, cudaStream_t st) {
  JFFT_K("cg_scalars", st, k_scalars<<<nb, 1024, 0, st>>>(stage, cg, partial, nparts, tol, stop_mode, max_iter));
  return cudaGetLastError();
}

// out[row] = sum_j partial[row * pstride + j], fixed order
__global__ void __launch_bounds__(256) k_reduce_rows(const double* __restrict__ partial, int nparts, int64_t pstride,
                                                     double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += partial[blockIdx.x * pstride + i];
  const double v = block_sum(acc);
  if (threadIdx.x == 0) out[blockIdx.x] = v;
}

cudaError_t launch_reduce_partials(const double* partial, int nparts, int rows, int64_t pstride, double* out,
                                   cudaStream_t st) {
  JFFT_K("reduce_rows", st, k_reduce_rows<<<rows, 256, 0, st>>>(partial, nparts, pstride, out));
  return cudaGetLastError();
}

// partial[(b d + a)][blk] = sum of field a of rhs b
__global__ void __launch_bounds__(256) k_field_sums(const double* __restrict__ x, int64_t N, double* __restrict__ partial) {
  const int row = blockIdx.y;
  const double* xr = x + (int64_t)row * N;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) acc += xr[i];
  const double s = block_sum(acc);
  if (threadIdx.x == 0) partial[(int64_t)row * kMaxPartials + blockIdx.x] = s;
}

cudaError_t launch_row_sums(const double* x, int rows, int64_t n, double* partial, int* nparts, cudaStream_t st) {
  const int bl = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 2));
  JFFT_K("row_sums", st, k_field_sums<<<dim3(bl, rows), 256, 0, st>>>(x, n, partial));
  *nparts = bl;
  return cudaGetLastError();
}

__global__ void k_sub_mean(double* __restrict__ x, int64_t N, const double* __restrict__ sums) {
  const int row = blockIdx.y;
  const double m = sums[row] / (double)N;
  double* xr = x + (int64_t)row * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) xr[i] -= m;
}

cudaError_t launch_sub_mean(double* x, int rows, int64_t n, const double* sums, cudaStream_t st) {
  const int bl = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 2));
  JFFT_K("sub_mean", st, k_sub_mean<<<dim3(bl, rows), 256, 0, st>>>(x, n, sums));
  return cudaGetLastError();
}

__global__ void k_fill(double* x, int64_t n, double v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] = v;
}

cudaError_t launch_fill(double* x, int64_t n, double v, cudaStream_t st) {
  const int bl = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8));
  JFFT_K("fill", st, k_fill<<<bl, 256, 0, st>>>(x, n, v));
  return cudaGetLastError();
}

}  // namespace jfft
