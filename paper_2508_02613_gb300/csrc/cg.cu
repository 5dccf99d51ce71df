// PCG vector updates, inner-product partials and the device-resident scalar
// recurrences (S4, S7; textbook PCG, Saad Alg. 9.1, as cited in paper Sec. 3).
// Scalars never leave the device during the iteration: each stage kernel reduces
// the per-block partials of one right-hand side in a fixed order and updates its
// CgState; the vector kernels read alpha / beta from there and skip right-hand
// sides that are done. Vector kernels are templated on the working precision T;
// the scalars and every reduction above the thread level stay in FP64.
#include "jfft_internal.cuh"
#include "reduce.cuh"

namespace jfft {

static int vec_blocks(int64_t n2) {  // n2 = number of 2-vectors per rhs
  return (int)std::max<int64_t>(1, std::min<int64_t>((n2 + 255) / 256, 152 * 4));
}

template <typename T> static const char* nm(const char* d64, const char* d32) { return sizeof(T) == 8 ? d64 : d32; }

// 16-byte vectors of the working precision (four floats or two doubles).
template <typename T> struct V16;
template <> struct V16<float> { using t = float4; static constexpr int n = 4; };
template <> struct V16<double> { using t = double2; static constexpr int n = 2; };

static int vec16_blocks(int64_t n16) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n16 + 511) / 512, 152 * 4));
}

// x += alpha p ; r -= alpha q ; partial ||r||^2. Each thread handles two 16-byte
// vectors per loop trip so that more loads are in flight.
template <typename T>
__global__ void __launch_bounds__(256) k_cg_xr(typename V16<T>::t* __restrict__ x, typename V16<T>::t* __restrict__ r,
                                               const typename V16<T>::t* __restrict__ p,
                                               const typename V16<T>::t* __restrict__ q, int64_t n16, int64_t stride16,
                                               CgState* __restrict__ cg, double* __restrict__ partial, StageCtl sc) {
  using V = typename V16<T>::t;
  constexpr int NV = V16<T>::n;
  const int b = blockIdx.y;
  if (cg[b].done) return;
  const T al = (T)cg[b].alpha;
  const int64_t off = (int64_t)b * stride16;
  T acc = T(0);
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n16; i += 2 * step) {
    const int64_t i2 = i + step;
    const bool two = i2 < n16;
    V xv[2], rv[2], pv[2], qv[2];
    xv[0] = x[off + i]; rv[0] = r[off + i]; pv[0] = p[off + i]; qv[0] = q[off + i];
    if (two) { xv[1] = x[off + i2]; rv[1] = r[off + i2]; pv[1] = p[off + i2]; qv[1] = q[off + i2]; }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (u == 1 && !two) break;
      T* xa = reinterpret_cast<T*>(&xv[u]);
      T* ra = reinterpret_cast<T*>(&rv[u]);
      const T* pa = reinterpret_cast<const T*>(&pv[u]);
      const T* qa = reinterpret_cast<const T*>(&qv[u]);
#pragma unroll
      for (int c = 0; c < NV; ++c) {
        xa[c] = fma(al, pa[c], xa[c]);
        ra[c] = fma(-al, qa[c], ra[c]);
        acc = fma(ra[c], ra[c], acc);
      }
    }
    x[off + i] = xv[0];
    r[off + i] = rv[0];
    if (two) { x[off + i2] = xv[1]; r[off + i2] = rv[1]; }
  }
  const double sm = block_sum((double)acc);
  if (threadIdx.x == 0) partial[(int64_t)b * kMaxPartials + blockIdx.x] = sm;
  fused_stage_tail(sc, cg, b, partial + (int64_t)b * kMaxPartials, gridDim.x);
}

template <typename T>
cudaError_t launch_cg_xr(const Grid& g, T* x, T* r, const T* p, const T* q, int nb, int64_t stride, CgState* cg,
                         double* partial, int* nparts, cudaStream_t st, StageCtl sc) {
  using V = typename V16<T>::t;
  const int64_t n16 = g.d * g.N / V16<T>::n;
  const int bl = vec16_blocks(n16);
  JFFT_K(nm<T>("cg_xr", "cg_xr_f32"), st,
         k_cg_xr<T><<<dim3(bl, nb), 256, 0, st>>>((V*)x, (V*)r, (const V*)p, (const V*)q, n16, stride / V16<T>::n,
                                                  cg, partial, sc));
  *nparts = bl;
  return cudaGetLastError();
}
template cudaError_t launch_cg_xr<double>(const Grid&, double*, double*, const double*, const double*, int, int64_t,
                                          CgState*, double*, int*, cudaStream_t, StageCtl);
template cudaError_t launch_cg_xr<float>(const Grid&, float*, float*, const float*, const float*, int, int64_t,
                                         CgState*, double*, int*, cudaStream_t, StageCtl);

// p = z + beta p (p = z where beta = 0, so that a p left over from an earlier run is
// never read then)
template <typename T>
__global__ void __launch_bounds__(256) k_cg_p(typename V16<T>::t* __restrict__ p, const typename V16<T>::t* __restrict__ z,
                                              int64_t n16, int64_t stride16, const CgState* __restrict__ cg) {
  using V = typename V16<T>::t;
  constexpr int NV = V16<T>::n;
  const int b = blockIdx.y;
  if (cg[b].done) return;
  const T be = (T)cg[b].beta;
  const int64_t off = (int64_t)b * stride16;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n16; i += 2 * step) {
    const int64_t i2 = i + step;
    const bool two = i2 < n16;
    V pv[2], zv[2];
    pv[0] = p[off + i]; zv[0] = z[off + i];
    if (two) { pv[1] = p[off + i2]; zv[1] = z[off + i2]; }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      T* pa = reinterpret_cast<T*>(&pv[u]);
      const T* za = reinterpret_cast<const T*>(&zv[u]);
#pragma unroll
      for (int c = 0; c < NV; ++c) pa[c] = be == T(0) ? za[c] : fma(be, pa[c], za[c]);
    }
    p[off + i] = pv[0];
    if (two) p[off + i2] = pv[1];
  }
}

template <typename T>
cudaError_t launch_cg_p(const Grid& g, T* p, const T* z, int nb, int64_t stride, CgState* cg, cudaStream_t st) {
  using V = typename V16<T>::t;
  const int64_t n16 = g.d * g.N / V16<T>::n;
  JFFT_K(nm<T>("cg_p", "cg_p_f32"), st,
         k_cg_p<T><<<dim3(vec16_blocks(n16), nb), 256, 0, st>>>((V*)p, (const V*)z, n16, stride / V16<T>::n, cg));
  return cudaGetLastError();
}
template cudaError_t launch_cg_p<double>(const Grid&, double*, const double*, int, int64_t, CgState*, cudaStream_t);
template cudaError_t launch_cg_p<float>(const Grid&, float*, const float*, int, int64_t, CgState*, cudaStream_t);

// z = J r (J = (J^1/2)^2 per DOF from the resolved table; identity: z = r), partial r.z
template <typename T>
__global__ void __launch_bounds__(256) k_jacobi_pc(Grid g, const T* __restrict__ r, T* __restrict__ z, int64_t stride,
                                                   const T* __restrict__ js, int identity, CgState* __restrict__ cg,
                                                   double* __restrict__ partial, StageCtl sc, int64_t jcs) {
  const int b = blockIdx.y;
  if (cg && cg[b].done) return;
  const int64_t off = (int64_t)b * stride;
  const int64_t n = g.d * g.N;
  T acc = T(0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T rv = r[off + i];
    T zv = rv;
    if (!identity) {
      const int a = (int)(i / g.N);
      const T jh = js[i - a * g.N + a * jcs];
      zv = jh * jh * rv;
    }
    z[off + i] = zv;
    acc = fma(rv, zv, acc);
  }
  const double s = block_sum((double)acc);
  if (threadIdx.x == 0) partial[(int64_t)b * kMaxPartials + blockIdx.x] = s;
  fused_stage_tail(sc, cg, b, partial + (int64_t)b * kMaxPartials, gridDim.x);
}

cudaError_t launch_jacobi_precond(const Grid& g, const double* r, double* z, int nb, int64_t stride, const double* js,
                                  bool identity, double* partial, int* nparts, CgState* done, cudaStream_t st,
                                  StageCtl sc, int64_t jcs) {
  const int bl = vec_blocks(g.d * g.N / 2);
  JFFT_K("jacobi_pc", st,
         k_jacobi_pc<double><<<dim3(bl, nb), 256, 0, st>>>(g, r, z, stride, js, identity ? 1 : 0, done, partial, sc,
                                                           jcs));
  *nparts = bl;
  return cudaGetLastError();
}

cudaError_t launch_jacobi_precond_f32(const Grid& g, const float* r, float* z, int nb, int64_t stride, const float* js,
                                      bool identity, double* partial, int* nparts, CgState* done, cudaStream_t st,
                                      StageCtl sc, int64_t jcs) {
  const int bl = vec_blocks(g.d * g.N / 2);
  JFFT_K("jacobi_pc_f32", st,
         k_jacobi_pc<float><<<dim3(bl, nb), 256, 0, st>>>(g, r, z, stride, js, identity ? 1 : 0, done, partial, sc,
                                                          jcs));
  *nparts = bl;
  return cudaGetLastError();
}

// partial[b][blk] = sum a_b . c_b
template <typename T>
__global__ void __launch_bounds__(256) k_dot(const T* __restrict__ a, const T* __restrict__ c, int64_t n,
                                             int64_t stride, double* __restrict__ partial, CgState* cg, StageCtl sc) {
  const int b = blockIdx.y;
  const int64_t off = (int64_t)b * stride;
  T acc = T(0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc = fma(a[off + i], c[off + i], acc);
  const double s = block_sum((double)acc);
  if (threadIdx.x == 0) partial[(int64_t)b * kMaxPartials + blockIdx.x] = s;
  fused_stage_tail(sc, cg, b, partial + (int64_t)b * kMaxPartials, gridDim.x);
}

template <typename T>
cudaError_t launch_dot(const Grid& g, const T* a, const T* c, int nb, int64_t stride, double* partial, int* nparts,
                       cudaStream_t st, CgState* cg, StageCtl sc) {
  const int bl = vec_blocks(g.d * g.N / 2);
  JFFT_K(nm<T>("dot", "dot_f32"), st, k_dot<T><<<dim3(bl, nb), 256, 0, st>>>(a, c, g.d * g.N, stride, partial, cg, sc));
  *nparts = bl;
  return cudaGetLastError();
}
template cudaError_t launch_dot<double>(const Grid&, const double*, const double*, int, int64_t, double*, int*,
                                        cudaStream_t, CgState*, StageCtl);
template cudaError_t launch_dot<float>(const Grid&, const float*, const float*, int, int64_t, double*, int*,
                                       cudaStream_t, CgState*, StageCtl);

// Loop condition of the device-side PCG loop (a CUDA graph WHILE node whose body is
// one chunk of iterations): counts the chunk and continues while any right-hand
// side is running and fewer than cap chunks have run.
__global__ void k_cg_continue(const CgState* __restrict__ cg, int nb, int* __restrict__ chunks, int cap,
                              cudaGraphConditionalHandle cond) {
  if (threadIdx.x != 0) return;
  const int n = chunks[0] + 1;
  chunks[0] = n;
  bool running = false;
  for (int b = 0; b < nb; ++b) running = running || cg[b].done == kRunning;
  cudaGraphSetConditional(cond, (running && n < cap) ? 1u : 0u);
}

cudaError_t launch_cg_continue(const CgState* cg, int nb, int* chunks, int cap, cudaGraphConditionalHandle cond,
                               cudaStream_t st) {
  JFFT_K("cg_continue", st, k_cg_continue<<<1, 32, 0, st>>>(cg, nb, chunks, cap, cond));
  return cudaGetLastError();
}

// Scalar stages as a separate launch; one block per rhs (the same reduction order
// and update as the fused tails of the producing kernels).
// keep (kStageInitFFKeep only, may be NULL): right-hand sides with keep[b] != 2 start
// afresh (kStageInitFF).
__global__ void __launch_bounds__(256) k_scalars(int stage, CgState* __restrict__ cg, const double* __restrict__ partial,
                                                 int nparts, double tol, int stop_mode, int max_iter,
                                                 const int* __restrict__ keep) {
  const int b = blockIdx.x;
  CgState& s = cg[b];
  if (stage == kStageInitFFKeep && keep && keep[b] != 2) stage = kStageInitFF;
  if (stage != kStageInitFF && stage != kStageInitFFKeep && s.done) return;
  const double v = canonical_sum(partial + (int64_t)b * kMaxPartials, nparts);
  if (threadIdx.x == 0) apply_stage(s, stage, v, tol, stop_mode, max_iter);
}

cudaError_t launch_cg_scalars(int stage, CgState* cg, const double* partial, int nparts, int nb, double tol,
                              int stop_mode, int max_iter, cudaStream_t st, const int* keep) {
  JFFT_K("cg_scalars", st, k_scalars<<<nb, 256, 0, st>>>(stage, cg, partial, nparts, tol, stop_mode, max_iter, keep));
  return cudaGetLastError();
}

// partial[b][blk] = sum (r64 - r32)^2 over right-hand side b: the distance between the
// FP64 residual and the FP32 recurrence residual it replaces.
__global__ void __launch_bounds__(256) k_gap(const double* __restrict__ r64, const float* __restrict__ r32, int64_t n,
                                             double* __restrict__ partial) {
  const int b = blockIdx.y;
  const int64_t off = (int64_t)b * n;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double e = r64[off + i] - (double)r32[off + i];
    acc = fma(e, e, acc);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) partial[(int64_t)b * kMaxPartials + blockIdx.x] = s;
}

cudaError_t launch_gap(const Grid& g, const double* r64, const float* r32, int nb, double* partial, int* nparts,
                       cudaStream_t st) {
  const int bl = vec_blocks(g.d * g.N / 2);
  JFFT_K("gap", st, k_gap<<<dim3(bl, nb), 256, 0, st>>>(r64, r32, g.d * g.N, partial));
  *nparts = bl;
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

// The same reduction for callers that must not read the thread's pending-error
// slot: the status returned is the launch's own.
cudaError_t launch_reduce_partials_own_status(const double* partial, int nparts, int rows, int64_t pstride,
                                              double* out, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(rows);
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  cudaError_t e = cudaSuccess;
  JFFT_K("reduce_rows", st, e = cudaLaunchKernelEx(&cfg, k_reduce_rows, partial, nparts, pstride, out));
  return e;
}

// partial[row][blk] = sum of row `row` of x viewed as [rows][n]
__global__ void __launch_bounds__(256) k_row_sums(const double* __restrict__ x, int64_t n, double* __restrict__ partial) {
  const int row = blockIdx.y;
  const double* xr = x + (int64_t)row * n;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) acc += xr[i];
  const double s = block_sum(acc);
  if (threadIdx.x == 0) partial[(int64_t)row * kMaxPartials + blockIdx.x] = s;
}

cudaError_t launch_row_sums(const double* x, int rows, int64_t n, double* partial, int* nparts, cudaStream_t st) {
  const int bl = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 2));
  JFFT_K("row_sums", st, k_row_sums<<<dim3(bl, rows), 256, 0, st>>>(x, n, partial));
  *nparts = bl;
  return cudaGetLastError();
}

__global__ void k_sub_mean(double* __restrict__ x, int64_t n, const double* __restrict__ sums) {
  const int row = blockIdx.y;
  const double m = sums[row] / (double)n;
  double* xr = x + (int64_t)row * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) xr[i] -= m;
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

// dst[b][i] = active[b] ? (float) src[b][i] : 0
__global__ void k_to_f32(const double* __restrict__ src, float* __restrict__ dst, int64_t n, const int* __restrict__ active) {
  const int b = blockIdx.y;
  const bool on = active == nullptr || active[b] != 0;
  const int64_t off = (int64_t)b * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[off + i] = on ? (float)src[off + i] : 0.f;
}

cudaError_t launch_to_f32(const double* src, float* dst, int64_t n_per_rhs, int nb, const int* active, cudaStream_t st) {
  const int bl = (int)std::max<int64_t>(1, std::min<int64_t>((n_per_rhs + 255) / 256, 152 * 8));
  JFFT_K("to_f32", st, k_to_f32<<<dim3(bl, nb), 256, 0, st>>>(src, dst, n_per_rhs, active));
  return cudaGetLastError();
}

// u += (double) d
__global__ void k_add_f32(double* __restrict__ u, const float* __restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    u[i] += (double)d[i];
}

cudaError_t launch_add_f32(double* u, const float* d, int64_t n, cudaStream_t st) {
  const int bl = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8));
  JFFT_K("add_f32", st, k_add_f32<<<bl, 256, 0, st>>>(u, d, n));
  return cudaGetLastError();
}

// r = f - q ; partial[b][blk] = sum r.r
__global__ void __launch_bounds__(256) k_sub_norm(const double* __restrict__ f, const double* __restrict__ q,
                                                  double* __restrict__ r, int64_t n, double* __restrict__ partial) {
  const int b = blockIdx.y;
  const int64_t off = (int64_t)b * n;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = f[off + i] - q[off + i];
    r[off + i] = v;
    acc = fma(v, v, acc);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) partial[(int64_t)b * kMaxPartials + blockIdx.x] = s;
}

cudaError_t launch_sub_norm(const Grid& g, const double* f, const double* q, double* r, int nb, double* partial,
                            int* nparts, cudaStream_t st) {
  const int bl = vec_blocks(g.d * g.N / 2);
  JFFT_K("sub_norm", st, k_sub_norm<<<dim3(bl, nb), 256, 0, st>>>(f, q, r, g.d * g.N, partial));
  *nparts = bl;
  return cudaGetLastError();
}

}  // namespace jfft
