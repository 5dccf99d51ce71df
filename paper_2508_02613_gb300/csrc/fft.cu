// Green preconditioner M^-1 = F^-1 G_hat F and its Jacobi-wrapped form
// J^1/2 F^-1 G_hat F J^1/2 (paper Eq. prec_lin_systemG_FFT, Eq. prec_lin_systemJG_2),
// with a hand-written FFT (S6), plus the forward transform used by Alg. 1 (S9).
//
// Transform layout. The real axis (last, contiguous) is transformed first with
// the half-length trick (n real = n/2 complex + a twiddle post-pass) and written
// transposed so that the next axis becomes contiguous; the axis-0 pass reads
// contiguous lines, applies the d x d block of G_hat per frequency between the
// forward and the inverse transform, and writes back in place; the inverse passes
// mirror the forward ones. Every line FFT runs in shared memory as radix-4
// Stockham stages (one radix-2 stage first when log2 L is odd), twiddles from a
// per-axis table exp(-2 pi i m / n_a).
//
// Scaling: the real-axis forward post-pass omits its factor 1/2 and every inverse
// pass is unnormalised, so the chain computes 2 N x the true F^-1 G F; the stored
// symbol table carries the factor 1 / (2 N).
//
// Every kernel is templated on the working precision T (double, or float for the
// mixed-precision inner solve); inner-product partials are summed per thread in T
// and across the block in double.
#include "jfft_internal.cuh"
#include "reduce.cuh"

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

template <typename T> __device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T, bool INV> __device__ __forceinline__ cplx<T> twmul(cplx<T> v, cplx<T> w) {
  if (INV) w.y = -w.y;
  return mk<T>(v.x * w.x - v.y * w.y, v.x * w.y + v.y * w.x);
}

// Stockham FFT of nl lines of length L (power of two) held in a (line stride ls);
// b is scratch of the same shape. Returns the buffer holding the result. All
// threads of the block must call it.
template <typename T, bool INV>
__device__ cplx<T>* fft_smem(cplx<T>* a, cplx<T>* b, int nl, int L, int logL, int ls, const cplx<T>* __restrict__ tw,
                             int tws) {
  using C = cplx<T>;
  C* src = a;
  C* dst = b;
  int Ns = 1;
  if (logL & 1) {
    const int h = L >> 1;
    for (int t = threadIdx.x; t < nl * h; t += blockDim.x) {
      const int line = t / h, j = t - line * h;
      const C* s = src + line * ls;
      C* d = dst + line * ls;
      const C v0 = s[j], v1 = s[j + h];
      d[2 * j] = cadd<T>(v0, v1);
      d[2 * j + 1] = csub<T>(v0, v1);
    }
    __syncthreads();
    C* t = src; src = dst; dst = t;
    Ns = 2;
  }
  const int q = L >> 2;
  while (Ns < L) {
    const int step = (L / (4 * Ns)) * tws;
    for (int t = threadIdx.x; t < nl * q; t += blockDim.x) {
      const int line = t / q, j = t - line * q;
      const C* s = src + line * ls;
      C* d = dst + line * ls;
      const int k = j & (Ns - 1);
      C v0 = s[j], v1 = s[j + q], v2 = s[j + 2 * q], v3 = s[j + 3 * q];
      if (Ns > 1) {
        const int m1 = k * step;
        v1 = twmul<T, INV>(v1, tw[m1]);
        v2 = twmul<T, INV>(v2, tw[2 * m1]);
        v3 = twmul<T, INV>(v3, tw[3 * m1]);
      }
      const C s02 = cadd<T>(v0, v2), d02 = csub<T>(v0, v2), s13 = cadd<T>(v1, v3), d13 = csub<T>(v1, v3);
      C y1, y3;
      if (!INV) {
        y1 = mk<T>(d02.x + d13.y, d02.y - d13.x);
        y3 = mk<T>(d02.x - d13.y, d02.y + d13.x);
      } else {
        y1 = mk<T>(d02.x - d13.y, d02.y + d13.x);
        y3 = mk<T>(d02.x + d13.y, d02.y - d13.x);
      }
      const int base = (j - k) * 4 + k;
      d[base] = cadd<T>(s02, s13);
      d[base + Ns] = y1;
      d[base + 2 * Ns] = csub<T>(s02, s13);
      d[base + 3 * Ns] = y3;
    }
    __syncthreads();
    C* t = src; src = dst; dst = t;
    Ns *= 4;
  }
  return src;
}

template <typename T> struct JScaleT {
  T k[3];     // kappa_a^-1/2 per component
  T void_js;  // J^1/2 at void nodes
};

template <typename T> __device__ __forceinline__ T kscale(const JScaleT<T>& jsc, int a) {
  return a == 0 ? jsc.k[0] : (a == 1 ? jsc.k[1] : jsc.k[2]);
}
template <typename T> __device__ __forceinline__ T jhalf(const T* __restrict__ js, T ka, T void_js, int64_t node) {
  const T s = js[node];
  return s > T(0) ? s * ka : void_js;
}

// Pass A: forward FFT along contiguous rows, written transposed.
// in: [S][R][Lin] (real or complex); out: [S][Lout][R].
template <typename T, bool REAL, bool JAC>
__global__ void __launch_bounds__(256) k_rows_fwd(int D, const T* __restrict__ rin, const cplx<T>* __restrict__ cin,
                                                  cplx<T>* __restrict__ out, int R, int Lin, int logL, int w,
                                                  const cplx<T>* __restrict__ tw, const T* __restrict__ js,
                                                  JScaleT<T> jsc, const CgState* __restrict__ cg, int slabs_per_b) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* sm2 = reinterpret_cast<C*>(sm_raw);
  const int S = blockIdx.y;
  if (cg && cg[S / slabs_per_b].done) return;
  const int r0 = blockIdx.x * w;
  const int L = REAL ? Lin / 2 : Lin;
  const int Lout = REAL ? L + 1 : L;
  const int ls = L + 1;
  C* A = sm2;
  C* B = sm2 + w * ls;
  T ka = T(0);
  if (JAC) ka = kscale<T>(jsc, S % D);
  for (int t = threadIdx.x; t < w * L; t += blockDim.x) {
    const int line = t / L, m = t - line * L;
    const int64_t row = r0 + line;
    C v;
    if (REAL) {
      v = reinterpret_cast<const C*>(rin + ((int64_t)S * R + row) * Lin)[m];
      if (JAC) {
        const int64_t node = row * Lin + 2 * m;
        v.x *= jhalf<T>(js, ka, jsc.void_js, node);
        v.y *= jhalf<T>(js, ka, jsc.void_js, node + 1);
      }
    } else {
      v = cin[((int64_t)S * R + row) * Lin + m];
    }
    A[line * ls + m] = v;
  }
  __syncthreads();
  C* res = fft_smem<T, false>(A, B, w, L, logL, ls, tw, REAL ? 2 : 1);
  if (REAL) {
    // X[k] = (Z[k] + conj Z[M-k]) - i W^k (Z[k] - conj Z[M-k]), k = 0..M (times 2)
    const int half = L / 2 + 1;
    for (int t = threadIdx.x; t < w * half; t += blockDim.x) {
      const int line = t / half, k = t - line * half;
      C* z = res + line * ls;
      const C zk = z[k], zm = z[(L - k) & (L - 1)];
      const C A_ = mk<T>(zk.x + zm.x, zk.y - zm.y);
      const C B_ = mk<T>(zk.x - zm.x, zk.y + zm.y);
      const C Cw = twmul<T, false>(B_, tw[k]);
      z[k] = mk<T>(A_.x + Cw.y, A_.y - Cw.x);
      z[L - k] = mk<T>(A_.x - Cw.y, -A_.y - Cw.x);
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < w * Lout; t += blockDim.x) {
    const int k = t / w, line = t - k * w;
    out[((int64_t)S * Lout + k) * R + r0 + line] = res[line * ls + k];
  }
}

// Pass C: contiguous lines of axis 0 for all d components of one frequency line:
// forward FFT, block multiply by the stored symbol, inverse FFT (or forward only).
template <typename T, int D, bool GREEN>
__global__ void __launch_bounds__(256) k_lines(cplx<T>* __restrict__ spec, int nlines, int L, int logL,
                                               const cplx<T>* __restrict__ tw, const T* __restrict__ G,
                                               const CgState* __restrict__ cg) {
  using C = cplx<T>;
  constexpr int NCMP = D * (D + 1) / 2;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* sm2 = reinterpret_cast<C*>(sm_raw);
  const int l = blockIdx.x, b = blockIdx.y;
  if (cg && cg[b].done) return;
  const int ls = L + 1;
  C* A = sm2;
  C* B = sm2 + D * ls;
  for (int t = threadIdx.x; t < D * L; t += blockDim.x) {
    const int a = t / L, k = t - a * L;
    A[a * ls + k] = spec[(((int64_t)b * D + a) * nlines + l) * L + k];
  }
  __syncthreads();
  C* res = fft_smem<T, false>(A, B, D, L, logL, ls, tw, 1);
  if (GREEN) {
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
      const T* gk = G + ((int64_t)l * L + k) * NCMP;
      T gm[NCMP];
#pragma unroll
      for (int c = 0; c < NCMP; ++c) gm[c] = gk[c];
      C v[D];
#pragma unroll
      for (int a = 0; a < D; ++a) v[a] = res[a * ls + k];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        C o = mk<T>(T(0), T(0));
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const int lo = a < c ? a : c, hi = a < c ? c : a;
          const int idx = (D == 2) ? (lo == 0 ? hi : 2) : (lo == 0 ? hi : (lo == 1 ? 2 + hi : 5));
          o.x += gm[idx] * v[c].x;
          o.y += gm[idx] * v[c].y;
        }
        res[a * ls + k] = o;
      }
    }
    __syncthreads();
    C* other = (res == A) ? B : A;
    res = fft_smem<T, true>(res, other, D, L, logL, ls, tw, 1);
  }
  for (int t = threadIdx.x; t < D * L; t += blockDim.x) {
    const int a = t / L, k = t - a * L;
    spec[(((int64_t)b * D + a) * nlines + l) * L + k] = res[a * ls + k];
  }
}

// Pass B: inverse FFT along rows whose frequencies are stored transposed.
// in: [S][Lin][R]; out: [S][R][Lout] (real: Lout = 2 (Lin - 1), with J^1/2 and the
// r . z partial; complex: Lout = Lin).
template <typename T, bool REAL, bool JAC>
__global__ void __launch_bounds__(256) k_cols_inv(int D, const cplx<T>* __restrict__ in, T* __restrict__ rout,
                                                  cplx<T>* __restrict__ cout, int R, int Lin, int logL, int w,
                                                  const cplx<T>* __restrict__ tw, const T* __restrict__ js,
                                                  JScaleT<T> jsc, const T* __restrict__ rdot,
                                                  double* __restrict__ partial, const CgState* __restrict__ cg,
                                                  int slabs_per_b) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* sm2 = reinterpret_cast<C*>(sm_raw);
  const int S = blockIdx.y;
  const int b = S / slabs_per_b;
  if (cg && cg[b].done) return;
  const int r0 = blockIdx.x * w;
  const int L = REAL ? Lin - 1 : Lin;
  const int ls = L + 1;
  C* A = sm2;
  C* B = sm2 + w * ls;
  for (int t = threadIdx.x; t < w * Lin; t += blockDim.x) {
    const int k = t / w, line = t - k * w;
    A[line * ls + k] = in[((int64_t)S * Lin + k) * R + r0 + line];
  }
  __syncthreads();
  if (REAL) {
    // Z[k] = E + i O, E = X[k] + conj X[M-k], O = (X[k] - conj X[M-k]) W^-k (times 2)
    const int half = L / 2 + 1;
    for (int t = threadIdx.x; t < w * half; t += blockDim.x) {
      const int line = t / half, k = t - line * half;
      C* x = A + line * ls;
      C xk = x[k], xm = x[L - k];
      if (k == 0) { xk.y = T(0); xm.y = T(0); }
      const C E = mk<T>(xk.x + xm.x, xk.y - xm.y);
      const C Bv = mk<T>(xk.x - xm.x, xk.y + xm.y);
      const C O = twmul<T, true>(Bv, tw[k]);
      x[k] = mk<T>(E.x - O.y, E.y + O.x);
      if (k != 0) x[L - k] = mk<T>(E.x + O.y, -E.y + O.x);
    }
    __syncthreads();
  }
  C* res = fft_smem<T, true>(A, B, w, L, logL, ls, tw, REAL ? 2 : 1);
  if (REAL) {
    T dot = T(0);
    const int n = 2 * L;
    const int a = S % D;
    T ka = T(0);
    if (JAC) ka = kscale<T>(jsc, a);
    for (int t = threadIdx.x; t < w * L; t += blockDim.x) {
      const int line = t / L, m = t - line * L;
      const int64_t row = r0 + line;
      C v = res[line * ls + m];
      const int64_t node = row * n + 2 * m;
      if (JAC) {
        v.x *= jhalf<T>(js, ka, jsc.void_js, node);
        v.y *= jhalf<T>(js, ka, jsc.void_js, node + 1);
      }
      const int64_t off = ((int64_t)S * R + row) * n + 2 * m;
      reinterpret_cast<C*>(rout + off)[0] = v;
      const C rv = reinterpret_cast<const C*>(rdot + off)[0];
      dot += rv.x * v.x + rv.y * v.y;
    }
    const double s = block_sum((double)dot);
    if (threadIdx.x == 0) partial[(int64_t)b * kMaxPartials + (int64_t)a * gridDim.x + blockIdx.x] = s;
  } else {
    for (int t = threadIdx.x; t < w * L; t += blockDim.x) {
      const int line = t / L, m = t - line * L;
      cout[((int64_t)S * R + r0 + line) * L + m] = res[line * ls + m];
    }
  }
}

static int ilog2(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }

template <typename T> static int rows_per_cta(int L, int R) {
  int w = 16;
  while (w > 1 && (size_t)2 * w * (L + 1) * sizeof(cplx<T>) > 98304) w >>= 1;
  while (w > R) w >>= 1;
  return w;
}

template <typename K> static cudaError_t set_smem(K kern, size_t bytes) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define JFFT_TRY(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return e_; } while (0)

template <typename T> static const char* nm(const char* d64, const char* d32) { return sizeof(T) == 8 ? d64 : d32; }

// Real rows (last axis) forward, S = nb * d slabs.
template <typename T>
static cudaError_t pass_rows_real_fwd(const Grid& g, const FftPlanT<T>& p, const T* r, int nb, bool jac, const T* js,
                                      const JScaleT<T>& jsc, const CgState* cg, cudaStream_t st) {
  const int Lin = g.n[g.d - 1];
  const int R = (int)(g.N / Lin);
  const int L = Lin / 2;
  const int w = rows_per_cta<T>(L, R);
  const size_t smem = (size_t)2 * w * (L + 1) * sizeof(cplx<T>);
  dim3 grid(R / w, nb * g.d);
  auto k = jac ? k_rows_fwd<T, true, true> : k_rows_fwd<T, true, false>;
  JFFT_TRY(set_smem(k, smem));
  JFFT_K(nm<T>("fft_rows_real_fwd", "fft_rows_real_fwd_f32"), st,
         k<<<grid, 256, smem, st>>>(g.d, r, nullptr, p.T, R, Lin, ilog2(L), w, p.tw[g.d - 1], js, jsc, cg, g.d));
  return cudaGetLastError();
}

// 3D: complex rows along axis 1 of T[S'][n0][n1] -> U[S'][n1][n0].
template <typename T>
static cudaError_t pass_rows_cplx_fwd(const Grid& g, const FftPlanT<T>& p, int nb, const CgState* cg, cudaStream_t st) {
  const int R = g.n[0], Lin = g.n[1];
  const int w = rows_per_cta<T>(Lin, R);
  const size_t smem = (size_t)2 * w * (Lin + 1) * sizeof(cplx<T>);
  const int slabs = nb * g.d * (g.M + 1);
  dim3 grid(R / w, slabs);
  auto k = k_rows_fwd<T, false, false>;
  JFFT_TRY(set_smem(k, smem));
  JScaleT<T> jsc = {};
  JFFT_K(nm<T>("fft_rows_cplx_fwd", "fft_rows_cplx_fwd_f32"), st,
         k<<<grid, 256, smem, st>>>(g.d, nullptr, p.T, p.U, R, Lin, ilog2(Lin), w, p.tw[1], nullptr, jsc, cg,
                                    g.d * (g.M + 1)));
  return cudaGetLastError();
}

template <typename T>
static cudaError_t pass_lines(const Grid& g, const FftPlanT<T>& p, int nb, bool green, const CgState* cg,
                              cudaStream_t st) {
  const int L = g.n[0];
  const int nlines = (int)(g.F / L);
  cplx<T>* spec = (g.d == 2) ? p.T : p.U;
  const size_t smem = (size_t)2 * g.d * (L + 1) * sizeof(cplx<T>);
  dim3 grid(nlines, nb);
  const char* name = green ? nm<T>("fft_lines", "fft_lines_f32") : nm<T>("fft_lines_fwd", "fft_lines_fwd_f32");
  if (g.d == 2) {
    auto k = green ? k_lines<T, 2, true> : k_lines<T, 2, false>;
    JFFT_TRY(set_smem(k, smem));
    JFFT_K(name, st, k<<<grid, 256, smem, st>>>(spec, nlines, L, ilog2(L), p.tw[0], p.G, cg));
  } else {
    auto k = green ? k_lines<T, 3, true> : k_lines<T, 3, false>;
    JFFT_TRY(set_smem(k, smem));
    JFFT_K(name, st, k<<<grid, 256, smem, st>>>(spec, nlines, L, ilog2(L), p.tw[0], p.G, cg));
  }
  return cudaGetLastError();
}

// 3D: complex inverse along axis 1, U[S'][n1][n0] -> T[S'][n0][n1].
template <typename T>
static cudaError_t pass_cols_cplx_inv(const Grid& g, const FftPlanT<T>& p, int nb, const CgState* cg, cudaStream_t st) {
  const int R = g.n[0], Lin = g.n[1];
  const int w = rows_per_cta<T>(Lin, R);
  const size_t smem = (size_t)2 * w * (Lin + 1) * sizeof(cplx<T>);
  const int slabs = nb * g.d * (g.M + 1);
  dim3 grid(R / w, slabs);
  auto k = k_cols_inv<T, false, false>;
  JFFT_TRY(set_smem(k, smem));
  JScaleT<T> jsc = {};
  JFFT_K(nm<T>("fft_cols_cplx_inv", "fft_cols_cplx_inv_f32"), st,
         k<<<grid, 256, smem, st>>>(g.d, p.U, nullptr, p.T, R, Lin, ilog2(Lin), w, p.tw[1], nullptr, jsc, nullptr,
                                    nullptr, cg, g.d * (g.M + 1)));
  return cudaGetLastError();
}

template <typename T>
static cudaError_t pass_cols_real_inv(const Grid& g, const FftPlanT<T>& p, T* z, int nb, bool jac, const T* js,
                                      const JScaleT<T>& jsc, const T* r, double* partial, int* nparts,
                                      const CgState* cg, cudaStream_t st) {
  const int n = g.n[g.d - 1];
  const int R = (int)(g.N / n);
  const int L = n / 2;
  const int w = rows_per_cta<T>(L, R);
  const size_t smem = (size_t)2 * w * (L + 1) * sizeof(cplx<T>);
  dim3 grid(R / w, nb * g.d);
  auto k = jac ? k_cols_inv<T, true, true> : k_cols_inv<T, true, false>;
  JFFT_TRY(set_smem(k, smem));
  JFFT_K(nm<T>("fft_cols_real_inv", "fft_cols_real_inv_f32"), st,
         k<<<grid, 256, smem, st>>>(g.d, p.T, z, nullptr, R, L + 1, ilog2(L), w, p.tw[g.d - 1], js, jsc, r, partial,
                                    cg, g.d));
  if (nparts) *nparts = grid.x * g.d;
  return cudaGetLastError();
}

template <typename T>
static cudaError_t green_precond_t(const Grid& g, const FftPlanT<T>& p, const T* r, T* z, int nb, const T* js,
                                   const double* jscale, double void_js, bool jacobi, double* partial, int* nparts,
                                   const CgState* done, cudaStream_t st) {
  JScaleT<T> jsc;
  for (int a = 0; a < 3; ++a) jsc.k[a] = (T)jscale[a];
  jsc.void_js = (T)void_js;
  JFFT_TRY(pass_rows_real_fwd<T>(g, p, r, nb, jacobi, js, jsc, done, st));
  if (g.d == 3) JFFT_TRY(pass_rows_cplx_fwd<T>(g, p, nb, done, st));
  JFFT_TRY(pass_lines<T>(g, p, nb, true, done, st));
  if (g.d == 3) JFFT_TRY(pass_cols_cplx_inv<T>(g, p, nb, done, st));
  return pass_cols_real_inv<T>(g, p, z, nb, jacobi, js, jsc, r, partial, nparts, done, st);
}

cudaError_t launch_green_precond(const Grid& g, const FftPlan& p, const double* r, double* z, int nb,
                                 int64_t /*field_stride*/, const double* js, const double* jscale, double void_js,
                                 bool jacobi, double* partial, int* nparts, const CgState* done, cudaStream_t st) {
  return green_precond_t<double>(g, p, r, z, nb, js, jscale, void_js, jacobi, partial, nparts, done, st);
}

cudaError_t launch_green_precond_f32(const Grid& g, const FftPlanT<float>& p, const float* r, float* z, int nb,
                                     const float* js, const double* jscale, double void_js, bool jacobi,
                                     double* partial, int* nparts, const CgState* done, cudaStream_t st) {
  return green_precond_t<float>(g, p, r, z, nb, js, jscale, void_js, jacobi, partial, nparts, done, st);
}

cudaError_t launch_forward_spectrum(const Grid& g, const FftPlan& p, const double* r, int nb,
                                    const double2** spec_out, cudaStream_t st) {
  JScaleT<double> jsc = {};
  JFFT_TRY(pass_rows_real_fwd<double>(g, p, r, nb, false, nullptr, jsc, nullptr, st));
  if (g.d == 3) JFFT_TRY(pass_rows_cplx_fwd<double>(g, p, nb, nullptr, st));
  JFFT_TRY(pass_lines<double>(g, p, nb, false, nullptr, st));
  *spec_out = (g.d == 2) ? p.T : p.U;
  return cudaSuccess;
}

}  // namespace jfft
