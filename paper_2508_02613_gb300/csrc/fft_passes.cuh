// Green preconditioner M^-1 = F^-1 G_hat F and its Jacobi-wrapped form
// J^1/2 F^-1 G_hat F J^1/2 (paper Eq. prec_lin_systemG_FFT, Eq. prec_lin_systemJG_2),
// with a hand-written FFT (S6), plus the forward transform used by Alg. 1 (S9).
//
// Transform layout. The real axis (last, contiguous) is transformed first with
// the half-length trick (n real = n/2 complex + a twiddle post-pass) and written
// transposed so that the next axis becomes contiguous; the axis-0 pass reads
// contiguous lines, applies the d x d block of G_hat per frequency between the
// forward and the inverse transform, and writes back in place; the inverse passes
// mirror the forward ones. Every line FFT runs on the register-resident Stockham
// engine of fft_engine.cuh (radix 8, then one smaller radix), twiddles from a per-axis
// table exp(-2 pi i m / n_a); line lengths 64 .. 2048 use the engine's compile-time
// form with per-stage twiddle tables, other lengths the runtime form.
//
// Scaling: the real-axis forward post-pass omits its factor 1/2 and every inverse
// pass is unnormalised, so the chain computes 2 N x the true F^-1 G F; the stored
// symbol table carries the factor 1 / (2 N).
//
// Every kernel is templated on the working precision T (double, or float for the
// mixed-precision inner solve); inner-product partials are summed per thread in T
// and across the block in double. The kernels and pass launchers live here; fft.cu
// instantiates them in FP64 and fft_f32.cu in FP32 (two translation units that build
// in parallel).
#pragma once

#include "fft_engine.cuh"
#include "reduce.cuh"

namespace jfft {

// 1 at run time for the engine's FP64 sums (see add1): the first entry of an axis twiddle
// table is exp(0) = (1, 0) exactly; FP32 sums need no such value.
template <typename T> __device__ __forceinline__ T runtime_one(const cplx<T>* __restrict__ tw) {
  if constexpr (sizeof(T) == 8) return tw[0].x;
  else return T(1);
}
template <typename T, bool INV> __device__ __forceinline__ cplx<T> twmul(cplx<T> v, cplx<T> w) {
  if (INV) w.y = -w.y;
  return mk<T>(v.x * w.x - v.y * w.y, v.x * w.y + v.y * w.x);
}

// Largest radix of the engine per precision, and the launch shape of the passes:
// threads per row / column block and the minimum resident blocks per SM they are
// compiled for (register budget). FP32 runs radix 8 at 64 registers (four
// 256-thread blocks per SM); radix 16 needs ~128 registers, halves the resident
// warps and measured slower on GB300.
template <typename T> struct FftOcc {
  static constexpr int radix = sizeof(T) == 4 ? 8 : 8;
  static constexpr int rows_threads = 256;
  static constexpr int rows = sizeof(T) == 4 ? 4 : 2;
  static constexpr int lines = sizeof(T) == 4 ? 2 : 1;
};
template <typename T> constexpr int radix_max() { return FftOcc<T>::radix; }

// Threads per line for the engine.
template <typename T> __host__ __device__ inline int lanes_per_line(int L) {
  return L >= radix_max<T>() ? L / radix_max<T>() : 1;
}

// The resolved J^1/2 table: the factor of DOF (a, node) is js[a cs + node] (cs = 0: one
// factor per node shared by the components, N: one per DOF); void nodes and the
// per-component unit diagonals are folded in when the table is built.
template <typename T> struct JScaleT {
  int64_t cs;
};
// Factors of samples 2m and 2m + 1 of a row: one 16-byte load in FP64, two 4-byte
// loads in FP32 (1.5 % faster than one 8-byte load in the FP32 row pass on GB300).
template <typename T> __device__ __forceinline__ cplx<T> jpair(const T* __restrict__ row, int m) {
  if (sizeof(T) == 8) return reinterpret_cast<const cplx<T>*>(row)[m];
  return mk<T>(row[2 * m], row[2 * m + 1]);
}

// PCG update fused into the forward real row pass of the preconditioner: before the
// transform, x += alpha p and r -= alpha q on the row's samples (the roundings of
// k_cg_xr), and the partial sums of ||r||^2 for the residual stage, whose tail the
// pass runs. Unused (XR = false) in every other pass.
template <typename T> struct XrUpdate {
  T* x;
  T* r;
  const T* p;
  const T* q;
  double* partial;
  CgState* cg;
  StageCtl sc;
};

// Pass A: forward FFT along contiguous rows, written transposed.
// in: [S][R][Lin] (real or complex); out: [S][Lout][R]. w rows per group, TPL lanes
// per row (block = w * TPL threads); a block takes the groups blockIdx.x, blockIdx.x +
// gridDim.x, ... (a capped grid keeps the partial-sum slots within kMaxPartials).
template <typename T, bool REAL, bool JAC, bool XR, int LC>
__global__ void __launch_bounds__(FftOcc<T>::rows_threads, FftOcc<T>::rows) k_rows_fwd(int D, const T* __restrict__ rin, const cplx<T>* __restrict__ cin,
                                                  cplx<T>* __restrict__ out, int R, int Lin, int lgTPL, int lgw,
                                                  const cplx<T>* __restrict__ tw, const cplx<T>* __restrict__ lft,
                                                  const T* __restrict__ js, JScaleT<T> jsc,
                                                  const CgState* __restrict__ cg, int slabs_per_b, XrUpdate<T> xr) {
  using C = cplx<T>;
  constexpr int RM = radix_max<T>();
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* sm2 = reinterpret_cast<C*>(sm_raw);
  const int S = blockIdx.y;
  if (cg && cg[S / slabs_per_b].done) return;
  const int w = 1 << lgw;
  if (LC) Lin = REAL ? 2 * LC : LC;
  const int L = LC ? LC : (REAL ? Lin / 2 : Lin);
  const int Lout = REAL ? L + 1 : L;
  const int ls = line_stride<T>(L, w);
  const int TPL = LC ? LC / RM : 1 << lgTPL;
  const int RME = L < RM ? L : RM;
  const int line = LC ? (int)threadIdx.x / TPL : (int)threadIdx.x >> lgTPL, j = threadIdx.x & (TPL - 1);
  // twiddle table of the axis (Lin entries) in shared memory; the engine's first
  // barrier orders these stores before any use
  // runtime length: the axis table; compile-time length: the post-pass twiddles
  // (k <= L/2) followed by the engine's per-stage tables
  C* twl = sm2;
  C* tst = twl;
  if constexpr (LC > 0) {
    const int npost = REAL ? L / 2 + 1 : 0;
    for (int i = threadIdx.x; i < npost; i += blockDim.x) twl[i] = tw[i];
    tst = twl + npost;
    stage_twiddles<T, RM, LC, REAL ? 2 : 1>(tst, tw, lft);
  } else {
    for (int i = threadIdx.x; i < Lin; i += blockDim.x) twl[i] = tw[i];
  }
  C* A = sm2 + Lin;
  C* B = A + w * ls;
  const T one = runtime_one<T>(tw);
  const T al = XR ? (T)xr.cg[S / slabs_per_b].alpha : T(0);
  T acc = T(0);  // XR: this thread's share of ||r||^2
  const int ngroups = R >> lgw;
#pragma unroll 1
  for (int grp = blockIdx.x;; grp += gridDim.x) {
    const int r0 = grp * w;
    const int64_t row = r0 + line;
    C v[RM];
    if constexpr (XR) {
      // all loads of the row's samples first, then the stores: no store can hold back a
      // later load (x, r, p, q may alias as far as the compiler knows)
      C rv[RM], qv[RM];
#pragma unroll
      for (int r = 0; r < RM; ++r)
        if (r < RME) {
          const int64_t off = ((int64_t)S * R + row) * Lin + 2 * (j + TPL * r);
          rv[r] = *reinterpret_cast<const C*>(xr.r + off);
          qv[r] = *reinterpret_cast<const C*>(xr.q + off);
        }
#pragma unroll
      for (int r = 0; r < RM; ++r)
        if (r < RME) {
          const int64_t off = ((int64_t)S * R + row) * Lin + 2 * (j + TPL * r);
          rv[r].x = fma(-al, qv[r].x, rv[r].x);
          rv[r].y = fma(-al, qv[r].y, rv[r].y);
          *reinterpret_cast<C*>(xr.r + off) = rv[r];
          acc = fma(rv[r].x, rv[r].x, acc);
          acc = fma(rv[r].y, rv[r].y, acc);
          v[r] = rv[r];
        }
    }
#pragma unroll
    for (int r = 0; r < RM; ++r) {
      if (r < RME) {
        const int m = j + TPL * r;
        C x;
        if (REAL) {
          if (XR) x = v[r];
          else x = reinterpret_cast<const C*>(rin + ((int64_t)S * R + row) * Lin)[m];
          if (JAC) {
            const cplx<T> j2 = jpair<T>(js + jsc.cs * (S % D) + row * Lin, m);
            x.x *= j2.x;
            x.y *= j2.y;
          }
        } else {
          x = cin[((int64_t)S * R + row) * Lin + m];
        }
        v[r] = x;
      }
    }
    C* res;
    if constexpr (LC > 0) res = line_fft_ct<T, RM, false, LC>(v, j, A + line * ls, B + line * ls, tst, one);
    else res = line_fft<T, RM, false>(v, j, L, A + line * ls, B + line * ls, twl, REAL ? 2 : 1, one);
    res -= line * ls;  // back to the block's buffer base
    if (REAL) {
      // X[k] = (Z[k] + conj Z[M-k]) - i W^k (Z[k] - conj Z[M-k]), k = 0..M (times 2);
      // the lanes of each line take the pairs (k, M - k) of their own line.
      C* z = res + line * ls;
      for (int k = j; k <= L / 2; k += TPL) {
        const C zk = z[spad(k)], zm = z[spad((L - k) & (L - 1))];
        const C A_ = mk<T>(add1(zk.x, zm.x, one), sub1(zk.y, zm.y, one));
        const C B_ = mk<T>(sub1(zk.x, zm.x, one), add1(zk.y, zm.y, one));
        const C Cw = twmul<T, false>(B_, twl[k]);
        z[spad(k)] = mk<T>(add1(A_.x, Cw.y, one), sub1(A_.y, Cw.x, one));
        z[spad(L - k)] = mk<T>(sub1(A_.x, Cw.y, one), sub1(-A_.y, Cw.x, one));
      }
      __syncthreads();
    }
    for (int t = threadIdx.x; t < w * Lout; t += blockDim.x) {
      const int k = t >> lgw, ln = t & (w - 1);
      out[((int64_t)S * Lout + k) * R + r0 + ln] = res[ln * ls + spad(k)];
    }
    if constexpr (XR) {
      // x += alpha p, after the transform where few registers are live
      C xv[RM], pv[RM];
#pragma unroll
      for (int r = 0; r < RM; ++r)
        if (r < RME) {
          const int64_t off = ((int64_t)S * R + row) * Lin + 2 * (j + TPL * r);
          xv[r] = *reinterpret_cast<const C*>(xr.x + off);
          pv[r] = *reinterpret_cast<const C*>(xr.p + off);
        }
#pragma unroll
      for (int r = 0; r < RM; ++r)
        if (r < RME) {
          const int64_t off = ((int64_t)S * R + row) * Lin + 2 * (j + TPL * r);
          xv[r].x = fma(al, pv[r].x, xv[r].x);
          xv[r].y = fma(al, pv[r].y, xv[r].y);
          *reinterpret_cast<C*>(xr.x + off) = xv[r];
        }
    }
    // only a pass with partial sums runs on a capped grid; the next group's transform
    // overwrites the buffers read above
    if (!XR || grp + (int)gridDim.x >= ngroups) break;
    __syncthreads();
  }
  if constexpr (XR) {
    const int b = S / slabs_per_b, a = S % slabs_per_b;
    const double s = block_sum((double)acc);
    if (threadIdx.x == 0) xr.partial[(int64_t)b * kMaxPartials + (int64_t)a * gridDim.x + blockIdx.x] = s;
    fused_stage_tail(xr.sc, xr.cg, b, xr.partial + (int64_t)b * kMaxPartials, slabs_per_b * gridDim.x);
  }
}

// Pass C: contiguous lines of axis 0 for all d components of one frequency line:
// forward FFT, block multiply by the stored symbol, inverse FFT (or forward only).
// Block = D * TPL threads; lanes [a TPL, (a+1) TPL) transform component a.
template <typename T, int D, bool GREEN, int LC>
__global__ void __launch_bounds__(512, FftOcc<T>::lines) k_lines(cplx<T>* __restrict__ spec, int nlines, int L, int lgTPL,
                                               const cplx<T>* __restrict__ tw, const cplx<T>* __restrict__ lft,
                                               const T* __restrict__ G, const CgState* __restrict__ cg) {
  using C = cplx<T>;
  constexpr int RM = radix_max<T>();
  constexpr int NCMP = D * (D + 1) / 2;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* sm2 = reinterpret_cast<C*>(sm_raw);
  const int l = blockIdx.x, b = blockIdx.y;
  if (cg && cg[b].done) return;
  if (LC) L = LC;
  const int ls = line_slots(L);
  const int TPL = LC ? LC / RM : 1 << lgTPL;
  const int RME = L < RM ? L : RM;
  const int a = LC ? (int)threadIdx.x / TPL : (int)threadIdx.x >> lgTPL, j = threadIdx.x & (TPL - 1);
  // twiddles (the axis table, or the per-stage tables of a compile-time length), ordered
  // by the engine's first barrier
  C* twl = sm2;
  if constexpr (LC > 0) stage_twiddles<T, RM, LC, 1>(twl, tw, lft);
  else
    for (int i = threadIdx.x; i < L; i += blockDim.x) twl[i] = tw[i];
  C* A = sm2 + L;
  C* B = A + D * ls;
  const C* gline = spec + (((int64_t)b * D + a) * nlines + l) * L;
  C v[RM];
#pragma unroll
  for (int r = 0; r < RM; ++r)
    if (r < RME) v[r] = gline[j + TPL * r];
  C* res;
  const T one = runtime_one<T>(tw);
  if constexpr (LC > 0) res = line_fft_ct<T, RM, false, LC>(v, j, A + a * ls, B + a * ls, twl, one) - a * ls;
  else res = line_fft<T, RM, false>(v, j, L, A + a * ls, B + a * ls, twl, 1, one) - a * ls;
  if (GREEN) {
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
      const T* gk = G + ((int64_t)l * L + k) * NCMP;
      T gm[NCMP];
#pragma unroll
      for (int c = 0; c < NCMP; ++c) gm[c] = gk[c];
      C vv[D];
#pragma unroll
      for (int c = 0; c < D; ++c) vv[c] = res[c * ls + spad(k)];
#pragma unroll
      for (int c1 = 0; c1 < D; ++c1) {
        C o = mk<T>(T(0), T(0));
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const int lo = c1 < c ? c1 : c, hi = c1 < c ? c : c1;
          const int idx = (D == 2) ? (lo == 0 ? hi : 2) : (lo == 0 ? hi : (lo == 1 ? 2 + hi : 5));
          o.x += gm[idx] * vv[c].x;
          o.y += gm[idx] * vv[c].y;
        }
        res[c1 * ls + spad(k)] = o;
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RM; ++r)
      if (r < RME) v[r] = res[a * ls + spad(j + TPL * r)];
    C* other = (res == A) ? B : A;
    // stage 1 writes `other` first, so no lane overwrites values still being read from res
    if constexpr (LC > 0) res = line_fft_ct<T, RM, true, LC>(v, j, other + a * ls, res + a * ls, twl, one) - a * ls;
    else res = line_fft<T, RM, true>(v, j, L, other + a * ls, res + a * ls, twl, 1, one) - a * ls;
  }
  C* gout = spec + (((int64_t)b * D + a) * nlines + l) * L;
#pragma unroll
  for (int r = 0; r < RM; ++r)
    if (r < RME) {
      const int k = j + TPL * r;
      gout[k] = res[a * ls + spad(k)];
    }
}

// Pass B: inverse FFT along rows whose frequencies are stored transposed.
// in: [S][Lin][R]; out: [S][R][Lout] (real: Lout = 2 (Lin - 1), with J^1/2 and the
// r . z partial; complex: Lout = Lin). w rows per group, TPL lanes per row; one group
// per block, or (MULTI, real pass on a capped grid) groups taken grid-stride as in pass A.
// The single-group instances keep the loop out of the register allocation.
template <typename T, bool REAL, bool JAC, bool MULTI, int LC>
__global__ void __launch_bounds__(FftOcc<T>::rows_threads, FftOcc<T>::rows) k_cols_inv(int D, const cplx<T>* __restrict__ in, T* __restrict__ rout,
                                                  cplx<T>* __restrict__ cout, int R, int Lin, int lgTPL, int lgw,
                                                  const cplx<T>* __restrict__ tw, const cplx<T>* __restrict__ lft,
                                                  const T* __restrict__ js, JScaleT<T> jsc, const T* __restrict__ rdot,
                                                  double* __restrict__ partial, CgState* __restrict__ cg,
                                                  int slabs_per_b, StageCtl sc) {
  using C = cplx<T>;
  constexpr int RM = radix_max<T>();
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* sm2 = reinterpret_cast<C*>(sm_raw);
  const int S = blockIdx.y;
  const int b = S / slabs_per_b;
  if (cg && cg[b].done) return;
  const int w = 1 << lgw;
  if (LC) Lin = REAL ? LC + 1 : LC;
  const int L = LC ? LC : (REAL ? Lin - 1 : Lin);
  const int ls = line_stride<T>(L, w);
  const int TPL = LC ? LC / RM : 1 << lgTPL;
  const int RME = L < RM ? L : RM;
  const int line = LC ? (int)threadIdx.x / TPL : (int)threadIdx.x >> lgTPL, j = threadIdx.x & (TPL - 1);
  const int ntw = REAL ? 2 * L : L;  // twiddle table of the axis in shared memory
  // runtime length: the axis table; compile-time length: the pre-pass twiddles
  // (k <= L/2) followed by the engine's per-stage tables
  C* twl = sm2;
  C* tst = twl;
  if constexpr (LC > 0) {
    const int npost = REAL ? L / 2 + 1 : 0;
    for (int i = threadIdx.x; i < npost; i += blockDim.x) twl[i] = tw[i];
    tst = twl + npost;
    stage_twiddles<T, RM, LC, REAL ? 2 : 1>(tst, tw, lft);
  } else {
    for (int i = threadIdx.x; i < ntw; i += blockDim.x) twl[i] = tw[i];
  }
  C* A = sm2 + ntw;
  C* B = A + w * ls;
  const T one = runtime_one<T>(tw);
  T dot = T(0);  // REAL: this thread's share of r . z
  const int ngroups = R >> lgw;
#pragma unroll 1
  for (int grp = blockIdx.x;; grp += gridDim.x) {
    const int r0 = grp * w;
    if constexpr (LC > 0) {
      // all of a thread's transposed loads (ceil(Lin / TPL), whatever w) in flight at once
      constexpr int PER = (LC + 1 + LC / RM - 1) / (LC / RM);
      C buf[PER];
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int t = threadIdx.x + u * blockDim.x;
        if (t < w * Lin) buf[u] = in[((int64_t)S * Lin + (t >> lgw)) * R + r0 + (t & (w - 1))];
      }
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int t = threadIdx.x + u * blockDim.x;
        if (t < w * Lin) A[(t & (w - 1)) * ls + spad(t >> lgw)] = buf[u];
      }
    } else {
      for (int t = threadIdx.x; t < w * Lin; t += blockDim.x) {
        const int k = t >> lgw, ln = t & (w - 1);
        A[ln * ls + spad(k)] = in[((int64_t)S * Lin + k) * R + r0 + ln];
      }
    }
    __syncthreads();
    if (REAL) {
      // Z[k] = E + i O, E = X[k] + conj X[M-k], O = (X[k] - conj X[M-k]) W^-k (times 2);
      // the lanes of each line take the pairs of their own line.
      C* x = A + line * ls;
      for (int k = j; k <= L / 2; k += TPL) {
        C xk = x[spad(k)], xm = x[spad(L - k)];
        if (k == 0) { xk.y = T(0); xm.y = T(0); }
        const C E = mk<T>(add1(xk.x, xm.x, one), sub1(xk.y, xm.y, one));
        const C Bv = mk<T>(sub1(xk.x, xm.x, one), add1(xk.y, xm.y, one));
        const C O = twmul<T, true>(Bv, twl[k]);
        x[spad(k)] = mk<T>(sub1(E.x, O.y, one), add1(E.y, O.x, one));
        if (k != 0) x[spad(L - k)] = mk<T>(add1(E.x, O.y, one), add1(-E.y, O.x, one));
      }
      __syncthreads();
    }
    C v[RM];
#pragma unroll
    for (int r = 0; r < RM; ++r)
      if (r < RME) v[r] = A[line * ls + spad(j + TPL * r)];
    C* res;
    if constexpr (LC > 0) res = line_fft_ct<T, RM, true, LC>(v, j, B + line * ls, A + line * ls, tst, one) - line * ls;
    else res = line_fft<T, RM, true>(v, j, L, B + line * ls, A + line * ls, twl, REAL ? 2 : 1, one) - line * ls;
    if (REAL) {
      const int n = 2 * L;
      const int a = S % D;
      const int64_t row = r0 + line;
#pragma unroll
      for (int i = 0; i < RM; ++i) {
        if (i >= RME) break;
        const int m = j + TPL * i;
        C x = res[line * ls + spad(m)];
        if (JAC) {
          const cplx<T> j2 = jpair<T>(js + jsc.cs * a + row * n, m);
          x.x *= j2.x;
          x.y *= j2.y;
        }
        const int64_t off = ((int64_t)S * R + row) * n + 2 * m;
        reinterpret_cast<C*>(rout + off)[0] = x;
        const C rv = reinterpret_cast<const C*>(rdot + off)[0];
        dot += rv.x * x.x + rv.y * x.y;
      }
    } else {
#pragma unroll
      for (int i = 0; i < RM; ++i) {
        if (i >= RME) break;
        const int m = j + TPL * i;
        cout[((int64_t)S * R + r0 + line) * L + m] = res[line * ls + spad(m)];
      }
    }
    // the next group's loads overwrite the buffers read above
    if (!MULTI || grp + (int)gridDim.x >= ngroups) break;
    __syncthreads();
  }
  if (REAL) {
    const int a = S % D;
    const double s = block_sum((double)dot);
    if (threadIdx.x == 0) partial[(int64_t)b * kMaxPartials + (int64_t)a * gridDim.x + blockIdx.x] = s;
    fused_stage_tail(sc, cg, b, partial + (int64_t)b * kMaxPartials, slabs_per_b * gridDim.x);
  }
}

static inline int ilog2(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }

// Lines per block for the row / column passes: up to FftOcc<T>::rows_threads
// threads and ~96 KB of shared memory (two buffers of w lines plus the ntw-entry
// twiddle table), never more lines than there are rows.
template <typename T> static int rows_per_cta(int L, int R, int ntw) {
  const int tpl = lanes_per_line<T>(L);
  int w = std::max(1, FftOcc<T>::rows_threads / tpl);
  while (w > 1 && ((size_t)2 * w * line_stride<T>(L, w) + ntw) * sizeof(cplx<T>) > 98304) w >>= 1;
  while (w > R) w >>= 1;
  return w;
}
template <typename T> static size_t rows_smem(int L, int w, int ntw) {
  return ((size_t)2 * w * line_stride<T>(L, w) + ntw) * sizeof(cplx<T>);
}

template <typename K> static cudaError_t set_smem(K kern, size_t bytes) {
  cudaError_t e = allow_dynamic_smem(kern, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
}

#define JFFT_TRY(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return e_; } while (0)

template <typename T> static const char* nm(const char* d64, const char* d32) { return sizeof(T) == 8 ? d64 : d32; }

// Kernel instance for line length L: the engine's compile-time form for the lengths of
// the usual grids (64 .. 2048), the runtime form otherwise.
#define JFFT_LC_SWITCH(L, KERNEL, ...)                 \
  switch (L) {                                         \
    case 64: return KERNEL<__VA_ARGS__, 64>;           \
    case 128: return KERNEL<__VA_ARGS__, 128>;         \
    case 256: return KERNEL<__VA_ARGS__, 256>;         \
    case 512: return KERNEL<__VA_ARGS__, 512>;         \
    case 1024: return KERNEL<__VA_ARGS__, 1024>;       \
    case 2048: return KERNEL<__VA_ARGS__, 2048>;       \
    default: return KERNEL<__VA_ARGS__, 0>;            \
  }
template <typename T, bool REAL, bool JAC, bool XR> static auto rows_kernel(int L) { JFFT_LC_SWITCH(L, k_rows_fwd, T, REAL, JAC, XR) }
template <typename T, bool REAL, bool JAC, bool MULTI> static auto cols_kernel(int L) { JFFT_LC_SWITCH(L, k_cols_inv, T, REAL, JAC, MULTI) }
template <typename T, int D, bool GREEN> static auto lines_kernel(int L) { JFFT_LC_SWITCH(L, k_lines, T, D, GREEN) }
#undef JFFT_LC_SWITCH

// Blocks along x of a pass that writes one partial sum per (component, block): at most
// kMaxPartials / d, the blocks then taking several row groups each.
static inline unsigned partial_blocks(int64_t groups, int d) {
  return (unsigned)std::min<int64_t>(groups, kMaxPartials / d);
}

// Real rows (last axis) forward, S = nb * d slabs. With xr.x set, the PCG update
// x += alpha p, r -= alpha q runs in the pass (r is xr.r) and its last block applies
// the residual stage xr.sc.
template <typename T>
static cudaError_t pass_rows_real_fwd(const Grid& g, const FftPlanT<T>& p, const T* r, int nb, bool jac, const T* js,
                                      const JScaleT<T>& jsc, const CgState* cg, cudaStream_t st,
                                      const XrUpdate<T>& xr, int* nparts) {
  const int Lin = g.n[g.d - 1];
  const int R = (int)(g.N / Lin);
  const int L = Lin / 2;
  const int w = std::max(1, rows_per_cta<T>(L, R, Lin) / std::max(1, g.tune[2]));
  const size_t smem = rows_smem<T>(L, w, Lin);
  const bool fused = xr.x != nullptr;
  dim3 grid(fused ? partial_blocks(R / w, g.d) : (unsigned)(R / w), nb * g.d);
  const int tpl = lanes_per_line<T>(L);
  auto k = fused ? (jac ? rows_kernel<T, true, true, true>(L) : rows_kernel<T, true, false, true>(L))
                 : (jac ? rows_kernel<T, true, true, false>(L) : rows_kernel<T, true, false, false>(L));
  JFFT_TRY(set_smem(k, smem));
  const char* name = fused ? nm<T>("fft_rows_real_fwd_xr", "fft_rows_real_fwd_xr_f32")
                           : nm<T>("fft_rows_real_fwd", "fft_rows_real_fwd_f32");
  JFFT_K(name, st,
         k<<<grid, w * tpl, smem, st>>>(g.d, fused ? nullptr : r, nullptr, p.T, R, Lin, ilog2(tpl), ilog2(w),
                                        p.tw[g.d - 1], p.lf[g.d - 1], js, jsc, cg, g.d, xr));
  if (fused && nparts) *nparts = grid.x * g.d;
  return cudaGetLastError();
}

// 3D: complex rows along axis 1 of T[S'][n0][n1] -> U[S'][n1][n0].
template <typename T>
static cudaError_t pass_rows_cplx_fwd(const Grid& g, const FftPlanT<T>& p, int nb, const CgState* cg, cudaStream_t st) {
  const int R = g.n[0], Lin = g.n[1];
  const int w = rows_per_cta<T>(Lin, R, Lin);
  const size_t smem = rows_smem<T>(Lin, w, Lin);
  const int slabs = nb * g.d * (g.M + 1);
  dim3 grid(R / w, slabs);
  const int tpl = lanes_per_line<T>(Lin);
  auto k = rows_kernel<T, false, false, false>(Lin);
  JFFT_TRY(set_smem(k, smem));
  JScaleT<T> jsc = {};
  JFFT_K(nm<T>("fft_rows_cplx_fwd", "fft_rows_cplx_fwd_f32"), st,
         k<<<grid, w * tpl, smem, st>>>(g.d, nullptr, p.T, p.U, R, Lin, ilog2(tpl), ilog2(w), p.tw[1], p.lf[1], nullptr,
                                        jsc, cg, g.d * (g.M + 1), XrUpdate<T>{}));
  return cudaGetLastError();
}

template <typename T>
static cudaError_t pass_lines(const Grid& g, const FftPlanT<T>& p, int nb, bool green, const CgState* cg,
                              cudaStream_t st) {
  const int L = g.n[0];
  const int nlines = (int)(g.F / L);
  cplx<T>* spec = (g.d == 2) ? p.T : p.U;
  const size_t smem = ((size_t)2 * g.d * line_slots(L) + L) * sizeof(cplx<T>);
  const int tpl = lanes_per_line<T>(L);
  dim3 grid(nlines, nb);
  const char* name = green ? nm<T>("fft_lines", "fft_lines_f32") : nm<T>("fft_lines_fwd", "fft_lines_fwd_f32");
  if (g.d == 2) {
    auto k = green ? lines_kernel<T, 2, true>(L) : lines_kernel<T, 2, false>(L);
    JFFT_TRY(set_smem(k, smem));
    JFFT_K(name, st, k<<<grid, 2 * tpl, smem, st>>>(spec, nlines, L, ilog2(tpl), p.tw[0], p.lf[0], p.G, cg));
  } else {
    auto k = green ? lines_kernel<T, 3, true>(L) : lines_kernel<T, 3, false>(L);
    JFFT_TRY(set_smem(k, smem));
    JFFT_K(name, st, k<<<grid, 3 * tpl, smem, st>>>(spec, nlines, L, ilog2(tpl), p.tw[0], p.lf[0], p.G, cg));
  }
  return cudaGetLastError();
}

// 3D: complex inverse along axis 1, U[S'][n1][n0] -> T[S'][n0][n1].
template <typename T>
static cudaError_t pass_cols_cplx_inv(const Grid& g, const FftPlanT<T>& p, int nb, CgState* cg, cudaStream_t st) {
  const int R = g.n[0], Lin = g.n[1];
  const int w = rows_per_cta<T>(Lin, R, Lin);
  const size_t smem = rows_smem<T>(Lin, w, Lin);
  const int slabs = nb * g.d * (g.M + 1);
  dim3 grid(R / w, slabs);
  const int tpl = lanes_per_line<T>(Lin);
  auto k = cols_kernel<T, false, false, false>(Lin);
  JFFT_TRY(set_smem(k, smem));
  JScaleT<T> jsc = {};
  JFFT_K(nm<T>("fft_cols_cplx_inv", "fft_cols_cplx_inv_f32"), st,
         k<<<grid, w * tpl, smem, st>>>(g.d, p.U, nullptr, p.T, R, Lin, ilog2(tpl), ilog2(w), p.tw[1], p.lf[1], nullptr,
                                        jsc, nullptr, nullptr, cg, g.d * (g.M + 1), no_stage()));
  return cudaGetLastError();
}

template <typename T>
static cudaError_t pass_cols_real_inv(const Grid& g, const FftPlanT<T>& p, T* z, int nb, bool jac, const T* js,
                                      const JScaleT<T>& jsc, const T* r, double* partial, int* nparts,
                                      CgState* cg, cudaStream_t st, StageCtl sc) {
  const int n = g.n[g.d - 1];
  const int R = (int)(g.N / n);
  const int L = n / 2;
  const int w = std::max(1, rows_per_cta<T>(L, R, n) / std::max(1, g.tune[3]));
  const size_t smem = rows_smem<T>(L, w, n);
  dim3 grid(partial_blocks(R / w, g.d), nb * g.d);
  const int tpl = lanes_per_line<T>(L);
  const bool multi = (int64_t)grid.x < R / w;
  auto k = multi ? (jac ? cols_kernel<T, true, true, true>(L) : cols_kernel<T, true, false, true>(L))
                 : (jac ? cols_kernel<T, true, true, false>(L) : cols_kernel<T, true, false, false>(L));
  JFFT_TRY(set_smem(k, smem));
  JFFT_K(nm<T>("fft_cols_real_inv", "fft_cols_real_inv_f32"), st,
         k<<<grid, w * tpl, smem, st>>>(g.d, p.T, z, nullptr, R, L + 1, ilog2(tpl), ilog2(w), p.tw[g.d - 1],
                                        p.lf[g.d - 1], js, jsc, r, partial, cg, g.d, sc));
  if (nparts) *nparts = grid.x * g.d;
  return cudaGetLastError();
}

template <typename T>
static cudaError_t green_precond_t(const Grid& g, const FftPlanT<T>& p, const T* r, T* z, int nb, const T* js,
                                   bool jacobi, double* partial, int* nparts, CgState* done, cudaStream_t st,
                                   StageCtl sc, int64_t jcs, const XrUpdate<T>& xr = XrUpdate<T>{}) {
  JScaleT<T> jsc;
  jsc.cs = jcs;
  JFFT_TRY(pass_rows_real_fwd<T>(g, p, r, nb, jacobi, js, jsc, done, st, xr, nullptr));
  if (g.d == 3) JFFT_TRY(pass_rows_cplx_fwd<T>(g, p, nb, done, st));
  JFFT_TRY(pass_lines<T>(g, p, nb, true, done, st));
  if (g.d == 3) JFFT_TRY(pass_cols_cplx_inv<T>(g, p, nb, done, st));
  return pass_cols_real_inv<T>(g, p, z, nb, jacobi, js, jsc, r, partial, nparts, done, st, sc);
}

template <typename T>
static cudaError_t green_precond_xr_t(const Grid& g, const FftPlanT<T>& p, T* x, T* r, const T* pv, const T* q, T* z,
                                      int nb, const T* js, bool jacobi, double* partial, int* nparts, CgState* cg,
                                      cudaStream_t st, StageCtl sc_rr, StageCtl sc, int64_t jcs) {
  const XrUpdate<T> xr{x, r, pv, q, partial, cg, sc_rr};
  return green_precond_t<T>(g, p, r, z, nb, js, jacobi, partial, nparts, cg, st, sc, jcs, xr);
}

}  // namespace jfft
