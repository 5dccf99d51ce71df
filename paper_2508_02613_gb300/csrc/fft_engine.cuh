// Register-resident Stockham engine for one line of length L (power of two).
//
// A line is handled by TPL = L / RM_eff threads (RM_eff = min(RM, L)); lane j of a
// line holds RM_eff values. The first stage takes its inputs from registers
// (positions j + TPL r) and runs radix RM_eff; later stages read their inputs from
// shared memory at Stockham positions b + r L/R, multiply by table twiddles
// W_{Ns R}^{r k}, run an in-register DFT of size R (16, 8, 4 or 2) and write
// (b - k) R + k + r Ns, alternating between two buffers with one barrier per stage.
// The result is left in natural order in the returned buffer.
//
// Shared-memory layout of a line: element p lives at spad(p) = p + p / 16. The
// stride-R writes of the first stages would otherwise put all lanes of a warp on
// the same banks; with the padding every stage's reads and writes are
// conflict-free for 8-byte elements.
#pragma once

#include "jfft_internal.cuh"

namespace jfft {

__host__ __device__ __forceinline__ int spad(int p) { return p + (p >> 4); }
// Shared-memory slots of a line holding elements 0..n (inclusive).
__host__ __device__ __forceinline__ int line_slots(int n) { return spad(n) + 1; }
// Stride between the w lines of a row-pass block: at least line_slots(L); for 8-byte
// elements on lines of 256 or more (a warp's lanes then work on one line in every
// stage) also congruent to 32 / w modulo 16 slots, so that a warp reading or writing
// element k of every line (the transposed input and output of the row passes: 32 / w
// consecutive k on each of w lines) touches every bank pair exactly twice.
template <typename T> __host__ __device__ __forceinline__ int line_stride(int L, int w) {
  const int s = line_slots(L);
  if (sizeof(cplx<T>) != 8 || L < 256 || w < 2 || w > 32) return s;
  const int want = (32 / w) & 15;
  return s + (((want - s) % 16) + 16) % 16;
}

// Sums and differences. GB300 issues FP64 FMA at 1.19x the rate of FP64 add (probe: 0.596
// vs 0.502 T instructions/s), so in FP64 a + b is formed as fma(a, one, b) with `one` = 1
// read at run time (a literal 1 would be folded back into an add); the rounding is that
// of a + b. FP32 adds and FMAs issue at the same rate.
template <typename T> __device__ __forceinline__ T add1(T a, T b, T one) {
  if constexpr (sizeof(T) == 8) return fma(a, one, b);
  else return a + b;
}
template <typename T> __device__ __forceinline__ T sub1(T a, T b, T one) {
  if constexpr (sizeof(T) == 8) return fma(b, -one, a);
  else return a - b;
}
template <typename T> __device__ __forceinline__ cplx<T> c_add(cplx<T> a, cplx<T> b, T one) {
  return mk<T>(add1(a.x, b.x, one), add1(a.y, b.y, one));
}
template <typename T> __device__ __forceinline__ cplx<T> c_sub(cplx<T> a, cplx<T> b, T one) {
  return mk<T>(sub1(a.x, b.x, one), sub1(a.y, b.y, one));
}
template <typename T> __device__ __forceinline__ cplx<T> c_mul(cplx<T> a, cplx<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// multiply by -i (forward) or +i (inverse)
template <typename T, bool INV> __device__ __forceinline__ cplx<T> c_mi(cplx<T> a) {
  return INV ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}

// In-register DFT of size R, natural order in and out.
template <typename T, int R, bool INV> struct Dft;

template <typename T, bool INV> struct Dft<T, 1, INV> {
  __device__ __forceinline__ static void run(cplx<T>*, T) {}
};

template <typename T, bool INV> struct Dft<T, 2, INV> {
  __device__ __forceinline__ static void run(cplx<T>* v, T one) {
    const cplx<T> a = v[0], b = v[1];
    v[0] = c_add<T>(a, b, one);
    v[1] = c_sub<T>(a, b, one);
  }
};

template <typename T, bool INV> struct Dft<T, 4, INV> {
  __device__ __forceinline__ static void run(cplx<T>* v, T one) {
    const cplx<T> s02 = c_add<T>(v[0], v[2], one), d02 = c_sub<T>(v[0], v[2], one);
    const cplx<T> s13 = c_add<T>(v[1], v[3], one), d13 = c_mi<T, INV>(c_sub<T>(v[1], v[3], one));
    v[0] = c_add<T>(s02, s13, one);
    v[2] = c_sub<T>(s02, s13, one);
    v[1] = c_add<T>(d02, d13, one);
    v[3] = c_sub<T>(d02, d13, one);
  }
};

// Radix-2 split of a size-2H DFT into two size-H DFTs (even / odd samples):
// X[k] = E[k] + W^k O[k], X[k + H] = E[k] - W^k O[k], W = exp(-+ 2 pi i / 2H).
// W^0 = 1 and W^(H/2) = -+i are applied without multiplications (same values up to
// the sign of zero results).
template <typename T, int H, bool INV> __device__ __forceinline__ void split2(cplx<T>* v, const cplx<T>* w, T one) {
  cplx<T> e[H], o[H];
#pragma unroll
  for (int k = 0; k < H; ++k) {
    e[k] = v[2 * k];
    o[k] = v[2 * k + 1];
  }
  Dft<T, H, INV>::run(e, one);
  Dft<T, H, INV>::run(o, one);
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const cplx<T> t = k == 0 ? o[k] : (2 * k == H ? c_mi<T, INV>(o[k]) : c_mul<T>(o[k], w[k]));
    v[k] = c_add<T>(e[k], t, one);
    v[k + H] = c_sub<T>(e[k], t, one);
  }
}

template <typename T, bool INV> struct Dft<T, 8, INV> {
  __device__ __forceinline__ static void run(cplx<T>* v, T one) {
    const T r = T(0.70710678118654752440);
    const T sg = INV ? T(1) : T(-1);
    const cplx<T> w[4] = {mk<T>(T(1), T(0)), mk<T>(r, sg * r), mk<T>(T(0), sg), mk<T>(-r, sg * r)};
    split2<T, 4, INV>(v, w, one);
  }
};

template <typename T, bool INV> struct Dft<T, 16, INV> {
  __device__ __forceinline__ static void run(cplx<T>* v, T one) {
    const T c1 = T(0.92387953251128675613), s1 = T(0.38268343236508977173), r = T(0.70710678118654752440);
    const T sg = INV ? T(1) : T(-1);
    const cplx<T> w[8] = {mk<T>(T(1), T(0)), mk<T>(c1, sg * s1), mk<T>(r, sg * r), mk<T>(s1, sg * c1),
                          mk<T>(T(0), sg),   mk<T>(-s1, sg * c1), mk<T>(-r, sg * r), mk<T>(-c1, sg * s1)};
    split2<T, 8, INV>(v, w, one);
  }
};

// Fused multiply-add butterflies for the twiddled stages of the FP64 compile-time
// engine (Linzer and Feig, "Modified FFTs for fused multiply-add architectures", Math.
// Comp. 60 (1993)): a twiddle w = c (1 + i t), c = Re w, t = Im w / Re w, turns
// a +- w b into u = b (1 + i t) (two FMAs) and a +- c u (two FMAs per output): six FP64
// instructions where a complex multiply and two complex adds take eight. A radix-R
// stage runs as log2 R radix-2 decimation-in-time layers, each with its own twiddles
// (R - 1 per index k, in the slots of the plain stage's table). Same accuracy as the
// plain form: |w b| rounds relative to |b| in both.
template <typename T, bool INV> __device__ __forceinline__ void lf_bfly(cplx<T>& a, cplx<T>& b, cplx<T> w) {
  const T t = INV ? -w.y : w.y;
  const T ux = fma(-t, b.y, b.x), uy = fma(t, b.x, b.y);
  const cplx<T> p = mk<T>(fma(w.x, ux, a.x), fma(w.x, uy, a.y));
  b = mk<T>(fma(-w.x, ux, a.x), fma(-w.x, uy, a.y));
  a = p;
}

// Exponent q of the layer twiddle W_{R NS}^q in slot e of index k (stage of span NS,
// radix R): the lowest layer pairs (x_c, x_{c + R/2}) with W_{2 NS}^k, the next pairs the
// results with W_{4 NS}^{k + NS m}, the top with W_{8 NS}^{k + NS m}, m = 0 .. R/2 - 1.
__host__ __device__ inline int lf_exponent(int R, int NS, int e, int k) {
  if (R == 2) return k;
  if (R == 4) return e == 0 ? 2 * k : k + (e - 1) * NS;
  if (e == 0) return 4 * k;
  if (e <= 2) return 2 * k + (e - 1) * 2 * NS;
  return k + (e - 3) * NS;
}

// x: the R stage inputs (positions b + r L / R), natural-order outputs on return; tk: the
// slot of index k in the stage table, slot e at tk[e * NS].
template <typename T, int R, bool INV, int NS>
__device__ __forceinline__ void lf_stage(cplx<T>* x, const cplx<T>* __restrict__ tk) {
  if constexpr (R == 2) {
    lf_bfly<T, INV>(x[0], x[1], tk[0]);
  } else if constexpr (R == 4) {
    const cplx<T> w0 = tk[0];
    lf_bfly<T, INV>(x[0], x[2], w0);   // x0 = E'0, x2 = E'1
    lf_bfly<T, INV>(x[1], x[3], w0);   // x1 = O'0, x3 = O'1
    lf_bfly<T, INV>(x[0], x[1], tk[NS]);       // X0, X2
    lf_bfly<T, INV>(x[2], x[3], tk[2 * NS]);   // X1, X3
    const cplx<T> x1 = x[1];
    x[1] = x[2];
    x[2] = x1;
  } else {
    static_assert(R == 8, "fused stages of radix 2, 4 or 8");
    const cplx<T> w0 = tk[0], w1 = tk[NS], w2 = tk[2 * NS];
#pragma unroll
    for (int c = 0; c < 4; ++c) lf_bfly<T, INV>(x[c], x[c + 4], w0);
    // even subsequence: x0 / x4 (pair 0, 4) with x2 / x6 (pair 2, 6); odd: 1 / 5 with 3 / 7
    lf_bfly<T, INV>(x[0], x[2], w1);   // E0, E2
    lf_bfly<T, INV>(x[4], x[6], w2);   // E1, E3
    lf_bfly<T, INV>(x[1], x[3], w1);   // O0, O2
    lf_bfly<T, INV>(x[5], x[7], w2);   // O1, O3
    lf_bfly<T, INV>(x[0], x[1], tk[3 * NS]);   // X0, X4
    lf_bfly<T, INV>(x[4], x[5], tk[4 * NS]);   // X1, X5
    lf_bfly<T, INV>(x[2], x[3], tk[5 * NS]);   // X2, X6
    lf_bfly<T, INV>(x[6], x[7], tk[6 * NS]);   // X3, X7
    const cplx<T> y[8] = {x[0], x[4], x[2], x[6], x[1], x[5], x[3], x[7]};
#pragma unroll
    for (int r = 0; r < 8; ++r) x[r] = y[r];
  }
}

// One Stockham stage of radix R: each of the TPL lanes does RME / R butterflies.
// FROM_REGS: inputs are v (stage 1 only, R == RME, positions j + TPL r).
// tw: twiddle table exp(-2 pi i m / (L tws)) in shared memory (read with plain loads).
template <typename T, int RME, int R, bool INV, bool FROM_REGS>
__device__ __forceinline__ void fft_stage(const cplx<T>* __restrict__ src, cplx<T>* __restrict__ dst, cplx<T>* v, int j,
                                          int TPL, int L, int Ns, const cplx<T>* __restrict__ tw, int tws, T one) {
  const int step = L / R;
#pragma unroll
  for (int i = 0; i < RME / R; ++i) {
    const int b = j + TPL * i;
    const int k = b & (Ns - 1);
    cplx<T> x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = FROM_REGS ? v[r] : src[spad(b + r * step)];
    if (!FROM_REGS && Ns > 1) {
      const int m1 = k * (L / (Ns * R)) * tws;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cplx<T> w = tw[r * m1];  // tw is the block's shared-memory copy of the table
        if (INV) w.y = -w.y;
        x[r] = c_mul<T>(x[r], w);
      }
    }
    Dft<T, R, INV>::run(x, one);
    const int base = (b - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[spad(base + r * Ns)] = x[r];
  }
}

// FFT of one line; every thread of the block calls it with the same L (one barrier
// per stage). v: the lane's RME inputs (positions j + TPL r). b0 / b1: the line's two
// shared-memory buffers. Returns the buffer holding the natural-order result.
template <typename T, int RM, bool INV>
__device__ cplx<T>* line_fft(cplx<T>* v, int j, int L, cplx<T>* b0, cplx<T>* b1, const cplx<T>* __restrict__ tw,
                             int tws, T one) {
  cplx<T>* cur = b0;
  cplx<T>* nxt = b1;
  int Ns;
  if (L >= RM) {
    const int TPL = L / RM;
    fft_stage<T, RM, RM, INV, true>(nullptr, cur, v, j, TPL, L, 1, tw, tws, one);
    Ns = RM;
  } else {
    // one lane holds the whole line (TPL = 1, j = 0)
    switch (L) {
      case 2: fft_stage<T, 2, 2, INV, true>(nullptr, cur, v, j, 1, L, 1, tw, tws, one); break;
      case 4: fft_stage<T, 4, 4, INV, true>(nullptr, cur, v, j, 1, L, 1, tw, tws, one); break;
      case 8: fft_stage<T, 8, 8, INV, true>(nullptr, cur, v, j, 1, L, 1, tw, tws, one); break;
      default: break;
    }
    Ns = L;
  }
  __syncthreads();
  const int TPL = L >= RM ? L / RM : 1;
  while (Ns < L) {
    const int rem = L / Ns;
    if (rem >= RM) {
      fft_stage<T, RM, RM, INV, false>(cur, nxt, v, j, TPL, L, Ns, tw, tws, one);
      Ns *= RM;
    } else {
      switch (rem) {
        case 2: fft_stage<T, RM, 2, INV, false>(cur, nxt, v, j, TPL, L, Ns, tw, tws, one); break;
        case 4: fft_stage<T, RM, 4, INV, false>(cur, nxt, v, j, TPL, L, Ns, tw, tws, one); break;
        case 8: fft_stage<T, RM, 8, INV, false>(cur, nxt, v, j, TPL, L, Ns, tw, tws, one); break;
        default: break;
      }
      Ns = L;
    }
    cplx<T>* t = cur;
    cur = nxt;
    nxt = t;
    __syncthreads();
  }
  return cur;
}

// The same FFT with the line length L (>= RM) known at compile time: the stages unroll
// with constant radix, Stockham stride and twiddle step, so the per-access index
// arithmetic folds into shifts and masks of the lane index j (the runtime form spends
// more issue slots on integer work than on the butterflies). The twiddles come from
// per-stage tables: the stage of span NS (> 1) and radix R keeps W_{NS R}^{r k}
// (forward sign) at NS - RM + (r - 1) NS + k, k < NS, 1 <= r < R, L - RM entries in all.
// Lanes read consecutive k there, where the strided reads of the axis table put up to
// eight lanes of a warp on one shared-memory bank. FP64 runs the fused multiply-add
// stages (lf_stage): the same slots hold (c, t) of W_{NS R}^{lf_exponent(R, NS, r - 1, k)},
// built once per plan (k_lf_table).
template <int RM, int L, int NS> struct StageRadix {
  static constexpr int R = (L / NS) >= RM ? RM : (L / NS);
};

// Fills the per-stage tables from the axis table tw_axis (exp(-2 pi i m / (L TWS))).
template <typename T, int RM, int L, int TWS, int NS = RM>
__device__ __forceinline__ void fill_stage_twiddles(cplx<T>* dst, const cplx<T>* __restrict__ tw_axis) {
  if constexpr (NS < L) {
    constexpr int R = StageRadix<RM, L, NS>::R;
    for (int i = threadIdx.x; i < NS * (R - 1); i += blockDim.x) {
      const int r = i / NS + 1, k = i % NS;
      dst[NS - RM + i] = tw_axis[r * k * (L / (NS * R)) * TWS];
    }
    fill_stage_twiddles<T, RM, L, TWS, NS * R>(dst, tw_axis);
  }
}

// The block's per-stage tables: FP64 copies the plan's fused-form table (lf, L - RM
// entries), FP32 gathers the plain twiddles from the axis table.
template <typename T, int RM, int L, int TWS>
__device__ __forceinline__ void stage_twiddles(cplx<T>* dst, const cplx<T>* __restrict__ tw_axis,
                                               const cplx<T>* __restrict__ lf) {
  if constexpr (sizeof(T) == 8) {
    for (int i = threadIdx.x; i < L - RM; i += blockDim.x) dst[i] = lf[i];
  } else {
    fill_stage_twiddles<T, RM, L, TWS>(dst, tw_axis);
  }
}

template <typename T, int RM, int R, bool INV, int L, int NS>
__device__ __forceinline__ void fft_stage_ct(const cplx<T>* __restrict__ src, cplx<T>* __restrict__ dst, int j,
                                             const cplx<T>* __restrict__ tst, T one) {
  constexpr int TPL = L / RM;
  constexpr int step = L / R;
#pragma unroll
  for (int i = 0; i < RM / R; ++i) {
    const int b = j + TPL * i;
    const int k = b & (NS - 1);
    cplx<T> x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = src[spad(b + r * step)];
    if constexpr (sizeof(T) == 8) {
      lf_stage<T, R, INV, NS>(x, tst + NS - RM + k);
    } else {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cplx<T> w = tst[NS - RM + (r - 1) * NS + k];
        if (INV) w.y = -w.y;
        x[r] = c_mul<T>(x[r], w);
      }
      Dft<T, R, INV>::run(x, one);
    }
    const int base = (b - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[spad(base + r * NS)] = x[r];
  }
}

template <typename T, int RM, bool INV, int L, int NS>
__device__ __forceinline__ void line_stages_ct(cplx<T>*& cur, cplx<T>*& nxt, int j, const cplx<T>* __restrict__ tst,
                                               T one) {
  if constexpr (NS < L) {
    constexpr int R = StageRadix<RM, L, NS>::R;
    fft_stage_ct<T, RM, R, INV, L, NS>(cur, nxt, j, tst, one);
    cplx<T>* t = cur;
    cur = nxt;
    nxt = t;
    __syncthreads();
    line_stages_ct<T, RM, INV, L, NS * R>(cur, nxt, j, tst, one);
  }
}

// tst: the block's per-stage tables (fill_stage_twiddles), ordered before the call by
// a barrier.
template <typename T, int RM, bool INV, int L>
__device__ __forceinline__ cplx<T>* line_fft_ct(cplx<T>* v, int j, cplx<T>* b0, cplx<T>* b1,
                                                const cplx<T>* __restrict__ tst, T one) {
  static_assert(L >= RM, "compile-time lines hold at least one radix-RM butterfly per lane");
  cplx<T>* cur = b0;
  cplx<T>* nxt = b1;
  fft_stage<T, RM, RM, INV, true>(nullptr, cur, v, j, L / RM, L, 1, nullptr, 1, one);
  __syncthreads();
  line_stages_ct<T, RM, INV, L, RM>(cur, nxt, j, tst, one);
  return cur;
}

}  // namespace jfft
