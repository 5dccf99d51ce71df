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
// eight lanes of a warp on one shared-memory bank.
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
#pragma unroll
    for (int r = 1; r < R; ++r) {
      cplx<T> w = tst[NS - RM + (r - 1) * NS + k];
      if (INV) w.y = -w.y;
      x[r] = c_mul<T>(x[r], w);
    }
    Dft<T, R, INV>::run(x, one);
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
