/*
 * Timed CPU baseline of the J-FFT solve (TEST INFRASTRUCTURE, not the product): the
 * oracle's PCG (Saad Alg. 9.1, x_0 = 0, relative residual test on the recursive
 * residual; paper Sec. 2.3, Sec. 4 "Termination criteria") with
 *   - the operator K = B^T W C B applied matrix-free: node I, component alpha
 *       (K p)_{alpha I} = sum over the 2^d elements e = I - o that contain I of
 *       E_e sum_{beta, c} A[(alpha, o), (beta, c)] (p_beta(e + c) - p_beta(e)),
 *     A the unit-modulus element matrix (local DOF alpha * 2^d + corner, corner
 *     o in {0,1}^d lexicographic, last axis fastest); gathering per node lets
 *     OpenMP threads own disjoint rows of the output;
 *   - the Green preconditioner F^-1 G_hat F (Eq. prec_lin_systemG_FFT) with a
 *     textbook iterative radix-2 complex FFT (bit reversal, then log2 L stages of
 *     butterflies) along every axis, unnormalised forward, 1/N on the inverse;
 *     G_hat real symmetric per frequency, applied as z_hat_b = sum_a G[a][b] r_hat_a;
 *   - Green-Jacobi: z = J^1/2 F^-1 G_hat F J^1/2 r (Eq. prec_lin_systemJG_2).
 * FP64 throughout; inner products are OpenMP reductions. The element matrix, the
 * symbol and J^1/2 come from the Python oracle (setup is not part of this file).
 * Shares no code with the CUDA library.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static const double TWO_PI = 6.283185307179586476925286766559;

typedef struct {
  double re, im;
} cplx;

typedef struct {
  int d;
  int64_t n[3];
  int64_t N;
  int nc;          /* 2^d corners */
  const double* E; /* [N] */
  const double* A; /* [(d nc)^2] */
  const double* G; /* [d][d][N] real symbol, full spectrum, C order */
  const double* J; /* [d][N] J^1/2 per DOF, or NULL (Green) */
  cplx* work;      /* [d][N] */
} problem;

static int64_t wrap(int64_t i, int64_t n) { return ((i % n) + n) % n; }

static int64_t flat(const problem* P, const int64_t* idx) {
  int64_t f = 0;
  for (int a = 0; a < P->d; ++a) f = f * P->n[a] + idx[a];
  return f;
}

/* q = K p */
static void apply_K(const problem* P, const double* p, double* q) {
  const int d = P->d, nc = P->nc, nd = d * nc;
  const int64_t N = P->N;
#pragma omp parallel for schedule(static)
  for (int64_t I = 0; I < N; ++I) {
    int64_t idx[3], rem = I;
    for (int a = d - 1; a >= 0; --a) {
      idx[a] = rem % P->n[a];
      rem /= P->n[a];
    }
    double acc[3] = {0.0, 0.0, 0.0};
    for (int o = 0; o < nc; ++o) {
      /* element e = I - o, with I at its corner o */
      int64_t e[3], cn[8];
      for (int a = 0; a < d; ++a) e[a] = wrap(idx[a] - ((o >> (d - 1 - a)) & 1), P->n[a]);
      for (int c = 0; c < nc; ++c) {
        int64_t v[3];
        for (int a = 0; a < d; ++a) v[a] = wrap(e[a] + ((c >> (d - 1 - a)) & 1), P->n[a]);
        cn[c] = flat(P, v);
      }
      const double Ee = P->E[cn[0]];
      for (int al = 0; al < d; ++al) {
        const double* row = P->A + (int64_t)(al * nc + o) * nd;
        double s = 0.0;
        for (int be = 0; be < d; ++be) {
          const double* pb = p + (int64_t)be * N;
          const double base = pb[cn[0]];
          for (int c = 1; c < nc; ++c) s += row[be * nc + c] * (pb[cn[c]] - base);
        }
        acc[al] += Ee * s;
      }
    }
    for (int al = 0; al < d; ++al) q[(int64_t)al * N + I] = acc[al];
  }
}

/* In-place radix-2 FFT of one line of length L (power of two); w[k] = exp(sign 2 pi i k / L)
   for k < L/2 (sign -1 forward, +1 inverse). */
static void fft_line(cplx* x, int64_t L, const cplx* w) {
  for (int64_t i = 1, j = 0; i < L; ++i) {
    int64_t bit = L >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      cplx t = x[i];
      x[i] = x[j];
      x[j] = t;
    }
  }
  for (int64_t len = 2; len <= L; len <<= 1) {
    const int64_t step = L / len;   /* exp(sign 2 pi i k / len) = w[k step] */
    for (int64_t i = 0; i < L; i += len) {
      for (int64_t k = 0; k < len / 2; ++k) {
        const double wr = w[k * step].re, wi = w[k * step].im;
        cplx u = x[i + k], v = x[i + k + len / 2];
        const double tr = v.re * wr - v.im * wi, ti = v.re * wi + v.im * wr;
        x[i + k].re = u.re + tr;
        x[i + k].im = u.im + ti;
        x[i + k + len / 2].re = u.re - tr;
        x[i + k + len / 2].im = u.im - ti;
      }
    }
  }
}

/* d-dimensional transform of one component field (C order) along every axis. */
static void fft_field(const problem* P, cplx* f, int sign) {
  const int d = P->d;
  for (int ax = 0; ax < d; ++ax) {
    const int64_t L = P->n[ax];
    int64_t stride = 1;
    for (int b = ax + 1; b < d; ++b) stride *= P->n[b];
    const int64_t lines = P->N / L;
    cplx* w = (cplx*)malloc(sizeof(cplx) * (size_t)(L / 2 + 1));
    for (int64_t k = 0; k < L / 2 + 1; ++k) {
      w[k].re = cos(sign * TWO_PI * (double)k / (double)L);
      w[k].im = sin(sign * TWO_PI * (double)k / (double)L);
    }
#pragma omp parallel
    {
      cplx* buf = (cplx*)malloc(sizeof(cplx) * (size_t)L);
#pragma omp for schedule(static)
      for (int64_t li = 0; li < lines; ++li) {
        /* line li: outer index (above ax) and inner index (below ax) */
        const int64_t inner = li % stride, outer = li / stride;
        cplx* base = f + outer * L * stride + inner;
        for (int64_t t = 0; t < L; ++t) buf[t] = base[t * stride];
        fft_line(buf, L, w);
        for (int64_t t = 0; t < L; ++t) base[t * stride] = buf[t];
      }
      free(buf);
    }
    free(w);
  }
}

/* z = M^-1 r */
static void precond(const problem* P, const double* r, double* z) {
  const int d = P->d;
  const int64_t N = P->N;
  for (int a = 0; a < d; ++a) {
    cplx* w = P->work + (int64_t)a * N;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
      w[i].re = P->J ? P->J[(int64_t)a * N + i] * r[(int64_t)a * N + i] : r[(int64_t)a * N + i];
      w[i].im = 0.0;
    }
    fft_field(P, w, -1);
  }
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < N; ++k) {
    cplx in[3], out[3];
    for (int a = 0; a < d; ++a) in[a] = P->work[(int64_t)a * N + k];
    for (int b = 0; b < d; ++b) {
      out[b].re = out[b].im = 0.0;
      for (int a = 0; a < d; ++a) {
        const double g = P->G[((int64_t)a * d + b) * N + k];
        out[b].re += g * in[a].re;
        out[b].im += g * in[a].im;
      }
    }
    for (int b = 0; b < d; ++b) P->work[(int64_t)b * N + k] = out[b];
  }
  for (int b = 0; b < d; ++b) {
    cplx* w = P->work + (int64_t)b * N;
    fft_field(P, w, +1);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
      const double v = w[i].re / (double)N;
      z[(int64_t)b * N + i] = P->J ? P->J[(int64_t)b * N + i] * v : v;
    }
  }
}

static double dot(const double* a, const double* b, int64_t n) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/*
 * PCG for K u = f. d in {2, 3}; n[d] powers of two; E [N]; A [(d 2^d)^2]; G [d][d][N];
 * J [d][N] or NULL (Green); f, u [d][N] (u written). Returns the iteration count
 * (number of operator applications), or -1 for invalid arguments / no memory; *conv is
 * set to 1 if the relative residual reached tol within max_iter.
 */
int jfft_cpu_pcg(int d, const int64_t* n, const double* E, const double* A, const double* G, const double* J,
                 const double* f, double tol, int max_iter, double* u, int* conv) {
  if (d != 2 && d != 3) return -1;
  problem P;
  P.d = d;
  P.N = 1;
  for (int a = 0; a < d; ++a) {
    if (n[a] < 2 || (n[a] & (n[a] - 1))) return -1;
    P.n[a] = n[a];
    P.N *= n[a];
  }
  P.nc = 1 << d;
  P.E = E;
  P.A = A;
  P.G = G;
  P.J = J;
  const int64_t M = (int64_t)d * P.N;
  P.work = (cplx*)malloc(sizeof(cplx) * (size_t)M);
  double* r = (double*)malloc(sizeof(double) * (size_t)M);
  double* z = (double*)malloc(sizeof(double) * (size_t)M);
  double* p = (double*)malloc(sizeof(double) * (size_t)M);
  double* q = (double*)malloc(sizeof(double) * (size_t)M);
  if (!P.work || !r || !z || !p || !q) {
    free(P.work), free(r), free(z), free(p), free(q);
    return -1;
  }
  *conv = 0;
  memset(u, 0, sizeof(double) * (size_t)M);
  memcpy(r, f, sizeof(double) * (size_t)M);
  double rr = dot(r, r, M);
  const double nf = sqrt(rr);
  int k = 0;
  if (nf == 0.0 || sqrt(rr) <= tol * nf) {
    *conv = 1;
  } else {
    precond(&P, r, z);
    memcpy(p, z, sizeof(double) * (size_t)M);
    double gamma = dot(r, z, M);
    while (k < max_iter) {
      apply_K(&P, p, q);
      const double alpha = gamma / dot(p, q, M);
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < M; ++i) {
        u[i] += alpha * p[i];
        r[i] -= alpha * q[i];
      }
      rr = dot(r, r, M);
      ++k;
      if (sqrt(rr) <= tol * nf) {
        *conv = 1;
        break;
      }
      precond(&P, r, z);
      const double gnew = dot(r, z, M);
      const double beta = gnew / gamma;
      gamma = gnew;
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < M; ++i) p[i] = z[i] + beta * p[i];
    }
  }
  free(P.work), free(r), free(z), free(p), free(q);
  return k;
}

int jfft_cpu_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
