// Many small periodic cells in one launch: one CTA per (cell, load case) runs a
// complete solve out of shared memory (the paper's Sec. 2 cell problem with the
// Green or Green-Jacobi PCG of Sec. 3): material map, Alg. 1 symbol with the
// cell's own reference material, Jacobi scaling J^1/2 = diag(K)^-1/2 from the
// closed form kappa_a sum_{e ni I} E_e, right-hand side, the PCG iterations with
// every scalar kept in the CTA, then the zero-mean displacement, the true residual
// and the homogenised stress. 2D, FP64, n0 and n1 powers of two in [4, 32].
//
// Differences from the multi-kernel path, by construction of a one-CTA solve:
//   * the operator runs element-centric over four element colours (elements of one
//     colour share no node), so the nodal sums need no atomics and are
//     deterministic;
//   * the two displacement components are packed as one complex field, so one
//     complex 2D FFT (radix-2 Stockham along each axis) transforms both; the block
//     multiply separates them with Z(k) and conj Z(-k) and repacks the result;
//   * the symbol table covers the full spectrum and carries the 1/N of the inverse.
#include <algorithm>
#include <cmath>

#include "element.cuh"
#include "jfft.h"
#include "jfft_internal.cuh"
#include "reduce.cuh"

namespace jfft {

namespace {

struct CellJob {
  int n0, n1, lg0, lg1, N;
  int n_loads;
  int kind;
  double e_max, exponent;
  const double* field;     // [n_cells][N]
  const double* e_min;     // [n_cells]
  const ElemConst* ec;     // [n_cells] unit material C_unit(nu) of each cell
  const double* jscale;    // [n_cells][2] kappa_a^-1/2
  const StrainShift* shifts;  // [n_loads]
  double tol;
  int stop_mode, max_iter, pc;
  double void_js;
  double* u;        // [n_cells][n_loads][2][N] or NULL
  double* chom;     // [n_cells][3][n_loads] or NULL
  int* iters;       // [n_cells][n_loads] or NULL
  double* rel_res;  // [n_cells][n_loads] or NULL
  int* status;      // [n_cells][n_loads]
};

struct CellSmem {
  double* E;     // [N]
  double* js;    // [N] diag-sum^-1/2 (0 at void nodes)
  double* x;     // [2N]
  double* r;
  double* p;
  double* q;
  double* z;
  double* G;     // [3][N] symbol / N
  double2* A;    // [N] FFT buffers
  double2* B;
  double2* tw0;  // [n0]
  double2* tw1;  // [n1]
  double* red;   // [4] broadcast slots
};

__device__ __forceinline__ int cnode(const CellJob& j, int i0, int i1) {
  return ((i0 & (j.n0 - 1)) << j.lg1) + (i1 & (j.n1 - 1));
}

// Block-wide sum of a[i] * b[i], i < n, broadcast to every thread (fixed order).
__device__ double cell_dot(const double* a, const double* b, int n, double* slot) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc = fma(a[i], b[i], acc);
  const double v = block_sum(acc);
  if (threadIdx.x == 0) *slot = v;
  __syncthreads();
  const double out = *slot;
  __syncthreads();
  return out;
}

__device__ double cell_sum(double v, double* slot) {
  const double s = block_sum(v);
  if (threadIdx.x == 0) *slot = s;
  __syncthreads();
  const double out = *slot;
  __syncthreads();
  return out;
}

// dst = sgn * (K src + K_shift) over the four element colours; E uniform when E == NULL.
template <bool HAS_X, bool SHIFT>
__device__ void cell_apply_K(const CellJob& j, const ElemConst& ec, const double* E, double e_uniform,
                             const double* src, double* dst, const StrainShift* sh, double sgn) {
  const int N = j.N;
  for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) dst[i] = 0.0;
  __syncthreads();
  const int lgh1 = j.lg1 - 1;
  for (int color = 0; color < 4; ++color) {
    const int c0 = color >> 1, c1 = color & 1;
    for (int e = threadIdx.x; e < (N >> 2); e += blockDim.x) {
      const int i0 = 2 * (e >> lgh1) + c0, i1 = 2 * (e & ((1 << lgh1) - 1)) + c1;
      int nd[4];
      double u[2][4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        nd[c] = cnode(j, i0 + (c >> 1), i1 + (c & 1));
        u[0][c] = HAS_X ? src[nd[c]] : 0.0;
        u[1][c] = HAS_X ? src[N + nd[c]] : 0.0;
      }
      const double Ee = E ? E[(i0 << j.lg1) + i1] : e_uniform;
      element_force<2, double, SHIFT>(ec, sh, u, Ee);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        dst[nd[c]] += sgn * u[0][c];
        dst[N + nd[c]] += sgn * u[1][c];
      }
    }
    __syncthreads();
  }
}

// Radix-2 Stockham passes along one axis of the [n0][n1] complex array; returns the
// buffer holding the result (src or dst).
__device__ double2* cell_fft_axis(double2* src, double2* dst, int axis, bool inv, const CellJob& j,
                                  const double2* tw) {
  const int L = axis == 0 ? j.n0 : j.n1;
  const int lgL = axis == 0 ? j.lg0 : j.lg1;
  const int lines = j.N >> lgL;
  const int half = L >> 1;
  for (int Ns = 1; Ns < L; Ns <<= 1) {
    const int tstep = L / (2 * Ns);
    for (int t = threadIdx.x; t < lines * half; t += blockDim.x) {
      const int line = t >> (lgL - 1), jj = t & (half - 1);
      const int k = jj & (Ns - 1);
      // element (line, pos): axis 1 -> line * n1 + pos ; axis 0 -> pos * n1 + line
      auto at = [&](int pos) { return axis == 1 ? (line << j.lg1) + pos : (pos << j.lg1) + line; };
      const double2 v0 = src[at(jj)];
      const double2 b = src[at(jj + half)];
      double2 w = tw[k * tstep];
      if (inv) w.y = -w.y;
      const double2 v1 = make_double2(b.x * w.x - b.y * w.y, b.x * w.y + b.y * w.x);
      const int d = (jj - k) * 2 + k;
      dst[at(d)] = make_double2(v0.x + v1.x, v0.y + v1.y);
      dst[at(d + Ns)] = make_double2(v0.x - v1.x, v0.y - v1.y);
    }
    __syncthreads();
    double2* t = src;
    src = dst;
    dst = t;
  }
  return src;
}

__device__ double2* cell_fft2(const CellSmem& s, const CellJob& j, double2* data, bool inv) {
  double2* other = data == s.A ? s.B : s.A;
  double2* r1 = cell_fft_axis(data, other, 1, inv, j, s.tw1);
  double2* o2 = r1 == s.A ? s.B : s.A;
  return cell_fft_axis(r1, o2, 0, inv, j, s.tw0);
}

__device__ __forceinline__ int neg_k(const CellJob& j, int k) {
  const int k0 = k >> j.lg1, k1 = k & (j.n1 - 1);
  return (((j.n0 - k0) & (j.n0 - 1)) << j.lg1) + ((j.n1 - k1) & (j.n1 - 1));
}

// z = M^-1 r (Green or Green-Jacobi); returns r . z.
__device__ double cell_precond(const CellSmem& s, const CellJob& j, double ks0, double ks1, const double* r,
                               double* z) {
  const int N = j.N;
  const bool jac = j.pc == JFFT_PC_GREEN_JACOBI;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    double a = r[i], b = r[N + i];
    if (jac) {
      const double sj = s.js[i];
      a *= sj > 0.0 ? sj * ks0 : j.void_js;
      b *= sj > 0.0 ? sj * ks1 : j.void_js;
    }
    s.A[i] = make_double2(a, b);
  }
  __syncthreads();
  double2* Z = cell_fft2(s, j, s.A, false);
  double2* W = Z == s.A ? s.B : s.A;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const double2 zk = Z[k], zm = Z[neg_k(j, k)];
    // T0 = (Z + conj Zm) / 2, T1 = (Z - conj Zm) / (2i)
    const double2 t0 = make_double2(0.5 * (zk.x + zm.x), 0.5 * (zk.y - zm.y));
    const double2 t1 = make_double2(0.5 * (zk.y + zm.y), -0.5 * (zk.x - zm.x));
    const double g00 = s.G[k], g01 = s.G[N + k], g11 = s.G[2 * N + k];
    const double2 v0 = make_double2(g00 * t0.x + g01 * t1.x, g00 * t0.y + g01 * t1.y);
    const double2 v1 = make_double2(g01 * t0.x + g11 * t1.x, g01 * t0.y + g11 * t1.y);
    W[k] = make_double2(v0.x - v1.y, v0.y + v1.x);  // V0 + i V1
  }
  __syncthreads();
  double2* out = cell_fft2(s, j, W, true);
  double acc = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    double a = out[i].x, b = out[i].y;
    if (jac) {
      const double sj = s.js[i];
      a *= sj > 0.0 ? sj * ks0 : j.void_js;
      b *= sj > 0.0 ? sj * ks1 : j.void_js;
    }
    z[i] = a;
    z[N + i] = b;
    acc = fma(r[i], a, fma(r[N + i], b, acc));
  }
  return cell_sum(acc, s.red);
}

__global__ void __launch_bounds__(256) k_cells(CellJob j) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int N = j.N;
  const int cell = blockIdx.x / j.n_loads, load = blockIdx.x % j.n_loads;
  CellSmem s;
  {
    double2* c2p = reinterpret_cast<double2*>(sm_raw);
    s.A = c2p;
    s.B = c2p + N;
    s.tw0 = c2p + 2 * N;
    s.tw1 = s.tw0 + j.n0;
    double* d = reinterpret_cast<double*>(s.tw1 + j.n1);
    s.E = d;
    s.js = d + N;
    s.x = d + 2 * N;
    s.r = d + 4 * N;
    s.p = d + 6 * N;
    s.q = d + 8 * N;
    s.z = d + 10 * N;
    s.G = d + 12 * N;
    s.red = d + 15 * N;
  }
  const ElemConst ec = j.ec[cell];
  const double ks0 = j.jscale[2 * cell], ks1 = j.jscale[2 * cell + 1];
  const StrainShift sh = j.shifts[load];
  // twiddles and material
  for (int m = threadIdx.x; m < j.n0; m += blockDim.x) {
    double sn, cs;
    sincospi(-2.0 * (double)m / (double)j.n0, &sn, &cs);
    s.tw0[m] = make_double2(cs, sn);
  }
  for (int m = threadIdx.x; m < j.n1; m += blockDim.x) {
    double sn, cs;
    sincospi(-2.0 * (double)m / (double)j.n1, &sn, &cs);
    s.tw1[m] = make_double2(cs, sn);
  }
  const double* fld = j.field + (int64_t)cell * N;
  const double emin = j.kind == JFFT_MAT_DENSITY ? j.e_min[cell] : 0.0;
  double esum_local = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double v = fld[i];
    const double Ei = j.kind == JFFT_MAT_DENSITY ? emin + (j.e_max - emin) * pow(v, j.exponent) : v;
    s.E[i] = Ei;
    esum_local += Ei;
  }
  const double e_ref = cell_sum(esum_local, s.red) / (double)N;  // C_ref = mean(E) C_unit(nu)
  // J^1/2 node factors: (sum of the 4 adjacent E)^-1/2, 0 at void nodes
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int i0 = i >> j.lg1, i1 = i & (j.n1 - 1);
    const double es = s.E[cnode(j, i0, i1)] + s.E[cnode(j, i0 - 1, i1)] + s.E[cnode(j, i0, i1 - 1)] +
                      s.E[cnode(j, i0 - 1, i1 - 1)];
    s.js[i] = es > 0.0 ? 1.0 / sqrt(es) : 0.0;
  }
  // Alg. 1: responses of K_ref to unit impulses at node 0, transformed; K_hat kept
  // real and even (real part of the separated spectra), symmetrised and inverted.
  for (int alpha = 0; alpha < 2; ++alpha) {
    for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) s.x[i] = (i == alpha * N) ? 1.0 : 0.0;
    __syncthreads();
    cell_apply_K<true, false>(j, ec, nullptr, e_ref, s.x, s.q, nullptr, 1.0);
    for (int i = threadIdx.x; i < N; i += blockDim.x) s.A[i] = make_double2(s.q[i], s.q[N + i]);
    __syncthreads();
    double2* Z = cell_fft2(s, j, s.A, false);
    double* kh = alpha == 0 ? s.r : s.z;  // K_hat[alpha][0], K_hat[alpha][1]
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
      const double2 zk = Z[k], zm = Z[neg_k(j, k)];
      kh[k] = 0.5 * (zk.x + zm.x);      // Re of the spectrum of component 0
      kh[N + k] = 0.5 * (zk.y + zm.y);  // Re of the spectrum of component 1
    }
    __syncthreads();
  }
  const double inv_n = 1.0 / (double)N;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const double k00 = s.r[k], k11 = s.z[N + k];
    const double k01 = 0.5 * (s.r[N + k] + s.z[k]);
    if (k == 0) {
      s.G[k] = s.G[N + k] = s.G[2 * N + k] = 0.0;
    } else {
      const double det = k00 * k11 - k01 * k01;
      s.G[k] = k11 / det * inv_n;
      s.G[N + k] = -k01 / det * inv_n;
      s.G[2 * N + k] = k00 / det * inv_n;
    }
  }
  __syncthreads();
  // right-hand side f = -K_shift, ||f||^2
  cell_apply_K<false, true>(j, ec, s.E, 0.0, nullptr, s.r, &sh, -1.0);
  const double ff = cell_dot(s.r, s.r, 2 * N, s.red);
  const double rr_stop = j.stop_mode == JFFT_STOP_REL ? j.tol * j.tol * ff : j.tol;
  for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) s.x[i] = 0.0;
  int iters = 0;
  int done = (ff == 0.0 || ff <= rr_stop) ? kConverged : kRunning;
  if (!isfinite(ff)) done = kBreakdown;
  double gamma = 0.0;
  if (done == kRunning) {
    gamma = cell_precond(s, j, ks0, ks1, s.r, s.z);
    for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) s.p[i] = s.z[i];
    if (!(gamma > 0.0) || !isfinite(gamma)) done = kBreakdown;
  }
  __syncthreads();
  while (done == kRunning) {
    cell_apply_K<true, false>(j, ec, s.E, 0.0, s.p, s.q, nullptr, 1.0);
    const double pq = cell_dot(s.p, s.q, 2 * N, s.red);
    if (!(pq > 0.0) || !isfinite(pq)) { done = kBreakdown; break; }
    const double alpha = gamma / pq;
    double acc = 0.0;
    for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) {
      s.x[i] = fma(alpha, s.p[i], s.x[i]);
      const double rv = fma(-alpha, s.q[i], s.r[i]);
      s.r[i] = rv;
      acc = fma(rv, rv, acc);
    }
    const double rr = cell_sum(acc, s.red);
    ++iters;
    if (!isfinite(rr)) { done = kBreakdown; break; }
    if (rr <= rr_stop) { done = kConverged; break; }
    if (iters >= j.max_iter) { done = kNoConv; break; }
    const double gnew = cell_precond(s, j, ks0, ks1, s.r, s.z);
    if (!isfinite(gnew)) { done = kBreakdown; break; }
    const double beta = gnew / gamma;
    gamma = gnew;
    for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) s.p[i] = fma(beta, s.p[i], s.z[i]);
    __syncthreads();
  }
  __syncthreads();
  // zero-mean displacement
  double m0 = 0.0, m1 = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) { m0 += s.x[i]; m1 += s.x[N + i]; }
  m0 = cell_sum(m0, s.red) / (double)N;
  m1 = cell_sum(m1, s.red) / (double)N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) { s.x[i] -= m0; s.x[N + i] -= m1; }
  __syncthreads();
  // true residual f - K u
  cell_apply_K<true, true>(j, ec, s.E, 0.0, s.x, s.q, &sh, -1.0);
  const double rt = cell_dot(s.q, s.q, 2 * N, s.red);
  // homogenised stress: mean over elements of the element-averaged stress
  double sg[3] = {0.0, 0.0, 0.0};
  for (int e = threadIdx.x; e < N; e += blockDim.x) {
    const int i0 = e >> j.lg1, i1 = e & (j.n1 - 1);
    double u[2][4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int nd = cnode(j, i0 + (c >> 1), i1 + (c & 1));
      u[0][c] = s.x[nd];
      u[1][c] = s.x[N + nd];
    }
    double sig[3];
    element_stress<2>(ec, &sh, u, s.E[e], sig);
    sg[0] += sig[0];
    sg[1] += sig[1];
    sg[2] += sig[2];
  }
  for (int c = 0; c < 3; ++c) sg[c] = cell_sum(sg[c], s.red) / (double)N;
  const int64_t slot = (int64_t)cell * j.n_loads + load;
  if (j.u) {
    double* uo = j.u + slot * 2 * N;
    for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) uo[i] = s.x[i];
  }
  if (threadIdx.x == 0) {
    if (j.chom)
      for (int c = 0; c < 3; ++c) j.chom[((int64_t)cell * 3 + c) * j.n_loads + load] = sg[c];
    if (j.iters) j.iters[slot] = iters;
    if (j.rel_res) j.rel_res[slot] = ff > 0.0 ? sqrt(rt / ff) : 0.0;
    j.status[slot] = done;
  }
}

}  // namespace

size_t cells_smem_bytes(int N, int n0, int n1) {
  return (size_t)(2 * N + n0 + n1) * sizeof(double2) + (size_t)(15 * N + 4) * sizeof(double);
}

cudaError_t launch_cells(int n0, int n1, int n_cells, int n_loads, int kind, double e_max, double exponent,
                         const double* field, const double* e_min, const ElemConst* ec, const double* jscale,
                         const StrainShift* shifts, double tol, int stop_mode, int max_iter, int pc, double void_js,
                         double* u, double* chom, int* iters, double* rel_res, int* status, cudaStream_t st) {
  CellJob j;
  j.n0 = n0;
  j.n1 = n1;
  j.lg0 = 0;
  while ((1 << j.lg0) < n0) ++j.lg0;
  j.lg1 = 0;
  while ((1 << j.lg1) < n1) ++j.lg1;
  j.N = n0 * n1;
  j.n_loads = n_loads;
  j.kind = kind;
  j.e_max = e_max;
  j.exponent = exponent;
  j.field = field;
  j.e_min = e_min;
  j.ec = ec;
  j.jscale = jscale;
  j.shifts = shifts;
  j.tol = tol;
  j.stop_mode = stop_mode;
  j.max_iter = max_iter;
  j.pc = pc;
  j.void_js = void_js;
  j.u = u;
  j.chom = chom;
  j.iters = iters;
  j.rel_res = rel_res;
  j.status = status;
  const size_t smem = cells_smem_bytes(j.N, n0, n1);
  cudaError_t e = allow_dynamic_smem(k_cells, smem);
  if (e != cudaSuccess) return e;
  JFFT_K("cells", st, k_cells<<<n_cells * n_loads, 256, smem, st>>>(j));
  return cudaGetLastError();
}

}  // namespace jfft
