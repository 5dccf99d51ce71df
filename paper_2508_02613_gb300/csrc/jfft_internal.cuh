// Internal declarations of the J-FFT CUDA library: device helpers, element
// constants and the kernel launchers shared by the translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

namespace jfft {

// ---------------------------------------------------------------- basics
template <typename T> struct c2;
template <> struct c2<double> { using t = double2; };
template <> struct c2<float> { using t = float2; };
template <typename T> using cplx = typename c2<T>::t;

template <typename T> __host__ __device__ __forceinline__ cplx<T> mk(T x, T y) { cplx<T> r; r.x = x; r.y = y; return r; }

constexpr int kMaxDim = 3;
constexpr int kMaxLoads = 64;

// Launch geometry of one grid, shared by every kernel.
struct Grid {
  int d;            // 2 or 3
  int n[3];         // nodal points per axis (n[d-1] is the contiguous axis)
  int log2n[3];
  int64_t N;        // product of n
  int M;            // n[d-1] / 2, half length of the real axis
  int64_t F;        // number of half-spectrum frequencies: N / n[d-1] * (M + 1)
  // Launch-shape choices (0 = the built-in default; set by the plan-time autotuner):
  // [0] node rows per warp segment of the 2D operator, [1] planes per segment of the 3D
  // FP32 operator, [2] / [3] divisor of the lines per block of the forward row pass /
  // inverse column pass of the FFT.
  int tune[4];
};

// Element constants of the Q1 operator in Walsh-Hadamard mode form.
//
// Per element, each displacement component X_a is expanded in the 2^d corner
// modes W_a[m] = sum_o prod_{b in m} (2 o_b - 1) u_a(o) (m a bit set over axes,
// axis 0 = highest bit). With the full 2^d Gauss rule, distinct monomials of the
// local coordinates are orthogonal, so the element energy splits by monomial mu
// (a set of axes, |mu| < d) with weight vol * 3^-|mu|. The mode forces are linear
// in the modes; the tables below hold those coefficients for unit E:
//   normal  F_a[mu+a] += nrm[k][a][b] W_b[mu+b]           (a, b not in mu)
//   shear   F_a[mu+b] += shr[k][b][b] W_a[mu+b] + shr[k][a][b] W_b[mu+a]  (a != b not in mu)
//   locked  F_c[mu+a] += shr[k][a][a] W_c[mu+a]            (a not in mu, c in mu)
// with k = |mu|, gs_a = (2 / h_a) / 2^d, kappa_k = vol 3^-k,
//   nrm[k][a][b] = (a == b ? lambda + 2 mu : lambda) kappa_k gs_a gs_b,
//   shr[k][a][b] = mu kappa_k gs_a gs_b.
// Nodal forces are the inverse transform of F times E_e.
template <typename T> struct ElemConstT {
  T nrm[3][3][3];
  T shr[3][3][3];
  T gs[3];       // (2 / h_a) / 2^d: mode -> displacement-gradient factor
  T lam, mu;     // Lame constants of the unit material
  T vol;         // element volume
  int elem;      // voxel discretisation: 0 = Q1 (full Gauss rule), 1 = two P1 triangles (2D)
};
using ElemConst = ElemConstT<double>;

// The same constants rounded to another working precision.
template <typename T> inline ElemConstT<T> elem_const_as(const ElemConst& e) {
  ElemConstT<T> o;
  for (int k = 0; k < 3; ++k)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        o.nrm[k][a][b] = (T)e.nrm[k][a][b];
        o.shr[k][a][b] = (T)e.shr[k][a][b];
      }
  for (int a = 0; a < 3; ++a) o.gs[a] = (T)e.gs[a];
  o.lam = (T)e.lam;
  o.mu = (T)e.mu;
  o.vol = (T)e.vol;
  o.elem = e.elem;
  return o;
}

// Macroscopic strain of one load case expressed as a shift of the single-axis
// modes: W_a[{b}] += shift[a][b] turns B u into eps_bar + B u at every Gauss point.
struct StrainShift {
  double s[kMaxDim][kMaxDim];
};

// PCG scalars of one right-hand side, resident on the device.
struct CgState {
  double gamma;     // r . z
  double alpha, beta;
  double rr;        // ||r||^2
  double ff;        // ||f||^2
  double rr_stop;   // threshold on rr
  int iters;
  int done;         // 0 running, 1 converged, 2 max_iter reached, 3 breakdown
  int max_iter;
  int pad;
};

enum CgDone { kRunning = 0, kConverged = 1, kNoConv = 2, kBreakdown = 3 };

// Raises a kernel's dynamic shared-memory limit to the largest value the device allows
// for it (opt-in maximum minus the kernel's static shared memory). Every caller sets the
// same value, so launches from several host threads cannot lower the limit under one
// another. cudaErrorInvalidValue if `bytes` exceeds that limit.
template <typename K> inline cudaError_t allow_dynamic_smem(K* kern, size_t bytes) {
  int dev = 0, mx = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa = {};
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  const size_t lim = (size_t)mx > fa.sharedSizeBytes ? (size_t)mx - fa.sharedSizeBytes : 0;
  if (bytes > lim) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
}

// Reduction buffers: partial sums per (row, block), reduced in a fixed order.
constexpr int kMaxPartials = 1 << 17;

// A scalar stage fused into the kernel that produces its partial sums: the last
// block to finish (per right-hand side, found with an atomic counter) reduces the
// partials in a fixed order and applies the stage to CgState. stage < 0: none.
struct StageCtl {
  int stage;
  int stop_mode;
  int max_iter;
  double tol;
  unsigned* cnt;     // per-rhs arrival counters, zero between uses
};
inline StageCtl no_stage() { return StageCtl{-1, 0, 0, 0.0, nullptr}; }

// Every kernel launch is bracketed by these hooks (launch counting and optional
// CUDA-event timing per kernel name); implemented by the API layer.
void hook_begin(const char* name, cudaStream_t st);
void hook_end(const char* name, cudaStream_t st);
#define JFFT_K(name, st, ...) \
  do { ::jfft::hook_begin(name, st); __VA_ARGS__; ::jfft::hook_end(name, st); } while (0)

// ---------------------------------------------------------------- launchers
// All launchers enqueue on `st` and return cudaGetLastError(). `nparts` receives
// the number of partial sums written per row.

// S1: E[i] = e_min + (e_max - e_min) field[i]^expo (kind 1) or E = field (kind 0).
// fine[I] = coarse[pixel of I], pixel index i_a >> shift[a] (geometry G_p on T_n).
cudaError_t launch_upsample(const Grid& g, const int* shift, const double* coarse, double* fine, cudaStream_t st);
cudaError_t launch_material(const double* field, double* E, int64_t N, int kind, double e_min, double e_max,
                            double expo, cudaStream_t st);

// bad += number of entries of f that are negative or not finite.
cudaError_t launch_check_field(const double* f, int64_t N, int* bad, cudaStream_t st);

// S2 / S3: y_b = sgn * B^T W C_e (shift_b + B x_b) for b in [0, nb). x == NULL: pure
// macro-strain load; E == NULL: uniform modulus e_uniform; shifts == NULL: no shift.
// dot_mode 1: partial[b][blk] = sum x.y ; 2: sum y.y ; 0: none. Rhs b is skipped
// when cg != NULL and cg[b].done.
cudaError_t launch_apply_K(const Grid& g, const ElemConst& ec, const double* E, double e_uniform, const double* x,
                           double* y, int nb, int64_t field_stride, const StrainShift* shifts, double sgn, int dot_mode,
                           double* partial, int* nparts, CgState* cg, cudaStream_t st, StageCtl sc = no_stage());

// S3, one rhs, with a caller-supplied partial buffer of `cap` entries (see operator.cu);
// nparts = -1 (nothing launched) if the launch would need more than `cap` partials.
// Returns the launch's own status (cudaLaunchKernelEx), never a pending earlier error.
cudaError_t launch_apply_K_dot_capped(const Grid& g, const ElemConst& ec, const double* E, const double* x, double* y,
                                      double* partial, int cap, int* nparts, cudaStream_t st);

// FP32 operator for the mixed-precision inner solve (no strain shift).
cudaError_t launch_apply_K_f32(const Grid& g, const ElemConst& ec, const float* E, const float* x, float* y, int nb,
                               int64_t field_stride, int dot_mode, double* partial, int* nparts, CgState* cg,
                               cudaStream_t st, StageCtl sc = no_stage());
// The same with E stored in BF16 (E16: N __nv_bfloat16 values), converted to FP32 on load.
cudaError_t launch_apply_K_f32_bf16(const Grid& g, const ElemConst& ec, const void* E16, const float* x, float* y,
                                    int nb, int64_t field_stride, int dot_mode, double* partial, int* nparts,
                                    CgState* cg, cudaStream_t st, StageCtl sc = no_stage());
// E16 = E rounded to BF16 (round to nearest even), n values.
cudaError_t launch_to_bf16(const double* E, void* E16, int64_t n, cudaStream_t st);

// S8: element-averaged Mandel stress [nb][d*][N] (stress may be NULL) and partial
// sums of vol * stress in partial[(b d* + s) * kMaxPartials + blk].
cudaError_t launch_stress(const Grid& g, const ElemConst& ec, const double* E, const double* u, int nb,
                          const StrainShift* shifts, double* stress, double* partial, int* nparts, cudaStream_t st);

// S5: esum[I] = sum of E over the 2^d voxels at node I.
cudaError_t launch_node_esum(const Grid& g, const double* E, double* esum, cudaStream_t st);
// Resolved J^1/2 table, comps x N entries: entry (a, i) = ka[a] s^-1/2 for the diagonal
// factor s = src[a src_cs + i] > 0, void_js where s = 0; FP64 into js and / or FP32
// into js32 (either may be NULL).
cudaError_t launch_jacobi_half(const double* src, int64_t src_cs, const double* ka, double void_js, int comps,
                               int64_t N, double* js, float* js32, cudaStream_t st);
// P1 voxels: diag[a][I] = sum over the 4 voxels around node I of E * kappa_o(a), o the
// corner of that voxel at I (kappa4: [4 corners][2 components], corner c = o0 * 2 + o1).
cudaError_t launch_diag_p1(const Grid& g, const double* E, const double* kappa4, double* diag, cudaStream_t st);
// diag[a][I] = kappa[a] * esum[I]
cudaError_t launch_diag_closed(const Grid& g, const double* esum, const double* kappa3, double* diag, cudaStream_t st);
// Alg. 2 helpers: comb field of one component / offset pattern, and extraction.
cudaError_t launch_fill_comb(const Grid& g, int comp, int offbits, double* x, cudaStream_t st);
cudaError_t launch_extract_comb(const Grid& g, int comp, int offbits, const double* y, double* diag, cudaStream_t st);
// S9 (Alg. 1): d unit-impulse fields [d][d][N]; block inversion into the table.
cudaError_t launch_impulses(const Grid& g, double* x, cudaStream_t st);
// Steps 2-3 of Alg. 1 from the impulse responses R [d][fstride] (field alpha = the
// response to the unit impulse in component alpha at node 0; component beta at
// offset beta * N): transform over the 3^d-node support, inversion, table of G_hat.
cudaError_t launch_green_table(const Grid& g, const double* R, int64_t fstride, double* G, double scale_store,
                               cudaStream_t st);
cudaError_t launch_green_export(const Grid& g, const double* G, double* out, double scale_store, cudaStream_t st);

// S6: twiddle table exp(-2 pi i m / n), m < n.
// First-stage radix of the FP64 FFT engine; the fused-form stage table of a line of
// length L > kFftRadix64 holds L - kFftRadix64 entries (launch_lf_table builds it).
constexpr int kFftRadix64 = 8;
cudaError_t launch_lf_table(double2* dst, int L, cudaStream_t st);
cudaError_t launch_twiddles(double2* tw, int n, cudaStream_t st);

template <typename R> struct FftPlanT {
  const cplx<R>* tw[3];
  // FP64: the fused-form stage tables of the lines along axis a (complex length n_a;
  // the last axis: its half length, the real passes' line), NULL where unused
  const cplx<R>* lf[3];
  cplx<R>* T;        // spectrum buffer (real-axis pass output)
  cplx<R>* U;        // second spectrum buffer (3D)
  const R* G;        // stored symbol table [F][d*]
};
using FftPlan = FftPlanT<double>;

// S5 + S6: z_b = M^-1 r_b (Green, or Green-Jacobi when jacobi), with the partial
// sums of r.z. js: the resolved J^1/2 table, factor of DOF (a, node) at js[a jcs + node].
cudaError_t launch_green_precond(const Grid& g, const FftPlan& p, const double* r, double* z, int nb,
                                 int64_t field_stride, const double* js, bool jacobi, double* partial, int* nparts,
                                 CgState* cg, cudaStream_t st, StageCtl sc = no_stage(), int64_t jcs = 0);
// The same in FP32 (mixed-precision inner solve).
cudaError_t launch_green_precond_f32(const Grid& g, const FftPlanT<float>& p, const float* r, float* z, int nb,
                                     const float* js, bool jacobi, double* partial, int* nparts, CgState* cg,
                                     cudaStream_t st, StageCtl sc = no_stage(), int64_t jcs = 0);
// The Green / Green-Jacobi preconditioner with the PCG update fused into its first pass:
// x += alpha p, r -= alpha q (alpha read from cg), the residual stage sc_rr applied by
// that pass's last block per right-hand side, then z = M^-1 r with the r.z partials and
// the stage sc as above. Defined for T = double and float.
template <typename T>
cudaError_t launch_green_precond_xr(const Grid& g, const FftPlanT<T>& p, T* x, T* r, const T* pv, const T* q, T* z,
                                    int nb, const T* js, bool jacobi, double* partial, int* nparts, CgState* cg,
                                    cudaStream_t st, StageCtl sc_rr, StageCtl sc, int64_t jcs);
// z = J r (J = diag(K)^-1 with the void rule) or z = r (identity), partial r.z.
cudaError_t launch_jacobi_precond(const Grid& g, const double* r, double* z, int nb, int64_t stride, const double* js,
                                  bool identity, double* partial, int* nparts, CgState* cg, cudaStream_t st,
                                  StageCtl sc = no_stage(), int64_t jcs = 0);

// S4: CG vector updates and inner products (T = double or float; scalars in FP64).
template <typename T>
cudaError_t launch_cg_xr(const Grid& g, T* x, T* r, const T* p, const T* q, int nb, int64_t stride, CgState* cg,
                         double* partial, int* nparts, cudaStream_t st, StageCtl sc = no_stage());
template <typename T>
cudaError_t launch_cg_p(const Grid& g, T* p, const T* z, int nb, int64_t stride, CgState* cg, cudaStream_t st);
template <typename T>
cudaError_t launch_dot(const Grid& g, const T* a, const T* c, int nb, int64_t stride, double* partial, int* nparts,
                       cudaStream_t st, CgState* cg = nullptr, StageCtl sc = no_stage());
// FP32 variant of the Jacobi / identity preconditioner.
cudaError_t launch_jacobi_precond_f32(const Grid& g, const float* r, float* z, int nb, int64_t stride, const float* js,
                                      bool identity, double* partial, int* nparts, CgState* cg, cudaStream_t st,
                                      StageCtl sc = no_stage(), int64_t jcs = 0);
// Precision conversions for the refinement loop: dst = (float) src per rhs, zeroed
// where active[b] == 0; u += (double) d; r = f - q with partial sums of r.r.
cudaError_t launch_to_f32(const double* src, float* dst, int64_t n_per_rhs, int nb, const int* active, cudaStream_t st);
cudaError_t launch_add_f32(double* u, const float* d, int64_t n, cudaStream_t st);
cudaError_t launch_sub_norm(const Grid& g, const double* f, const double* q, double* r, int nb, double* partial,
                            int* nparts, cudaStream_t st);
// S4 / S7: scalar stages, one block per rhs.
// Condition kernel of the device-side PCG loop (graph WHILE node): chunks[0] += 1,
// condition = (any cg[b].done == running) && chunks[0] < cap.
cudaError_t launch_cg_continue(const CgState* cg, int nb, int* chunks, int cap, cudaGraphConditionalHandle cond,
                               cudaStream_t st);

// Small cells (2D, n0, n1 powers of two in [4, 32], FP64): one CTA per (cell, load)
// runs the whole solve in shared memory. Arrays: field [n_cells][N], e_min, ec,
// jscale [n_cells][2], shifts [n_loads]; outputs u [n_cells][n_loads][2][N] (may be
// NULL), chom [n_cells][3][n_loads], iters / rel_res / status [n_cells][n_loads].
size_t cells_smem_bytes(int N, int n0, int n1);
cudaError_t launch_cells(int n0, int n1, int n_cells, int n_loads, int kind, double e_max, double exponent,
                         const double* field, const double* e_min, const ElemConst* ec, const double* jscale,
                         const StrainShift* shifts, double tol, int stop_mode, int max_iter, int pc, double void_js,
                         double* u, double* chom, int* iters, double* rel_res, int* status, cudaStream_t st);

enum ScalarStage {
  kStageInitFF = 0,
  kStageInitGamma = 1,
  kStageAlpha = 2,
  kStageRR = 3,
  kStageBeta = 4,
  kStageInitFFKeep = 5,  // kStageInitFF that keeps gamma (a continued recurrence)
  kStageReplace = 6      // first r.z after the residual was replaced: beta = v / gamma, gamma = v
};
cudaError_t launch_cg_scalars(int stage, CgState* cg, const double* partial, int nparts, int nb, double tol,
                              int stop_mode, int max_iter, cudaStream_t st, const int* keep = nullptr);
// Per right-hand side, partial sums of (r64 - r32)^2 (rows of kMaxPartials).
cudaError_t launch_gap(const Grid& g, const double* r64, const float* r32, int nb, double* partial, int* nparts,
                       cudaStream_t st);
// out[row] = sum_j partial[row * pstride + j] in a fixed order.
cudaError_t launch_reduce_partials(const double* partial, int nparts, int rows, int64_t pstride, double* out,
                                   cudaStream_t st);
// The same, returning the launch's own status (cudaLaunchKernelEx) without reading
// or clearing an error left pending by earlier work.
cudaError_t launch_reduce_partials_own_status(const double* partial, int nparts, int rows, int64_t pstride,
                                              double* out, cudaStream_t st);
// Row sums of x viewed as [rows][n] into partials; x[row][:] -= sums[row] / n.
cudaError_t launch_row_sums(const double* x, int rows, int64_t n, double* partial, int* nparts, cudaStream_t st);
cudaError_t launch_sub_mean(double* x, int rows, int64_t n, const double* sums, cudaStream_t st);
cudaError_t launch_fill(double* x, int64_t n, double v, cudaStream_t st);

}  // namespace jfft
