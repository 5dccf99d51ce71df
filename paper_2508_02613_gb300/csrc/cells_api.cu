// C ABI of the small-cell batch solver (include/jfft.h, jfft_cells_*): many 2D
// cells of one small grid, each with its own material field, Poisson ratio and
// lower Young's modulus, solved for the same macroscopic strains in one launch.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "element.cuh"
#include "jfft.h"
#include "jfft_internal.cuh"

using namespace jfft;

struct jfft_cells {
  int n0 = 0, n1 = 0, N = 0;
  int max_cells = 0, max_loads = 0;
  jfft_options opt = {};
  cudaStream_t st = nullptr;
  bool own_stream = false;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<void*> allocs;
  double *field = nullptr, *e_min = nullptr, *jscale = nullptr, *u = nullptr, *chom = nullptr, *rel = nullptr;
  ElemConst* ec = nullptr;
  StrainShift* shifts = nullptr;
  int *iters = nullptr, *status = nullptr, *bad = nullptr;
  int64_t launches = 0;
  std::string err;
};

static thread_local std::string g_cells_create_err;

static jfft_status cfail(jfft_cells* h, jfft_status s, const std::string& m) {
  if (h) h->err = m;
  return s;
}
static jfft_status ccuda(jfft_cells* h, cudaError_t e, const char* where) {
  return cfail(h, JFFT_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define CCK(call)                                          \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return ccuda(h, e_, #call);     \
  } while (0)

static void cells_free(jfft_cells* h) {
  if (!h) return;
  cudaSetDevice(h->opt.device);
  if (h->st) cudaStreamSynchronize(h->st);
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->own_stream) {
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    cudaStreamDestroy(h->st);
    h->st = nullptr;
    h->own_stream = false;
  }
}

static bool pow2_in(int64_t v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

extern "C" jfft_status jfft_cells_create(jfft_cells** out, const jfft_grid* grid, int max_cells,
                                         const jfft_options* opt) {
  if (!out) return JFFT_ERR_ARG;
  *out = nullptr;
  g_cells_create_err.clear();
  auto bad = [&](jfft_status s, const char* m) { g_cells_create_err = m; return s; };
  if (!grid) return bad(JFFT_ERR_ARG, "grid is NULL");
  if (grid->dim != 2) return bad(JFFT_ERR_UNSUPPORTED, "small-cell batches are 2D");
  if (!pow2_in(grid->n[0], 4, 32) || !pow2_in(grid->n[1], 4, 32))
    return bad(JFFT_ERR_UNSUPPORTED, "small-cell grids need n0, n1 powers of two in [4, 32]");
  if (max_cells < 1) return bad(JFFT_ERR_ARG, "max_cells must be >= 1");
  jfft_options o;
  jfft_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != JFFT_PREC_FP64) return bad(JFFT_ERR_UNSUPPORTED, "small-cell batches run in FP64");
  if (o.max_iter < 1 || o.max_loads < 1 || o.max_loads > kMaxLoads) return bad(JFFT_ERR_ARG, "bad max_iter or max_loads");
  if (!(o.void_value > 0.0) || !std::isfinite(o.void_value)) return bad(JFFT_ERR_ARG, "void_value must be finite and > 0");
  jfft_cells* h = new jfft_cells();
  h->n0 = (int)grid->n[0];
  h->n1 = (int)grid->n[1];
  h->N = h->n0 * h->n1;
  h->max_cells = max_cells;
  h->max_loads = o.max_loads;
  h->opt = o;
  auto bail = [&](jfft_status s) {
    g_cells_create_err = h->err.empty() ? jfft_status_string(s) : h->err;
    cells_free(h);
    delete h;
    return s;
  };
  cudaError_t e = cudaSetDevice(o.device);
  if (e != cudaSuccess) return bail(ccuda(h, e, "cudaSetDevice"));
  h->st = (cudaStream_t)o.stream;
  if (!h->st) {
    e = cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(ccuda(h, e, "cudaStreamCreateWithFlags"));
    h->own_stream = true;
    e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(ccuda(h, e, "cudaEventCreateWithFlags"));
  }
  const size_t smem = cells_smem_bytes(h->N, h->n0, h->n1);
  int dev_smem = 0;
  cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, o.device);
  if (smem > (size_t)dev_smem) return bail(cfail(h, JFFT_ERR_UNSUPPORTED, "cell does not fit one block's shared memory"));
  const size_t mc = (size_t)max_cells, ml = (size_t)o.max_loads, N = (size_t)h->N;
  struct A { void** p; size_t bytes; } list[] = {
      {(void**)&h->field, mc * N * sizeof(double)},       {(void**)&h->e_min, mc * sizeof(double)},
      {(void**)&h->jscale, 2 * mc * sizeof(double)},      {(void**)&h->ec, mc * sizeof(ElemConst)},
      {(void**)&h->shifts, ml * sizeof(StrainShift)},     {(void**)&h->u, mc * ml * 2 * N * sizeof(double)},
      {(void**)&h->chom, mc * 3 * ml * sizeof(double)},   {(void**)&h->rel, mc * ml * sizeof(double)},
      {(void**)&h->iters, mc * ml * sizeof(int)},         {(void**)&h->status, mc * ml * sizeof(int)},
      {(void**)&h->bad, sizeof(int)}};
  size_t total = 0;
  for (auto& a : list) total += a.bytes;
  if (o.hbm_budget && total > o.hbm_budget) return bail(cfail(h, JFFT_ERR_OOM, "workspace exceeds hbm_budget"));
  for (auto& a : list) {
    e = cudaMalloc(a.p, a.bytes);
    if (e != cudaSuccess) return bail(cfail(h, JFFT_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e)));
    h->allocs.push_back(*a.p);
  }
  *out = h;
  return JFFT_OK;
}

extern "C" void jfft_cells_destroy(jfft_cells* h) {
  if (!h) return;
  cells_free(h);
  delete h;
}

extern "C" const char* jfft_cells_last_error(const jfft_cells* h) {
  return h ? h->err.c_str() : g_cells_create_err.c_str();
}

extern "C" jfft_status jfft_cells_solve(jfft_cells* h, int n_cells, const jfft_material* mat, const double* nu_cells,
                                        const double* e_min_cells, int n_loads, const double* eps_bar, double tol,
                                        jfft_precond pc, jfft_result* res) {
  if (!h) return JFFT_ERR_ARG;
  if (!mat || !mat->field || !eps_bar || !res) return cfail(h, JFFT_ERR_ARG, "NULL material, strains or result");
  if (n_cells < 1 || n_cells > h->max_cells) return cfail(h, JFFT_ERR_ARG, "n_cells outside [1, max_cells]");
  if (n_loads < 1 || n_loads > h->max_loads) return cfail(h, JFFT_ERR_ARG, "n_loads outside [1, max_loads]");
  if (pc != JFFT_PC_GREEN && pc != JFFT_PC_GREEN_JACOBI)
    return cfail(h, JFFT_ERR_UNSUPPORTED, "small-cell batches run the Green or Green-Jacobi preconditioner");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return cfail(h, JFFT_ERR_ARG, "tol must be finite and >= 0");
  if (mat->kind != JFFT_MAT_YOUNG && mat->kind != JFFT_MAT_DENSITY) return cfail(h, JFFT_ERR_ARG, "unknown material kind");
  if (mat->kind == JFFT_MAT_DENSITY &&
      (!(mat->exponent > 0.0) || !std::isfinite(mat->exponent) || !std::isfinite(mat->e_max)))
    return cfail(h, JFFT_ERR_ARG, "density map needs a finite e_max and exponent > 0");
  cudaSetDevice(h->opt.device);
  const bool dev_io = h->opt.io_memory == JFFT_MEM_DEVICE;
  const int N = h->N;
  // per-cell constants (host)
  std::vector<ElemConst> ec(n_cells);
  std::vector<double> js(2 * n_cells), emin(n_cells);
  const double hh[2] = {1.0 / h->n0, 1.0 / h->n1};
  for (int c = 0; c < n_cells; ++c) {
    const double nu = nu_cells ? nu_cells[c] : mat->nu;
    if (!(nu > -1.0 && nu < 0.5)) return cfail(h, JFFT_ERR_ARG, "Poisson ratio must lie in (-1, 0.5)");
    emin[c] = e_min_cells ? e_min_cells[c] : mat->e_min;
    if (mat->kind == JFFT_MAT_DENSITY && !(emin[c] >= 0.0 && emin[c] <= mat->e_max))
      return cfail(h, JFFT_ERR_ARG, "density map needs 0 <= e_min <= e_max");
    ec[c] = make_elem_const(2, hh, nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), 1.0 / (2.0 * (1.0 + nu)));
    for (int a = 0; a < 2; ++a) {
      double u[2][4] = {};
      u[a][0] = 1.0;
      element_force<2, double, false>(ec[c], nullptr, u, 1.0);
      js[2 * c + a] = 1.0 / std::sqrt(u[a][0]);
    }
  }
  std::vector<StrainShift> sh(n_loads);
  for (int b = 0; b < n_loads; ++b) {
    for (int k = 0; k < 3; ++k)
      if (!std::isfinite(eps_bar[b * 3 + k])) return cfail(h, JFFT_ERR_ARG, "non-finite macroscopic strain");
    sh[b] = make_shift(2, ec[0], eps_bar + b * 3);
  }
  if (!dev_io) {
    for (int64_t i = 0; i < (int64_t)n_cells * N; ++i) {
      const double v = mat->field[i];
      if (!std::isfinite(v) || v < 0.0) return cfail(h, JFFT_ERR_ARG, "material field must be finite and >= 0");
    }
  }
  if (h->own_stream) {
    cudaEventRecord(h->ev_in, cudaStreamLegacy);
    cudaStreamWaitEvent(h->st, h->ev_in, 0);
  }
  const cudaMemcpyKind in_kind = dev_io ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CCK(cudaMemcpyAsync(h->field, mat->field, (size_t)n_cells * N * sizeof(double), in_kind, h->st));
  CCK(cudaMemcpyAsync(h->ec, ec.data(), n_cells * sizeof(ElemConst), cudaMemcpyHostToDevice, h->st));
  CCK(cudaMemcpyAsync(h->jscale, js.data(), 2 * n_cells * sizeof(double), cudaMemcpyHostToDevice, h->st));
  CCK(cudaMemcpyAsync(h->e_min, emin.data(), n_cells * sizeof(double), cudaMemcpyHostToDevice, h->st));
  CCK(cudaMemcpyAsync(h->shifts, sh.data(), n_loads * sizeof(StrainShift), cudaMemcpyHostToDevice, h->st));
  if (dev_io) {
    int bad_h = 0;
    CCK(cudaMemsetAsync(h->bad, 0, sizeof(int), h->st));
    CCK(launch_check_field(h->field, (int64_t)n_cells * N, h->bad, h->st));
    CCK(cudaMemcpyAsync(&bad_h, h->bad, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CCK(cudaStreamSynchronize(h->st));
    if (bad_h) return cfail(h, JFFT_ERR_ARG, "material field must be finite and >= 0");
  }
  CCK(launch_cells(h->n0, h->n1, n_cells, n_loads, mat->kind, mat->e_max, mat->exponent, h->field, h->e_min, h->ec,
                   h->jscale, h->shifts, tol, h->opt.stop_mode, h->opt.max_iter, (int)pc, 1.0 / std::sqrt(h->opt.void_value),
                   res->u ? h->u : nullptr, h->chom, h->iters, h->rel, h->status, h->st));
  h->launches += 1;
  const size_t slots = (size_t)n_cells * n_loads;
  const cudaMemcpyKind out_kind = dev_io ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (res->u) CCK(cudaMemcpyAsync(res->u, h->u, slots * 2 * N * sizeof(double), out_kind, h->st));
  if (res->C_hom) CCK(cudaMemcpyAsync(res->C_hom, h->chom, (size_t)n_cells * 3 * n_loads * sizeof(double), out_kind, h->st));
  if (res->iters) CCK(cudaMemcpyAsync(res->iters, h->iters, slots * sizeof(int), out_kind, h->st));
  if (res->rel_res) CCK(cudaMemcpyAsync(res->rel_res, h->rel, slots * sizeof(double), out_kind, h->st));
  std::vector<int> status(slots);
  CCK(cudaMemcpyAsync(status.data(), h->status, slots * sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CCK(cudaStreamSynchronize(h->st));
  if (h->own_stream) {
    cudaEventRecord(h->ev_out, h->st);
    cudaStreamWaitEvent(cudaStreamLegacy, h->ev_out, 0);
  }
  int worst = kConverged;
  for (int v : status) {
    if (v == kBreakdown) worst = kBreakdown;
    else if (v == kNoConv && worst != kBreakdown) worst = kNoConv;
  }
  if (worst == kBreakdown) return cfail(h, JFFT_ERR_BREAKDOWN, "PCG breakdown in at least one cell");
  if (worst == kNoConv) return cfail(h, JFFT_ERR_NOCONV, "at least one cell reached max_iter");
  return JFFT_OK;
}

extern "C" int64_t jfft_cells_launch_count(const jfft_cells* h) { return h ? h->launches : 0; }
