// C ABI of the J-FFT solver (include/jfft.h): handle lifecycle, device workspace,
// setup (material S1, Jacobi S5, Green symbol S9 by Alg. 1 on the device), the PCG
// driver (S2-S7) and post-processing (S8).
#include "jfft.h"
#include "element.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

using namespace jfft;

struct jfft_solver {
  int device = 0;
  cudaStream_t st = nullptr;
  Grid g = {};
  int ds = 3;
  jfft_options opt = {};
  int io = JFFT_MEM_HOST;
  int max_iter = 100000;
  int max_loads = 6;
  double nu = 0.3;
  ElemConst ec = {};      // unit material C_unit(nu)
  ElemConst ec_ref = {};  // reference material C_ref
  bool cref_mean = true;
  double cref_lam = 0.0, cref_mu = 0.0;
  double e_ref = 1.0;
  double kappa[3] = {0, 0, 0}, jscale[3] = {0, 0, 0}, void_js = 1.0;
  int element = 0;                 // JFFT_ELEM_Q1 or JFFT_ELEM_P1
  int64_t jcs = 0;                 // component stride of the resolved J^1/2 table (0: one factor per node)
  double kappa_p1[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // P1: diagonal of the unit voxel, [corner][component]
  double scale_store = 1.0;
  // device workspace
  double *field = nullptr, *E = nullptr, *esum = nullptr, *js = nullptr, *G = nullptr;
  double2* tw[3] = {nullptr, nullptr, nullptr};
  double2* lf[3] = {nullptr, nullptr, nullptr};  // FP64 fused-form FFT stage tables (FftPlanT::lf)
  double2 *T = nullptr, *U = nullptr;
  double *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr;
  double *partial = nullptr, *red = nullptr;
  CgState* cg = nullptr;
  unsigned* stage_cnt = nullptr;  // per-rhs arrival counters of the fused scalar stages
  StrainShift* shifts = nullptr;
  // FP32 copies and vectors of the mixed-precision inner solve
  int precision = JFFT_PREC_FP64;
  float *E32 = nullptr, *js32 = nullptr, *G32 = nullptr;
  void* E16 = nullptr;             // BF16 copy of E (options.material_bf16; E32 is then not allocated)
  float2* tw32[3] = {nullptr, nullptr, nullptr};
  float2 *T32 = nullptr, *U32 = nullptr;
  float *x32 = nullptr, *r32 = nullptr, *p32 = nullptr, *q32 = nullptr, *z32 = nullptr;
  int* active = nullptr;
  int* active_h = nullptr;
  std::vector<void*> allocs;
  // pinned host mirrors
  CgState* cg_h = nullptr;
  double* red_h = nullptr;
  size_t ws_bytes = 0;
  std::string err;
  int64_t launches = 0;
  bool profiling = false;
  struct Pend { const char* name; cudaEvent_t a, b; };
  std::vector<Pend> pend;
  std::vector<cudaEvent_t> pool;
  std::map<std::string, std::pair<int64_t, double>> prof;
  std::string prof_json;
  // own stream (options.stream == NULL), ordered against the legacy default stream
  bool own_stream = false;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // CUDA graph of one check_every-iteration PCG chunk, per working precision
  struct ChunkGraph {
    cudaGraphExec_t exec = nullptr;
    int nb = -1, pc = -1, stop_mode = -1, max_iter = -1, chunk = -1;
    double tol = -1.0;
    int64_t launches = 0;
    bool prof = false;         // captured with per-kernel timing events
    std::vector<Pend> events;  // those events, re-recorded by every replay
  };
  ChunkGraph graph[2];
  ChunkGraph* replayed = nullptr;  // graph whose events the next sync reads
  // CUDA graph of a whole PCG solve: a WHILE node around one chunk, ended on the
  // device when every right-hand side is done (no host polling), per precision
  struct LoopGraph {
    cudaGraphExec_t exec = nullptr;
    int nb = -1, pc = -1, stop_mode = -1, max_iter = -1, chunk = -1;
    double tol = -1.0;
    int64_t launches_per_chunk = 0;
  };
  LoopGraph loop[2];
  bool loop_ok = true;      // cleared if the loop graph cannot be built here
  int* chunks_d = nullptr;  // chunks run by the last device-side loop
  int* chunks_h = nullptr;
  bool graphs_ok = true;  // cleared if a capture fails; kernels are then launched directly
  bool capturing = false;
  int64_t graph_replays = 0;
};

// ------------------------------------------------------------- launch hooks
static thread_local jfft_solver* g_cur = nullptr;
static thread_local std::string g_create_err;  // message of the last failed jfft_create

namespace jfft {
void hook_begin(const char* name, cudaStream_t st) {
  jfft_solver* h = g_cur;
  if (!h) return;
  h->launches++;
  if (!h->profiling) return;
  jfft_solver::Pend pe;
  pe.name = name;
  for (int i = 0; i < 2; ++i) {
    cudaEvent_t ev;
    if (!h->pool.empty()) { ev = h->pool.back(); h->pool.pop_back(); }
    else cudaEventCreate(&ev);
    (i == 0 ? pe.a : pe.b) = ev;
  }
  // inside a graph capture the record must be an event-record node (External),
  // not a capture-internal dependency, so that the replay's timing can be read
  cudaEventRecordWithFlags(pe.a, st, h->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
  h->pend.push_back(pe);
}
void hook_end(const char* /*name*/, cudaStream_t st) {
  jfft_solver* h = g_cur;
  if (!h || !h->profiling || h->pend.empty()) return;
  cudaEventRecordWithFlags(h->pend.back().b, st, h->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
}
}  // namespace jfft

// Per-call scope: selects the solver and device; for a solver on its own stream,
// orders the call after earlier legacy-stream work and later legacy-stream work
// after the call.
struct CurGuard {
  jfft_solver* prev;
  jfft_solver* cur;
  explicit CurGuard(jfft_solver* h) : prev(g_cur), cur(h) {
    g_cur = h;
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->own_stream) {
      cudaEventRecord(h->ev_in, cudaStreamLegacy);
      cudaStreamWaitEvent(h->st, h->ev_in, 0);
    }
  }
  ~CurGuard() {
    if (cur && cur->own_stream) {
      cudaEventRecord(cur->ev_out, cur->st);
      cudaStreamWaitEvent(cudaStreamLegacy, cur->ev_out, 0);
    }
    g_cur = prev;
  }
};

static void accumulate(jfft_solver* h, const jfft_solver::Pend& pe) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, pe.a, pe.b) == cudaSuccess) {
    auto& e = h->prof[pe.name];
    e.first += 1;
    e.second += ms;
  } else {
    cudaGetLastError();  // a timing that cannot be read is dropped, not reported as a failure
  }
}

static void drain_profile(jfft_solver* h) {
  if (h->replayed) {
    for (auto& pe : h->replayed->events) accumulate(h, pe);
    h->replayed = nullptr;
  }
  for (auto& pe : h->pend) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pe.a, pe.b) == cudaSuccess) {
      auto& e = h->prof[pe.name];
      e.first += 1;
      e.second += ms;
    }
    h->pool.push_back(pe.a);
    h->pool.push_back(pe.b);
  }
  h->pend.clear();
}

// ------------------------------------------------------------- helpers
static jfft_status fail(jfft_solver* h, jfft_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

static jfft_status cuda_fail(jfft_solver* h, cudaError_t e, const char* where) {
  return fail(h, JFFT_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

static bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
static int ilog2i(int64_t v) { int l = 0; while ((int64_t(1) << l) < v) ++l; return l; }

static jfft_status sync(jfft_solver* h) {
  CK(cudaStreamSynchronize(h->st));
  CK(cudaGetLastError());
  if (h->profiling) drain_profile(h);
  h->replayed = nullptr;
  return JFFT_OK;
}

// Every CUDA graph capture, instantiation and destruction of the library runs under one
// process-wide lock: solvers driven from several host threads (the request server's
// workers) built and tore down their loop graphs concurrently, and the template graph's
// destruction then crashed inside the driver now and then. Kernel launches and graph
// replays stay concurrent; only the (rare) graph construction and teardown serialise.
static std::recursive_mutex& graph_mutex() {
  static std::recursive_mutex m;
  return m;
}

static void destroy_exec(cudaGraphExec_t& exec) {
  if (!exec) return;
  std::lock_guard<std::recursive_mutex> lock(graph_mutex());
  cudaGraphExecDestroy(exec);
  exec = nullptr;
}

static void drop_graph(jfft_solver* h, jfft_solver::ChunkGraph& gr) {
  destroy_exec(gr.exec);
  gr.exec = nullptr;
  for (auto& pe : gr.events) {
    h->pool.push_back(pe.a);
    h->pool.push_back(pe.b);
  }
  gr.events.clear();
  if (h->replayed == &gr) h->replayed = nullptr;
}

static int64_t field_elems(const jfft_solver* h) { return (int64_t)h->g.d * h->g.N; }

// copy count fields into / out of a device buffer according to the io mode
static jfft_status copy_in(jfft_solver* h, double* dst, const double* src, size_t n) {
  CK(cudaMemcpyAsync(dst, src, n * sizeof(double), h->io == JFFT_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                                              : cudaMemcpyHostToDevice, h->st));
  return JFFT_OK;
}
static jfft_status copy_out(jfft_solver* h, void* dst, const void* src, size_t bytes) {
  CK(cudaMemcpyAsync(dst, src, bytes, h->io == JFFT_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     h->st));
  return JFFT_OK;
}

static void isotropic_mandel(int d, double lam, double mu, double* C) {
  const int ds = d * (d + 1) / 2;
  for (int i = 0; i < ds * ds; ++i) C[i] = 0.0;
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) C[a * ds + b] = lam + (a == b ? 2.0 * mu : 0.0);
  for (int s = d; s < ds; ++s) C[s * ds + s] = 2.0 * mu;
}

// ------------------------------------------------------------- lifecycle
extern "C" void jfft_default_options(jfft_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = JFFT_PREC_FP64;
  o->max_iter = 100000;
  o->stop_mode = JFFT_STOP_REL;
  o->stream = nullptr;
  o->hbm_budget = 0;
  o->check_every = 8;
  o->io_memory = JFFT_MEM_HOST;
  o->max_loads = 6;
  o->void_value = 1.0;
  o->device = 0;
  o->inner_tol = 1e-3;
  o->max_refine = 30;
  o->graphs = 1;
  o->element = JFFT_ELEM_Q1;
  o->autotune = 0;
  o->reliable = 0;
  o->material_bf16 = 0;
}

static jfft_status dalloc(jfft_solver* h, void** ptr, size_t bytes) {
  CK(cudaMalloc(ptr, bytes));
  h->allocs.push_back(*ptr);
  h->ws_bytes += bytes;
  return JFFT_OK;
}

static void free_all(jfft_solver* h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->st) cudaStreamSynchronize(h->st);
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->cg_h) cudaFreeHost(h->cg_h);
  if (h->red_h) cudaFreeHost(h->red_h);
  if (h->active_h) cudaFreeHost(h->active_h);
  h->cg_h = nullptr;
  h->red_h = nullptr;
  h->active_h = nullptr;
  for (auto& gr : h->graph) drop_graph(h, gr);
  for (auto& lg : h->loop) destroy_exec(lg.exec);
  if (h->chunks_h) cudaFreeHost(h->chunks_h);
  h->chunks_h = nullptr;
  for (auto& pe : h->pend) { h->pool.push_back(pe.a); h->pool.push_back(pe.b); }
  for (auto ev : h->pool) cudaEventDestroy(ev);
  h->pool.clear();
  h->pend.clear();
  if (h->own_stream) {
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    cudaStreamDestroy(h->st);
    h->ev_in = h->ev_out = nullptr;
    h->st = nullptr;
    h->own_stream = false;
  }
}

static jfft_status validate_material(jfft_solver* h, const jfft_material* m, int64_t N, bool field_on_device = false) {
  if (!m || !m->field) return fail(h, JFFT_ERR_ARG, "material or material field is NULL");
  if (m->kind != JFFT_MAT_YOUNG && m->kind != JFFT_MAT_DENSITY) return fail(h, JFFT_ERR_ARG, "unknown material kind");
  if (!(m->nu > -1.0 && m->nu < 0.5)) return fail(h, JFFT_ERR_ARG, "Poisson ratio must lie in (-1, 0.5)");
  if (m->kind == JFFT_MAT_DENSITY) {
    if (!(std::isfinite(m->e_min) && std::isfinite(m->e_max) && m->e_min >= 0.0 && m->e_max >= m->e_min))
      return fail(h, JFFT_ERR_ARG, "density material needs finite 0 <= e_min <= e_max");
    if (!(m->exponent > 0.0 && std::isfinite(m->exponent))) return fail(h, JFFT_ERR_ARG, "exponent must be > 0");
  }
  if (field_on_device) return JFFT_OK;  // checked on the device after the copy
  for (int64_t i = 0; i < N; ++i) {
    const double v = m->field[i];
    if (!std::isfinite(v) || v < 0.0) return fail(h, JFFT_ERR_ARG, "material field must be finite and >= 0");
  }
  return JFFT_OK;
}

// Alg. 1 on the device: impulse responses of K_ref, their transform (evaluated over
// the responses' 3^d-node support, free of low-frequency cancellation), inversion.
static jfft_status build_symbol(jfft_solver* h) {
  const Grid& g = h->g;
  CK(launch_impulses(g, h->x, h->st));
  CK(launch_apply_K(g, h->ec_ref, nullptr, 1.0, h->x, h->z, g.d, field_elems(h), nullptr, 1.0, 0, nullptr, nullptr,
                    nullptr, h->st));
  CK(launch_green_table(g, h->z, field_elems(h), h->G, h->scale_store, h->st));
  return JFFT_OK;
}

// Components of the resolved J^1/2 table: one factor per node when every component
// scales alike (Q1 on a grid with equal spacing on every axis), one per DOF otherwise
// (P1 voxels, or Q1 elements that are not cubes).
static int js_components(const Grid& g, int element) {
  if (element == JFFT_ELEM_P1) return g.d;
  for (int a = 1; a < g.d; ++a)
    if (g.n[a] != g.n[0]) return g.d;
  return 1;
}

// Line length of the FFT passes along axis a: n_a, the last axis its half length (the
// real passes' complex line).
static int lf_length(const Grid& g, int a) { return a == g.d - 1 ? g.n[a] / 2 : g.n[a]; }

// Device workspace of a solver (bytes), as allocated by jfft_create.
static size_t plan_bytes(const Grid& g, int ds, int nbmax, int precision, int element = 0, int material_bf16 = 0) {
  const int d = g.d;
  const int64_t fe = (int64_t)d * g.N;
  const int64_t spec_n = (int64_t)nbmax * d * g.F;
  size_t total = 0;
  const int jsn = js_components(g, element);
  total += (3 + jsn) * g.N * sizeof(double);                        // field, E, esum, J^1/2 table
  total += (size_t)g.F * ds * sizeof(double);                       // G
  for (int a = 0; a < d; ++a) total += (size_t)g.n[a] * sizeof(double2);
  for (int a = 0; a < d; ++a)                                       // fused-form stage tables
    if (lf_length(g, a) > kFftRadix64) total += (size_t)(lf_length(g, a) - kFftRadix64) * sizeof(double2);
  total += (size_t)spec_n * sizeof(double2) * (d == 3 ? 2 : 1);     // T (U)
  total += 5 * (size_t)nbmax * fe * sizeof(double);                 // x r p q z
  total += (size_t)nbmax * 6 * kMaxPartials * sizeof(double);       // partial sums
  total += 1024 * sizeof(double) + nbmax * (sizeof(CgState) + sizeof(StrainShift) + sizeof(int) + sizeof(unsigned));
  total += sizeof(int);                                             // chunk counter
  if (precision == JFFT_PREC_MIXED) {
    total += (material_bf16 ? 2 : sizeof(float)) * g.N + jsn * g.N * sizeof(float) + (size_t)g.F * ds * sizeof(float);
    for (int a = 0; a < d; ++a) total += (size_t)g.n[a] * sizeof(float2);
    total += (size_t)spec_n * sizeof(float2) * (d == 3 ? 2 : 1);
    total += 5 * (size_t)nbmax * fe * sizeof(float);
  }
  return total;
}

// Grid of a jfft_grid, or an error message.
static const char* make_grid(const jfft_grid* grid, Grid& g) {
  if (!grid) return "grid is NULL";
  const int d = grid->dim;
  if (d != 2 && d != 3) return "dim must be 2 or 3";
  const int nmax = d == 2 ? 2048 : 1024;
  g = Grid{};
  g.d = d;
  g.N = 1;
  for (int a = 0; a < d; ++a) {
    const int64_t n = grid->n[a];
    if (!is_pow2(n) || n < 4) return "each n must be a power of two >= 4";
    if (n > nmax) return "grid exceeds the largest supported axis length";
    g.n[a] = (int)n;
    g.log2n[a] = ilog2i(n);
    g.N *= n;
  }
  g.M = g.n[d - 1] / 2;
  g.F = g.N / g.n[d - 1] * (g.M + 1);
  return nullptr;
}

// Unit material C_unit(nu) of the operator, and the Jacobi constants derived from it:
// kappa_a = diagonal entry of the unit element matrix for component a (the same at
// every corner), jscale_a = kappa_a^-1/2.
static void set_unit_material(jfft_solver* h, double nu) {
  const Grid& g = h->g;
  const int d = g.d;
  h->nu = nu;
  const double lam_u = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu_u = 1.0 / (2.0 * (1.0 + nu));
  double hh[3];
  for (int a = 0; a < d; ++a) hh[a] = 1.0 / g.n[a];
  h->ec = make_elem_const(d, hh, lam_u, mu_u);
  h->ec.elem = h->element;
  for (int a = 0; a < 3; ++a) h->kappa[a] = 1.0;
  if (h->element == JFFT_ELEM_P1) {
    // corner-dependent diagonal of the two-triangle voxel; the node factors carry it all
    for (int c = 0; c < 4; ++c)
      for (int a = 0; a < 2; ++a) {
        double u[2][4] = {};
        u[a][c] = 1.0;
        tri_pair_force<double, false>(h->ec, nullptr, u, 1.0);
        h->kappa_p1[c * 2 + a] = u[a][c];
      }
    for (int a = 0; a < 3; ++a) h->jscale[a] = 1.0;
    return;
  }
  for (int a = 0; a < d; ++a) {
    if (d == 2) {
      double u[2][4] = {};
      u[a][0] = 1.0;
      element_force<2, double, false>(h->ec, nullptr, u, 1.0);
      h->kappa[a] = u[a][0];
    } else {
      double u[3][8] = {};
      u[a][0] = 1.0;
      element_force<3, double, false>(h->ec, nullptr, u, 1.0);
      h->kappa[a] = u[a][0];
    }
    h->jscale[a] = 1.0 / std::sqrt(h->kappa[a]);
  }
  // On a grid with equal spacing the axes are equivalent and the unit diagonal is the
  // same for every component; the mode form can round it differently per axis, so
  // one value (axis 0's) is kept for all.
  if (js_components(g, h->element) == 1)
    for (int a = 1; a < d; ++a) {
      h->kappa[a] = h->kappa[0];
      h->jscale[a] = h->jscale[0];
    }
}

// coarse: pixels per axis of a geometry G_p (NULL: the field has one value per voxel).
static jfft_status setup_material(jfft_solver* h, const jfft_material* m, bool field_on_device,
                                  const int64_t* coarse = nullptr) {
  const Grid& g = h->g;
  int shift[3] = {0, 0, 0};
  int64_t count = g.N;
  if (coarse) {
    count = 1;
    for (int a = 0; a < g.d; ++a) {
      const int64_t p = coarse[a];
      if (!is_pow2(p) || p > g.n[a]) return fail(h, JFFT_ERR_ARG, "pixels per axis must be powers of two <= n");
      shift[a] = g.log2n[a] - ilog2i(p);
      count *= p;
    }
  }
  jfft_status s = validate_material(h, m, count, field_on_device);
  if (s) return s;
  if (m->nu != h->nu) {
    if (!h->cref_mean) return fail(h, JFFT_ERR_ARG, "the Poisson ratio is fixed when C_ref was given explicitly");
    s = sync(h);
    if (s) return s;
    set_unit_material(h, m->nu);
    // captured graphs hold the element constants and Jacobi scales by value
    for (auto& gr : h->graph) drop_graph(h, gr);
    for (auto& lg : h->loop) destroy_exec(lg.exec);
  }
  // a coarse geometry is staged in the E buffer and expanded into the voxel field
  double* dst = coarse ? h->E : h->field;
  CK(cudaMemcpyAsync(dst, m->field, count * sizeof(double),
                     field_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
  if (coarse) CK(launch_upsample(g, shift, h->E, h->field, h->st));
  if (field_on_device) {
    int* bad = reinterpret_cast<int*>(h->red);
    CK(cudaMemsetAsync(bad, 0, sizeof(int), h->st));
    CK(launch_check_field(h->field, g.N, bad, h->st));
    int bad_h = 0;
    CK(cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    s = sync(h);
    if (s) return s;
    if (bad_h) return fail(h, JFFT_ERR_ARG, "material field must be finite and >= 0");
  }
  CK(launch_material(h->field, h->E, g.N, m->kind, m->e_min, m->e_max, m->exponent, h->st));
  CK(launch_node_esum(g, h->E, h->esum, h->st));
  // resolved J^1/2 table: js[a jcs + node] = diag^-1/2 (void nodes: void_js)
  const double* dsrc = h->esum;
  int64_t dsrc_cs = 0;
  if (h->element == JFFT_ELEM_P1) {
    CK(launch_diag_p1(g, h->E, h->kappa_p1, h->x, h->st));   // x is free outside a solve
    dsrc = h->x;
    dsrc_cs = g.N;
  }
  const int jsn = js_components(g, h->element);
  CK(launch_jacobi_half(dsrc, dsrc_cs, h->jscale, h->void_js, jsn, g.N, h->js,
                        h->precision == JFFT_PREC_MIXED ? h->js32 : nullptr, h->st));
  double lam, mu;
  if (h->cref_mean) {
    int np = 0;
    CK(launch_row_sums(h->E, 1, g.N, h->partial, &np, h->st));
    CK(launch_reduce_partials(h->partial, np, 1, kMaxPartials, h->red, h->st));
    CK(cudaMemcpyAsync(h->red_h, h->red, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    s = sync(h);
    if (s) return s;
    const double mean = h->red_h[0] / (double)g.N;
    if (!(mean > 0.0)) return fail(h, JFFT_ERR_ARG, "mean(E) is zero: the mean reference material is undefined");
    h->e_ref = mean;
    lam = mean * h->ec.lam;
    mu = mean * h->ec.mu;
  } else {
    lam = h->cref_lam;
    mu = h->cref_mu;
  }
  double hh[3];
  for (int a = 0; a < g.d; ++a) hh[a] = 1.0 / g.n[a];
  h->ec_ref = make_elem_const(g.d, hh, lam, mu);
  h->ec_ref.elem = h->element;
  s = build_symbol(h);
  if (s) return s;
  if (h->precision == JFFT_PREC_MIXED) {
    if (h->E16) CK(launch_to_bf16(h->E, h->E16, g.N, h->st));
    else CK(launch_to_f32(h->E, h->E32, g.N, 1, nullptr, h->st));
    CK(launch_to_f32(h->G, h->G32, g.F * h->ds, 1, nullptr, h->st));
    for (int a = 0; a < g.d; ++a)
      CK(launch_to_f32(reinterpret_cast<const double*>(h->tw[a]), reinterpret_cast<float*>(h->tw32[a]), 2 * g.n[a], 1,
                       nullptr, h->st));
  }
  return sync(h);
}

static jfft_status autotune(jfft_solver* h);

extern "C" jfft_status jfft_create(jfft_solver** out, const jfft_grid* grid, const jfft_material* mat,
                                   const double* C_ref, const jfft_options* opt) {
  if (!out) return JFFT_ERR_ARG;
  *out = nullptr;
  jfft_solver* h = new jfft_solver();
  CurGuard guard(nullptr);
  auto bail = [&](jfft_status s) {
    g_create_err = h->err.empty() ? jfft_status_string(s) : h->err;
    free_all(h);
    delete h;
    return s;
  };
  jfft_options o;
  jfft_default_options(&o);
  if (opt) o = *opt;
  h->opt = o;
  Grid& g = h->g;
  if (const char* ge = make_grid(grid, g))
    return bail(fail(h, grid && (grid->dim == 2 || grid->dim == 3) ? JFFT_ERR_UNSUPPORTED : JFFT_ERR_ARG, ge));
  const int d = g.d;
  h->ds = d * (d + 1) / 2;
  if (o.precision != JFFT_PREC_FP64 && o.precision != JFFT_PREC_MIXED)
    return bail(fail(h, JFFT_ERR_ARG, "unknown precision"));
  if (o.precision == JFFT_PREC_MIXED) {
    if (!(o.inner_tol > 0.0 && o.inner_tol < 1.0)) return bail(fail(h, JFFT_ERR_ARG, "inner_tol must lie in (0, 1)"));
    if (o.max_refine <= 0) return bail(fail(h, JFFT_ERR_ARG, "max_refine must be positive"));
  }
  if (o.material_bf16 && o.precision != JFFT_PREC_MIXED)
    return bail(fail(h, JFFT_ERR_ARG, "material_bf16 requires precision MIXED"));
  h->precision = o.precision;
  if (o.max_iter <= 0) return bail(fail(h, JFFT_ERR_ARG, "max_iter must be positive"));
  if (o.stop_mode != JFFT_STOP_REL && o.stop_mode != JFFT_STOP_ABS_SQ) return bail(fail(h, JFFT_ERR_ARG, "bad stop_mode"));
  if (o.check_every <= 0) o.check_every = 8;
  if (o.max_loads <= 0) o.max_loads = 6;
  if (o.max_loads < d) o.max_loads = d;
  if (o.max_loads > kMaxLoads) return bail(fail(h, JFFT_ERR_ARG, "max_loads too large"));
  if (!(o.void_value > 0.0 && std::isfinite(o.void_value))) return bail(fail(h, JFFT_ERR_ARG, "void_value must be > 0"));
  if (o.io_memory != JFFT_MEM_HOST && o.io_memory != JFFT_MEM_DEVICE) return bail(fail(h, JFFT_ERR_ARG, "bad io_memory"));
  h->opt = o;
  h->io = o.io_memory;
  h->max_iter = o.max_iter;
  h->max_loads = o.max_loads;
  h->device = o.device;
  if (!mat) return bail(fail(h, JFFT_ERR_ARG, "material is NULL"));
  h->nu = mat->nu;
  jfft_status s = validate_material(h, mat, g.N);
  if (s) return bail(s);

  if (o.element != JFFT_ELEM_Q1 && o.element != JFFT_ELEM_P1) return bail(fail(h, JFFT_ERR_ARG, "unknown element"));
  if (o.element == JFFT_ELEM_P1 && d != 2) return bail(fail(h, JFFT_ERR_UNSUPPORTED, "P1 triangles are 2D"));
  h->element = o.element;
  h->jcs = js_components(g, h->element) > 1 ? g.N : 0;
  // unit material and reference material
  set_unit_material(h, mat->nu);
  if (C_ref) {
    const int ds = h->ds;
    const double lam = C_ref[1], mu = 0.5 * (C_ref[0] - C_ref[1]);
    double want[36];
    isotropic_mandel(d, lam, mu, want);
    double scale = 0.0;
    for (int i = 0; i < ds * ds; ++i) scale = std::max(scale, std::fabs(want[i]));
    for (int i = 0; i < ds * ds; ++i)
      if (!(std::fabs(C_ref[i] - want[i]) <= 1e-12 * scale))
        return bail(fail(h, JFFT_ERR_UNSUPPORTED, "C_ref must be an isotropic Mandel matrix"));
    if (!(mu > 0.0) || !(lam + 2.0 * mu / d > 0.0))
      return bail(fail(h, JFFT_ERR_ARG, "C_ref must be positive definite"));
    h->cref_mean = false;
    h->cref_lam = lam;
    h->cref_mu = mu;
  }
  h->void_js = 1.0 / std::sqrt(o.void_value);
  h->scale_store = 1.0 / (2.0 * (double)g.N);

  cudaError_t ce = cudaSetDevice(h->device);
  if (ce != cudaSuccess) return bail(cuda_fail(h, ce, "cudaSetDevice"));
  h->st = (cudaStream_t)o.stream;
  if (!h->st) {
    ce = cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return bail(cuda_fail(h, ce, "cudaStreamCreateWithFlags"));
    h->own_stream = true;
    ce = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming);
    if (ce != cudaSuccess) return bail(cuda_fail(h, ce, "cudaEventCreateWithFlags"));
    cudaEventRecord(h->ev_in, cudaStreamLegacy);
    cudaStreamWaitEvent(h->st, h->ev_in, 0);
  }
  g_cur = h;

  // workspace plan
  const int64_t fe = field_elems(h);
  const int nbmax = h->max_loads;
  const int64_t spec_n = (int64_t)nbmax * d * g.F;
  const size_t part_rows = (size_t)nbmax * 6;
  const size_t total = plan_bytes(g, h->ds, nbmax, o.precision, h->element, o.material_bf16);
  if (o.hbm_budget && total > o.hbm_budget) {
    char msg[160];
    snprintf(msg, sizeof msg, "workspace of %zu bytes exceeds hbm_budget %zu", total, o.hbm_budget);
    return bail(fail(h, JFFT_ERR_OOM, msg));
  }
  size_t fr = 0, tot = 0;
  ce = cudaMemGetInfo(&fr, &tot);
  if (ce != cudaSuccess) return bail(cuda_fail(h, ce, "cudaMemGetInfo"));
  if (total > fr) return bail(fail(h, JFFT_ERR_OOM, "workspace does not fit the free device memory"));

#define AL(ptr, bytes) do { jfft_status s_ = dalloc(h, (void**)&(ptr), (bytes)); if (s_) return bail(s_); } while (0)
  AL(h->field, g.N * sizeof(double));
  AL(h->E, g.N * sizeof(double));
  AL(h->esum, g.N * sizeof(double));
  AL(h->js, g.N * sizeof(double) * js_components(g, h->element));
  AL(h->G, (size_t)g.F * h->ds * sizeof(double));
  for (int a = 0; a < d; ++a) AL(h->tw[a], (size_t)g.n[a] * sizeof(double2));
  for (int a = 0; a < d; ++a)
    if (lf_length(g, a) > kFftRadix64) AL(h->lf[a], (size_t)(lf_length(g, a) - kFftRadix64) * sizeof(double2));
  AL(h->T, (size_t)spec_n * sizeof(double2));
  if (d == 3) AL(h->U, (size_t)spec_n * sizeof(double2));
  AL(h->x, (size_t)nbmax * fe * sizeof(double));
  AL(h->r, (size_t)nbmax * fe * sizeof(double));
  AL(h->p, (size_t)nbmax * fe * sizeof(double));
  AL(h->q, (size_t)nbmax * fe * sizeof(double));
  AL(h->z, (size_t)nbmax * fe * sizeof(double));
  AL(h->partial, part_rows * kMaxPartials * sizeof(double));
  AL(h->red, 1024 * sizeof(double));
  AL(h->cg, nbmax * sizeof(CgState));
  AL(h->stage_cnt, nbmax * sizeof(unsigned));
  AL(h->chunks_d, sizeof(int));
  ce = cudaMemset(h->stage_cnt, 0, nbmax * sizeof(unsigned));
  if (ce != cudaSuccess) return bail(cuda_fail(h, ce, "cudaMemset"));
  AL(h->shifts, nbmax * sizeof(StrainShift));
  AL(h->active, nbmax * sizeof(int));
  if (o.precision == JFFT_PREC_MIXED) {
    if (o.material_bf16) AL(h->E16, g.N * 2);
    else AL(h->E32, g.N * sizeof(float));
    AL(h->js32, g.N * sizeof(float) * js_components(g, h->element));
    AL(h->G32, (size_t)g.F * h->ds * sizeof(float));
    for (int a = 0; a < d; ++a) AL(h->tw32[a], (size_t)g.n[a] * sizeof(float2));
    AL(h->T32, (size_t)spec_n * sizeof(float2));
    if (d == 3) AL(h->U32, (size_t)spec_n * sizeof(float2));
    AL(h->x32, (size_t)nbmax * fe * sizeof(float));
    AL(h->r32, (size_t)nbmax * fe * sizeof(float));
    AL(h->p32, (size_t)nbmax * fe * sizeof(float));
    AL(h->q32, (size_t)nbmax * fe * sizeof(float));
    AL(h->z32, (size_t)nbmax * fe * sizeof(float));
  }
#undef AL
  ce = cudaMallocHost((void**)&h->cg_h, nbmax * sizeof(CgState));
  if (ce != cudaSuccess) return bail(cuda_fail(h, ce, "cudaMallocHost"));
  ce = cudaMallocHost((void**)&h->red_h, 1024 * sizeof(double));
  if (ce != cudaSuccess) return bail(cuda_fail(h, ce, "cudaMallocHost"));
  ce = cudaMallocHost((void**)&h->active_h, nbmax * sizeof(int));
  if (ce != cudaSuccess) return bail(cuda_fail(h, ce, "cudaMallocHost"));
  ce = cudaMallocHost((void**)&h->chunks_h, sizeof(int));
  if (ce != cudaSuccess) return bail(cuda_fail(h, ce, "cudaMallocHost"));

  for (int a = 0; a < d; ++a) {
    ce = launch_twiddles(h->tw[a], g.n[a], h->st);
    if (ce == cudaSuccess && h->lf[a]) ce = launch_lf_table(h->lf[a], lf_length(g, a), h->st);
    if (ce != cudaSuccess) return bail(cuda_fail(h, ce, "twiddles"));
  }
  s = setup_material(h, mat, false);
  if (s) return bail(s);
  if (o.autotune) {
    s = autotune(h);
    if (s) return bail(s);
  }
  g_cur = nullptr;
  *out = h;
  return JFFT_OK;
}

extern "C" void jfft_destroy(jfft_solver* h) {
  if (!h) return;
  free_all(h);
  delete h;
}

extern "C" jfft_status jfft_set_material(jfft_solver* h, const jfft_material* m) {
  if (!h) return JFFT_ERR_ARG;
  CurGuard guard(h);
  return setup_material(h, m, h->io == JFFT_MEM_DEVICE);
}

extern "C" jfft_status jfft_set_material_coarse(jfft_solver* h, const jfft_material* m, const int64_t* pixels) {
  if (!h || !pixels) return JFFT_ERR_ARG;
  CurGuard guard(h);
  return setup_material(h, m, h->io == JFFT_MEM_DEVICE, pixels);
}

extern "C" const char* jfft_status_string(jfft_status s) {
  switch (s) {
    case JFFT_OK: return "ok";
    case JFFT_ERR_ARG: return "invalid argument";
    case JFFT_ERR_OOM: return "out of device memory or over budget";
    case JFFT_ERR_CUDA: return "CUDA error";
    case JFFT_ERR_NOCONV: return "not converged within max_iter";
    case JFFT_ERR_BREAKDOWN: return "CG breakdown";
    case JFFT_ERR_TIMEOUT: return "device wait timed out";
    case JFFT_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

extern "C" const char* jfft_last_error(const jfft_solver* h) { return h ? h->err.c_str() : g_create_err.c_str(); }

extern "C" jfft_status jfft_set_io_memory(jfft_solver* h, int io) {
  if (!h) return JFFT_ERR_ARG;
  if (io != JFFT_MEM_HOST && io != JFFT_MEM_DEVICE) return fail(h, JFFT_ERR_ARG, "bad io memory");
  h->io = io;
  return JFFT_OK;
}

extern "C" jfft_status jfft_set_max_iter(jfft_solver* h, int max_iter) {
  if (!h) return JFFT_ERR_ARG;
  if (max_iter <= 0) return fail(h, JFFT_ERR_ARG, "max_iter must be positive");
  h->max_iter = max_iter;
  return JFFT_OK;
}

// ------------------------------------------------------------- PCG driver
static bool valid_pc(int pc) {
  return pc == JFFT_PC_NONE || pc == JFFT_PC_GREEN || pc == JFFT_PC_GREEN_JACOBI || pc == JFFT_PC_JACOBI;
}

// Buffers of one working precision.
template <typename T> struct Work {
  T *x, *r, *p, *q, *z;
  const T* E;
  const T* js;
  FftPlanT<T> pl;
};

static Work<double> work64(jfft_solver* h) {
  return {h->x, h->r, h->p, h->q, h->z, h->E, h->js,
          {{h->tw[0], h->tw[1], h->tw[2]}, {h->lf[0], h->lf[1], h->lf[2]}, h->T, h->U, h->G}};
}
static Work<float> work32(jfft_solver* h) {
  return {h->x32, h->r32, h->p32, h->q32, h->z32, h->E32, h->js32, {{h->tw32[0], h->tw32[1], h->tw32[2]}, {}, h->T32,
                                                                    h->U32, h->G32}};
}

static cudaError_t apply_op(jfft_solver* h, const Work<double>& w, const double* x, double* y, int nb, int dot, int* np,
                            CgState* cg, StageCtl sc = no_stage()) {
  return launch_apply_K(h->g, h->ec, w.E, 0.0, x, y, nb, field_elems(h), nullptr, 1.0, dot, h->partial, np, cg, h->st,
                        sc);
}
static cudaError_t apply_op(jfft_solver* h, const Work<float>& w, const float* x, float* y, int nb, int dot, int* np,
                            CgState* cg, StageCtl sc = no_stage()) {
  if (h->E16)
    return launch_apply_K_f32_bf16(h->g, h->ec, h->E16, x, y, nb, field_elems(h), dot, h->partial, np, cg, h->st, sc);
  return launch_apply_K_f32(h->g, h->ec, w.E, x, y, nb, field_elems(h), dot, h->partial, np, cg, h->st, sc);
}

static cudaError_t precond_op(jfft_solver* h, const Work<double>& w, int pc, const double* r, double* z, int nb,
                              CgState* cg, int* np, StageCtl sc = no_stage()) {
  if (pc == JFFT_PC_GREEN || pc == JFFT_PC_GREEN_JACOBI)
    return launch_green_precond(h->g, w.pl, r, z, nb, field_elems(h), w.js, pc == JFFT_PC_GREEN_JACOBI, h->partial,
                                np, cg, h->st, sc, h->jcs);
  return launch_jacobi_precond(h->g, r, z, nb, field_elems(h), w.js, pc == JFFT_PC_NONE, h->partial, np, cg, h->st,
                               sc, h->jcs);
}
static cudaError_t precond_op(jfft_solver* h, const Work<float>& w, int pc, const float* r, float* z, int nb,
                              CgState* cg, int* np, StageCtl sc = no_stage()) {
  if (pc == JFFT_PC_GREEN || pc == JFFT_PC_GREEN_JACOBI)
    return launch_green_precond_f32(h->g, w.pl, r, z, nb, w.js, pc == JFFT_PC_GREEN_JACOBI, h->partial, np, cg,
                                    h->st, sc, h->jcs);
  return launch_jacobi_precond_f32(h->g, r, z, nb, field_elems(h), w.js, pc == JFFT_PC_NONE, h->partial, np, cg,
                                   h->st, sc, h->jcs);
}

// Plan-time autotuner: times the candidate launch shapes of the working precision's
// operator and FFT passes on this grid and batch size (a few launches each, after one
// warm-up, CUDA events on the solver's stream) and keeps the fastest in g.tune. The
// shapes change only how the work is split into blocks, so results differ from the
// defaults at most by the rounding of the partial-sum reductions.
template <typename T>
static jfft_status autotune_t(jfft_solver* h, const Work<T>& w) {
  const Grid& g = h->g;
  const int nb = h->max_loads;
  const int64_t fe = field_elems(h);
  CK(cudaMemsetAsync(w.p, 0, nb * fe * sizeof(T), h->st));
  CK(cudaMemsetAsync(w.r, 0, nb * fe * sizeof(T), h->st));
  cudaEvent_t a = nullptr, b = nullptr;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  int np = 0;
  auto time = [&](auto&& launch) -> float {
    if (launch() != cudaSuccess) return 1e30f;
    cudaEventRecord(a, h->st);
    for (int i = 0; i < 5; ++i)
      if (launch() != cudaSuccess) return 1e30f;
    cudaEventRecord(b, h->st);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
  };
  auto pick = [&](int slot, std::initializer_list<int> cands, auto&& launch) {
    float best = 1e30f;
    int arg = 0;
    for (int c : cands) {
      h->g.tune[slot] = c;
      const float t = time(launch);
      if (t < best) { best = t; arg = c; }
    }
    h->g.tune[slot] = arg;
  };
  auto op = [&]() { return apply_op(h, w, w.p, w.q, nb, 1, &np, nullptr); };
  auto pre = [&]() { return precond_op(h, w, JFFT_PC_GREEN_JACOBI, w.r, w.z, nb, nullptr, &np); };
  if (g.d == 2) pick(0, {8, 16, 32, 64}, op);
  else if (sizeof(T) == 4) pick(1, {4, 8, 16}, op);
  pick(2, {1, 2, 4}, pre);
  pick(3, {1, 2, 4}, pre);
  cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return sync(h);
}

static jfft_status autotune(jfft_solver* h) {
  if (h->precision == JFFT_PREC_MIXED) return autotune_t<float>(h, work32(h));
  return autotune_t<double>(h, work64(h));
}

static jfft_status precond(jfft_solver* h, int pc, const double* r, double* z, int nb, CgState* cg, int* np) {
  CK(precond_op(h, work64(h), pc, r, z, nb, cg, np));
  return JFFT_OK;
}

// One check_every-iteration chunk of the PCG loop: q = K p (alpha), x and r update
// (residual test), z = M^-1 r (beta), p = z + beta p. Right-hand sides that are
// done skip every kernel, so a chunk may run past convergence at no cost. With the
// Green preconditioners the x and r update runs inside the first FFT pass (the same
// roundings of x and r; only the summation order of ||r||^2 differs).
template <typename T>
static cudaError_t pcg_chunk(jfft_solver* h, const Work<T>& w, int nb, int pc, double tol, int stop_mode, int chunk) {
  const Grid& g = h->g;
  const int64_t fe = field_elems(h);
  auto stage = [&](int k) { return StageCtl{k, stop_mode, h->max_iter, tol, h->stage_cnt}; };
  int np = 0;
  cudaError_t e;
  for (int c = 0; c < chunk; ++c) {
    if ((e = apply_op(h, w, w.p, w.q, nb, 1, &np, h->cg, stage(kStageAlpha))) != cudaSuccess) return e;
    if (pc == JFFT_PC_GREEN || pc == JFFT_PC_GREEN_JACOBI) {
      if ((e = launch_green_precond_xr<T>(g, w.pl, w.x, w.r, w.p, w.q, w.z, nb, w.js, pc == JFFT_PC_GREEN_JACOBI,
                                          h->partial, &np, h->cg, h->st, stage(kStageRR), stage(kStageBeta),
                                          h->jcs)) != cudaSuccess)
        return e;
    } else {
      if ((e = launch_cg_xr<T>(g, w.x, w.r, w.p, w.q, nb, fe, h->cg, h->partial, &np, h->st, stage(kStageRR))) !=
          cudaSuccess)
        return e;
      if ((e = precond_op(h, w, pc, w.r, w.z, nb, h->cg, &np, stage(kStageBeta))) != cudaSuccess) return e;
    }
    if ((e = launch_cg_p<T>(g, w.p, w.z, nb, fe, h->cg, h->st)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Launches one chunk, replaying a captured CUDA graph of it when allowed. The graph
// is captured on first use for a (nb, preconditioner, stopping rule, cap, chunk)
// combination; kernel arguments and buffers are otherwise fixed per solver.
template <typename T>
static cudaError_t pcg_chunk_launch(jfft_solver* h, const Work<T>& w, int nb, int pc, double tol, int stop_mode,
                                    int chunk) {
  if (!h->opt.graphs || !h->graphs_ok) return pcg_chunk<T>(h, w, nb, pc, tol, stop_mode, chunk);
  jfft_solver::ChunkGraph& gr = h->graph[sizeof(T) == 4 ? 1 : 0];
  if (!gr.exec || gr.nb != nb || gr.pc != pc || gr.tol != tol || gr.stop_mode != stop_mode ||
      gr.max_iter != h->max_iter || gr.chunk != chunk || gr.prof != h->profiling) {
    drop_graph(h, gr);
    std::lock_guard<std::recursive_mutex> lock(graph_mutex());
    cudaGraph_t graph = nullptr;
    const int64_t l0 = h->launches;
    const size_t p0 = h->pend.size();  // timing events recorded inside the capture belong to the graph
    cudaError_t e = cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      h->capturing = true;
      const cudaError_t el = pcg_chunk<T>(h, w, nb, pc, tol, stop_mode, chunk);
      h->capturing = false;
      e = cudaStreamEndCapture(h->st, &graph);
      if (e == cudaSuccess) e = el;
    }
    const int64_t captured = h->launches - l0;
    h->launches = l0;
    gr.events.assign(h->pend.begin() + p0, h->pend.end());
    h->pend.resize(p0);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gr.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      // capture is unavailable here: clear the error state and launch directly from now on
      cudaGetLastError();
      drop_graph(h, gr);
      h->graphs_ok = false;
      return pcg_chunk<T>(h, w, nb, pc, tol, stop_mode, chunk);
    }
    gr.nb = nb;
    gr.pc = pc;
    gr.tol = tol;
    gr.stop_mode = stop_mode;
    gr.max_iter = h->max_iter;
    gr.chunk = chunk;
    gr.launches = captured;
    gr.prof = h->profiling;
  }
  h->launches += gr.launches;
  h->graph_replays++;
  if (gr.prof) h->replayed = &gr;  // the caller syncs before the next replay
  return cudaGraphLaunch(gr.exec, h->st);
}

// Builds (or reuses) the CUDA graph of a whole PCG solve: a WHILE conditional node
// whose body is one chunk followed by the condition kernel. Returns false if the
// graph cannot be built here (the caller then polls from the host).
template <typename T>
static bool loop_graph_ready(jfft_solver* h, const Work<T>& w, int nb, int pc, double tol, int stop_mode, int chunk,
                             int cap_chunks) {
  jfft_solver::LoopGraph& lg = h->loop[sizeof(T) == 4 ? 1 : 0];
  if (lg.exec && lg.nb == nb && lg.pc == pc && lg.tol == tol && lg.stop_mode == stop_mode &&
      lg.max_iter == h->max_iter && lg.chunk == chunk)
    return true;
  std::lock_guard<std::recursive_mutex> lock(graph_mutex());
  destroy_exec(lg.exec);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaGraphCreate(&graph, 0);
  cudaGraphConditionalHandle cond = 0;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
  const int64_t l0 = h->launches;
  if (e == cudaSuccess) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(h->st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      h->capturing = true;
      cudaError_t el = pcg_chunk<T>(h, w, nb, pc, tol, stop_mode, chunk);
      if (el == cudaSuccess) el = launch_cg_continue(h->cg, nb, h->chunks_d, cap_chunks, cond, h->st);
      h->capturing = false;
      cudaGraph_t captured = nullptr;
      e = cudaStreamEndCapture(h->st, &captured);
      if (e == cudaSuccess) e = el;
    }
  }
  const int64_t per_chunk = h->launches - l0;
  h->launches = l0;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&lg.exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    destroy_exec(lg.exec);
    h->loop_ok = false;
    return false;
  }
  lg.nb = nb;
  lg.pc = pc;
  lg.tol = tol;
  lg.stop_mode = stop_mode;
  lg.max_iter = h->max_iter;
  lg.chunk = chunk;
  lg.launches_per_chunk = per_chunk;
  return true;
}

// Runs PCG in working precision T on w.r (holding the right-hand side) from x = 0
// for nb right-hand sides. The INIT_FF stage must have run on w.r.
template <typename T>
// keep: continue the recurrence of the previous call (reliable update): w.p and the
// kept gamma carry over, the first direction is z + (r.z / gamma) p; the caller has
// replaced w.r and started the states with kStageInitFFKeep.
static jfft_status pcg_core_t(jfft_solver* h, const Work<T>& w, int nb, int pc, double tol, int stop_mode,
                              int* status_out, bool keep = false) {
  const Grid& g = h->g;
  const int64_t fe = field_elems(h);
  int np = 0;
  jfft_status s;
  CK(cudaMemsetAsync(w.x, 0, nb * fe * sizeof(T), h->st));
  if (!keep) CK(cudaMemsetAsync(w.p, 0, nb * fe * sizeof(T), h->st));
  CK(cudaMemsetAsync(h->stage_cnt, 0, nb * sizeof(unsigned), h->st));
  // Each scalar stage runs in the last block of the kernel that produces its partials.
  CK(precond_op(h, w, pc, w.r, w.z, nb, h->cg, &np,
                StageCtl{keep ? kStageReplace : kStageInitGamma, stop_mode, h->max_iter, tol, h->stage_cnt}));
  CK(launch_cg_p<T>(g, w.p, w.z, nb, fe, h->cg, h->st));
  const int chunk = h->opt.check_every;
  int64_t launched = 0;
  const int64_t cap = (int64_t)h->max_iter + chunk;
  const int cap_chunks = (int)std::min<int64_t>(cap / chunk + 2, 1 << 30);
  // Device-side loop: one graph launch runs chunks until every right-hand side is
  // done (or cap_chunks chunks have run); the host reads the states once.
  const bool device_loop = h->opt.graphs && h->graphs_ok && h->loop_ok && !h->profiling &&
                           loop_graph_ready<T>(h, w, nb, pc, tol, stop_mode, chunk, cap_chunks);
  if (device_loop) {
    const jfft_solver::LoopGraph& lg = h->loop[sizeof(T) == 4 ? 1 : 0];
    CK(cudaMemsetAsync(h->chunks_d, 0, sizeof(int), h->st));
    CK(cudaGraphLaunch(lg.exec, h->st));
    CK(cudaMemcpyAsync(h->cg_h, h->cg, nb * sizeof(CgState), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(h->chunks_h, h->chunks_d, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    s = sync(h);
    if (s) return s;
    h->launches += (int64_t)h->chunks_h[0] * lg.launches_per_chunk;
    h->graph_replays += h->chunks_h[0];
    for (int b = 0; b < nb; ++b)
      if (h->cg_h[b].done == kRunning) return fail(h, JFFT_ERR_CUDA, "PCG driver exceeded its iteration cap");
  }
  while (!device_loop) {
    CK(pcg_chunk_launch<T>(h, w, nb, pc, tol, stop_mode, chunk));
    launched += chunk;
    CK(cudaMemcpyAsync(h->cg_h, h->cg, nb * sizeof(CgState), cudaMemcpyDeviceToHost, h->st));
    s = sync(h);
    if (s) return s;
    bool all = true;
    for (int b = 0; b < nb; ++b) all = all && h->cg_h[b].done != kRunning;
    if (all) break;
    if (launched > cap) return fail(h, JFFT_ERR_CUDA, "PCG driver exceeded its iteration cap");
  }
  int worst = kConverged;
  for (int b = 0; b < nb; ++b) {
    const int dn = h->cg_h[b].done;
    if (dn == kBreakdown) worst = kBreakdown;
    else if (dn == kNoConv && worst != kBreakdown) worst = kNoConv;
  }
  *status_out = worst;
  return JFFT_OK;
}

static jfft_status pcg_core(jfft_solver* h, int nb, int pc, double tol, int* status_out) {
  return pcg_core_t<double>(h, work64(h), nb, pc, tol, h->opt.stop_mode, status_out);
}

// Reliable updates continue the FP32 recurrence across a residual replacement only
// where ||r64 - r32|| <= kReliableGap ||r64||; a larger gap means the recurrence has
// drifted from the true residual and its search direction is dropped (restart).
#ifndef JFFT_RELIABLE_GAP
#define JFFT_RELIABLE_GAP 0.1
#endif
constexpr double kReliableGap = JFFT_RELIABLE_GAP;

// FP64 iterative refinement around the FP32 PCG (JFFT_PREC_MIXED). The right-hand
// side is the macroscopic-strain load of h->shifts (macro) or the FP64 field f.
// On return h->x holds u, its[b] the summed inner iterations, refine[b] the number
// of inner solves, ff[b] = ||f||^2 and *status_out the worst outcome.
static jfft_status solve_mixed(jfft_solver* h, int nb, int pc, double tol, bool macro, const double* f, int* its,
                               int* refine, double* ff, int* status_out) {
  const Grid& g = h->g;
  const int64_t fe = field_elems(h);
  const Work<float> w = work32(h);
  int np = 0;
  jfft_status s;
  if (macro) {
    CK(launch_apply_K(g, h->ec, h->E, 0.0, nullptr, h->r, nb, fe, h->shifts, -1.0, 2, h->partial, &np, nullptr,
                      h->st));
  } else {
    CK(launch_dot<double>(g, f, f, nb, fe, h->partial, &np, h->st));
  }
  CK(launch_reduce_partials(h->partial, np, nb, kMaxPartials, h->red, h->st));
  CK(cudaMemcpyAsync(h->red_h, h->red, nb * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemsetAsync(h->x, 0, nb * fe * sizeof(double), h->st));
  s = sync(h);
  if (s) return s;
  for (int b = 0; b < nb; ++b) {
    ff[b] = h->red_h[b];
    its[b] = 0;
    refine[b] = 0;
  }
  const int stop_mode = h->opt.stop_mode;
  bool all_conv = false;
  for (int k = 0; k <= h->opt.max_refine; ++k) {
    // FP64 residual r = f - K u and its norm
    if (macro) {
      CK(launch_apply_K(g, h->ec, h->E, 0.0, h->x, h->r, nb, fe, h->shifts, -1.0, 2, h->partial, &np, nullptr,
                        h->st));
    } else {
      CK(launch_apply_K(g, h->ec, h->E, 0.0, h->x, h->q, nb, fe, nullptr, 1.0, 0, nullptr, nullptr, nullptr, h->st));
      CK(launch_sub_norm(g, f, h->q, h->r, nb, h->partial, &np, h->st));
    }
    CK(launch_reduce_partials(h->partial, np, nb, kMaxPartials, h->red, h->st));
    // reliable updates: distance of the FP64 residual from the FP32 recurrence residual
    // it is about to replace (rows nb .. 2 nb - 1 of the partial sums)
    const bool cont = h->opt.reliable && k > 0;
    if (cont) {
      int npg = 0;
      CK(launch_gap(g, h->r, w.r, nb, h->partial + (int64_t)nb * kMaxPartials, &npg, h->st));
      CK(launch_reduce_partials(h->partial + (int64_t)nb * kMaxPartials, npg, nb, kMaxPartials, h->red + nb, h->st));
    }
    CK(cudaMemcpyAsync(h->red_h, h->red, (cont ? 2 : 1) * nb * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    s = sync(h);
    if (s) return s;
    bool any = false;
    all_conv = true;
    for (int b = 0; b < nb; ++b) {
      const double rr = h->red_h[b];
      const bool conv = ff[b] == 0.0 || (stop_mode == JFFT_STOP_REL ? rr <= tol * tol * ff[b] : rr <= tol);
      all_conv = all_conv && conv;
      // 2: continue the recurrence (the replaced residual is within kReliableGap of the
      // recurrence one); 1: restart it
      const bool near = cont && h->red_h[nb + b] <= kReliableGap * kReliableGap * rr;
      h->active_h[b] = (!conv && k < h->opt.max_refine) ? (near ? 2 : 1) : 0;
      any = any || h->active_h[b];
    }
    if (!any) break;
    CK(cudaMemcpyAsync(h->active, h->active_h, nb * sizeof(int), cudaMemcpyHostToDevice, h->st));
    CK(launch_to_f32(h->r, w.r, fe, nb, h->active, h->st));
    CK(launch_dot<float>(g, w.r, w.r, nb, fe, h->partial, &np, h->st));
    CK(launch_cg_scalars(cont ? kStageInitFFKeep : kStageInitFF, h->cg, h->partial, np, nb, h->opt.inner_tol,
                         JFFT_STOP_REL, h->max_iter, h->st, h->active));
    const bool keep = cont;
    int inner_status = kConverged;
    s = pcg_core_t<float>(h, w, nb, pc, h->opt.inner_tol, JFFT_STOP_REL, &inner_status, keep);
    if (s) return s;
    CK(launch_add_f32(h->x, w.x, nb * fe, h->st));
    for (int b = 0; b < nb; ++b)
      if (h->active_h[b]) {
        its[b] += h->cg_h[b].iters;
        refine[b] += 1;
      }
  }
  *status_out = all_conv ? kConverged : kNoConv;
  return JFFT_OK;
}

static jfft_status upload_shifts(jfft_solver* h, int n, const double* eps) {
  std::vector<StrainShift> sh(n);
  for (int b = 0; b < n; ++b) {
    for (int c = 0; c < h->ds; ++c)
      if (!std::isfinite(eps[b * h->ds + c])) return fail(h, JFFT_ERR_ARG, "macroscopic strain must be finite");
    sh[b] = make_shift(h->g.d, h->ec, eps + b * h->ds);
  }
  CK(cudaMemcpyAsync(h->shifts, sh.data(), n * sizeof(StrainShift), cudaMemcpyHostToDevice, h->st));
  // the pageable source must stay alive until the copy has been staged
  CK(cudaStreamSynchronize(h->st));
  return JFFT_OK;
}

static jfft_status check_count(jfft_solver* h, int count) {
  if (count <= 0 || count > h->max_loads) return fail(h, JFFT_ERR_ARG, "count must be in [1, max_loads]");
  return JFFT_OK;
}

extern "C" jfft_status jfft_solve(jfft_solver* h, int n_loads, const double* eps_bar, double tol, int pc,
                                  jfft_result* res) {
  if (!h) return JFFT_ERR_ARG;
  CurGuard guard(h);
  jfft_status s = check_count(h, n_loads);
  if (s) return s;
  if (!eps_bar) return fail(h, JFFT_ERR_ARG, "eps_bar is NULL");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(h, JFFT_ERR_ARG, "tol must be finite and >= 0");
  if (!valid_pc(pc)) return fail(h, JFFT_ERR_ARG, "unknown preconditioner");
  if (h->io == JFFT_MEM_DEVICE) {
    std::vector<double> eh(n_loads * h->ds);
    CK(cudaMemcpy(eh.data(), eps_bar, eh.size() * sizeof(double), cudaMemcpyDeviceToHost));
    s = upload_shifts(h, n_loads, eh.data());
  } else {
    s = upload_shifts(h, n_loads, eps_bar);
  }
  if (s) return s;
  const Grid& g = h->g;
  const int64_t fe = field_elems(h);
  const int nb = n_loads;
  int np = 0;
  int st = kConverged;
  std::vector<int> mixed_its(nb, 0), mixed_ref(nb, 1);
  std::vector<double> mixed_ff(nb, 0.0);
  if (h->precision == JFFT_PREC_MIXED) {
    s = solve_mixed(h, nb, pc, tol, true, nullptr, mixed_its.data(), mixed_ref.data(), mixed_ff.data(), &st);
    if (s) return s;
  } else {
    // S2: r = f = -B^T W C eps_bar, ||f||^2
    CK(launch_apply_K(g, h->ec, h->E, 0.0, nullptr, h->r, nb, fe, h->shifts, -1.0, 2, h->partial, &np, nullptr, h->st));
    CK(launch_cg_scalars(kStageInitFF, h->cg, h->partial, np, nb, tol, h->opt.stop_mode, h->max_iter, h->st));
    s = pcg_core(h, nb, pc, tol, &st);
    if (s) return s;
  }
  // S8: zero-mean fluctuation
  CK(launch_row_sums(h->x, nb * g.d, g.N, h->partial, &np, h->st));
  CK(launch_reduce_partials(h->partial, np, nb * g.d, kMaxPartials, h->red, h->st));
  CK(launch_sub_mean(h->x, nb * g.d, g.N, h->red, h->st));
  // true residual f - K u = -B^T W C (eps_bar + B u)
  CK(launch_apply_K(g, h->ec, h->E, 0.0, h->x, h->q, nb, fe, h->shifts, -1.0, 2, h->partial, &np, nullptr, h->st));
  CK(launch_reduce_partials(h->partial, np, nb, kMaxPartials, h->red, h->st));
  // stresses and homogenised stiffness
  double* stress_dev = (res && res->stress) ? h->z : nullptr;
  if (stress_dev && (int64_t)h->ds * g.N * nb > (int64_t)h->max_loads * fe) stress_dev = nullptr;
  CK(launch_stress(g, h->ec, h->E, h->x, nb, h->shifts, stress_dev, h->partial, &np, h->st));
  CK(launch_reduce_partials(h->partial, np, nb * h->ds, kMaxPartials, h->red + nb, h->st));
  CK(cudaMemcpyAsync(h->red_h, h->red, nb * (1 + h->ds) * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  if (h->precision != JFFT_PREC_MIXED)
    CK(cudaMemcpyAsync(h->cg_h, h->cg, nb * sizeof(CgState), cudaMemcpyDeviceToHost, h->st));
  s = sync(h);
  if (s) return s;
  if (h->precision != JFFT_PREC_MIXED)
    for (int b = 0; b < nb; ++b) {
      mixed_ff[b] = h->cg_h[b].ff;
      mixed_its[b] = h->cg_h[b].iters;
    }
  if (res) {
    if (res->u) { s = copy_out(h, res->u, h->x, nb * fe * sizeof(double)); if (s) return s; }
    if (res->stress) {
      if (stress_dev) {
        s = copy_out(h, res->stress, stress_dev, (size_t)nb * h->ds * g.N * sizeof(double));
      } else {
        // stress of many loads: one load at a time through the z buffer
        for (int b = 0; b < nb && !s; ++b) {
          CK(launch_stress(g, h->ec, h->E, h->x + b * fe, 1, h->shifts + b, h->z, h->partial, &np, h->st));
          s = copy_out(h, res->stress + (size_t)b * h->ds * g.N, h->z, (size_t)h->ds * g.N * sizeof(double));
        }
      }
      if (s) return s;
    }
    std::vector<double> chom(h->ds * nb), rel(nb);
    for (int b = 0; b < nb; ++b) {
      const double ff = mixed_ff[b];
      rel[b] = ff > 0.0 ? std::sqrt(h->red_h[b] / ff) : 0.0;
      for (int c = 0; c < h->ds; ++c) chom[c * nb + b] = h->red_h[nb + b * h->ds + c];
    }
    if (h->io == JFFT_MEM_DEVICE) {
      if (res->C_hom) CK(cudaMemcpy(res->C_hom, chom.data(), chom.size() * sizeof(double), cudaMemcpyHostToDevice));
      if (res->rel_res) CK(cudaMemcpy(res->rel_res, rel.data(), nb * sizeof(double), cudaMemcpyHostToDevice));
      if (res->iters) CK(cudaMemcpy(res->iters, mixed_its.data(), nb * sizeof(int), cudaMemcpyHostToDevice));
      if (res->refine_steps)
        CK(cudaMemcpy(res->refine_steps, mixed_ref.data(), nb * sizeof(int), cudaMemcpyHostToDevice));
    } else {
      if (res->C_hom) std::memcpy(res->C_hom, chom.data(), chom.size() * sizeof(double));
      if (res->rel_res) std::memcpy(res->rel_res, rel.data(), nb * sizeof(double));
      if (res->iters) std::memcpy(res->iters, mixed_its.data(), nb * sizeof(int));
      if (res->refine_steps) std::memcpy(res->refine_steps, mixed_ref.data(), nb * sizeof(int));
    }
  }
  s = sync(h);
  if (s) return s;
  if (st == kBreakdown) return fail(h, JFFT_ERR_BREAKDOWN, "CG breakdown (non-positive or non-finite p.Kp or r.z)");
  if (st == kNoConv) return fail(h, JFFT_ERR_NOCONV, "max_iter reached before the stopping rule held");
  return JFFT_OK;
}

// ------------------------------------------------------------- building blocks
extern "C" jfft_status jfft_get_material(jfft_solver* h, double* E) {
  if (!h || !E) return h ? fail(h, JFFT_ERR_ARG, "NULL output") : JFFT_ERR_ARG;
  CurGuard guard(h);
  jfft_status s = copy_out(h, E, h->E, h->g.N * sizeof(double));
  if (s) return s;
  return sync(h);
}

extern "C" jfft_status jfft_rhs(jfft_solver* h, int count, const double* eps, double* f) {
  if (!h) return JFFT_ERR_ARG;
  CurGuard guard(h);
  jfft_status s = check_count(h, count);
  if (s) return s;
  if (!eps || !f) return fail(h, JFFT_ERR_ARG, "NULL argument");
  std::vector<double> eh(count * h->ds);
  if (h->io == JFFT_MEM_DEVICE) CK(cudaMemcpy(eh.data(), eps, eh.size() * sizeof(double), cudaMemcpyDeviceToHost));
  else std::memcpy(eh.data(), eps, eh.size() * sizeof(double));
  s = upload_shifts(h, count, eh.data());
  if (s) return s;
  CK(launch_apply_K(h->g, h->ec, h->E, 0.0, nullptr, h->r, count, field_elems(h), h->shifts, -1.0, 0, nullptr, nullptr,
                    nullptr, h->st));
  s = copy_out(h, f, h->r, count * field_elems(h) * sizeof(double));
  if (s) return s;
  return sync(h);
}

extern "C" jfft_status jfft_apply_K(jfft_solver* h, int count, const double* x, double* y) {
  if (!h) return JFFT_ERR_ARG;
  CurGuard guard(h);
  jfft_status s = check_count(h, count);
  if (s) return s;
  if (!x || !y) return fail(h, JFFT_ERR_ARG, "NULL argument");
  const int64_t fe = field_elems(h);
  s = copy_in(h, h->p, x, count * fe);
  if (s) return s;
  if (h->precision == JFFT_PREC_MIXED) {
    CK(launch_to_f32(h->p, h->p32, count * fe, 1, nullptr, h->st));
    CK(apply_op(h, work32(h), h->p32, h->q32, count, 0, nullptr, nullptr));
    CK(cudaMemsetAsync(h->q, 0, count * fe * sizeof(double), h->st));
    CK(launch_add_f32(h->q, h->q32, count * fe, h->st));
  } else {
    CK(launch_apply_K(h->g, h->ec, h->E, 0.0, h->p, h->q, count, fe, nullptr, 1.0, 0, nullptr, nullptr, nullptr, h->st));
  }
  s = copy_out(h, y, h->q, count * fe * sizeof(double));
  if (s) return s;
  return sync(h);
}

extern "C" jfft_status jfft_get_diag(jfft_solver* h, int method, double* diag) {
  if (!h) return JFFT_ERR_ARG;
  CurGuard guard(h);
  if (!diag) return fail(h, JFFT_ERR_ARG, "NULL output");
  const Grid& g = h->g;
  if (method == JFFT_DIAG_CLOSED_FORM) {
    if (h->element == JFFT_ELEM_P1) CK(launch_diag_p1(g, h->E, h->kappa_p1, h->z, h->st));
    else CK(launch_diag_closed(g, h->esum, h->kappa, h->z, h->st));
  } else if (method == JFFT_DIAG_COMBS) {
    for (int a = 0; a < g.d; ++a)
      for (int off = 0; off < (1 << g.d); ++off) {
        CK(launch_fill_comb(g, a, off, h->p, h->st));
        CK(launch_apply_K(g, h->ec, h->E, 0.0, h->p, h->q, 1, field_elems(h), nullptr, 1.0, 0, nullptr, nullptr,
                          nullptr, h->st));
        CK(launch_extract_comb(g, a, off, h->q, h->z, h->st));
      }
  } else {
    return fail(h, JFFT_ERR_ARG, "unknown diagonal method");
  }
  jfft_status s = copy_out(h, diag, h->z, field_elems(h) * sizeof(double));
  if (s) return s;
  return sync(h);
}

extern "C" jfft_status jfft_get_green(jfft_solver* h, double* G) {
  if (!h) return JFFT_ERR_ARG;
  CurGuard guard(h);
  if (!G) return fail(h, JFFT_ERR_ARG, "NULL output");
  const Grid& g = h->g;
  CK(launch_green_export(g, h->G, h->z, h->scale_store, h->st));
  jfft_status s = copy_out(h, G, h->z, (size_t)g.F * g.d * g.d * sizeof(double));
  if (s) return s;
  return sync(h);
}

extern "C" jfft_status jfft_apply_precond(jfft_solver* h, int pc, int count, const double* r, double* z) {
  if (!h) return JFFT_ERR_ARG;
  CurGuard guard(h);
  jfft_status s = check_count(h, count);
  if (s) return s;
  if (!valid_pc(pc)) return fail(h, JFFT_ERR_ARG, "unknown preconditioner");
  if (!r || !z) return fail(h, JFFT_ERR_ARG, "NULL argument");
  const int64_t fe = field_elems(h);
  s = copy_in(h, h->r, r, count * fe);
  if (s) return s;
  int np = 0;
  if (h->precision == JFFT_PREC_MIXED) {
    CK(launch_to_f32(h->r, h->r32, count * fe, 1, nullptr, h->st));
    CK(precond_op(h, work32(h), pc, h->r32, h->z32, count, nullptr, &np));
    CK(cudaMemsetAsync(h->z, 0, count * fe * sizeof(double), h->st));
    CK(launch_add_f32(h->z, h->z32, count * fe, h->st));
  } else {
    s = precond(h, pc, h->r, h->z, count, nullptr, &np);
    if (s) return s;
  }
  s = copy_out(h, z, h->z, count * fe * sizeof(double));
  if (s) return s;
  return sync(h);
}

extern "C" jfft_status jfft_solve_rhs(jfft_solver* h, int count, const double* f, double tol, int pc, double* u,
                                      int* iters) {
  if (!h) return JFFT_ERR_ARG;
  CurGuard guard(h);
  jfft_status s = check_count(h, count);
  if (s) return s;
  if (!f) return fail(h, JFFT_ERR_ARG, "f is NULL");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(h, JFFT_ERR_ARG, "tol must be finite and >= 0");
  if (!valid_pc(pc)) return fail(h, JFFT_ERR_ARG, "unknown preconditioner");
  const int64_t fe = field_elems(h);
  int np = 0;
  int st = kConverged;
  std::vector<int> its(count, 0), ref(count, 1);
  if (h->precision == JFFT_PREC_MIXED) {
    s = copy_in(h, h->z, f, count * fe);  // the FP64 z buffer is free in mixed mode
    if (s) return s;
    std::vector<double> ff(count);
    s = solve_mixed(h, count, pc, tol, false, h->z, its.data(), ref.data(), ff.data(), &st);
    if (s) return s;
  } else {
    s = copy_in(h, h->r, f, count * fe);
    if (s) return s;
    CK(launch_dot<double>(h->g, h->r, h->r, count, fe, h->partial, &np, h->st));
    CK(launch_cg_scalars(kStageInitFF, h->cg, h->partial, np, count, tol, h->opt.stop_mode, h->max_iter, h->st));
    s = pcg_core(h, count, pc, tol, &st);
    if (s) return s;
    for (int b = 0; b < count; ++b) its[b] = h->cg_h[b].iters;
  }
  if (u) { s = copy_out(h, u, h->x, count * fe * sizeof(double)); if (s) return s; }
  if (iters) {
    if (h->io == JFFT_MEM_DEVICE) CK(cudaMemcpy(iters, its.data(), count * sizeof(int), cudaMemcpyHostToDevice));
    else std::memcpy(iters, its.data(), count * sizeof(int));
  }
  s = sync(h);
  if (s) return s;
  if (st == kBreakdown) return fail(h, JFFT_ERR_BREAKDOWN, "CG breakdown");
  if (st == kNoConv && tol > 0.0) return fail(h, JFFT_ERR_NOCONV, "max_iter reached before the stopping rule held");
  return JFFT_OK;
}

extern "C" jfft_status jfft_postprocess(jfft_solver* h, int count, const double* eps, const double* u, double* stress,
                                        double* C_hom) {
  if (!h) return JFFT_ERR_ARG;
  CurGuard guard(h);
  jfft_status s = check_count(h, count);
  if (s) return s;
  if (!eps || !u) return fail(h, JFFT_ERR_ARG, "NULL argument");
  const Grid& g = h->g;
  const int64_t fe = field_elems(h);
  std::vector<double> eh(count * h->ds);
  if (h->io == JFFT_MEM_DEVICE) CK(cudaMemcpy(eh.data(), eps, eh.size() * sizeof(double), cudaMemcpyDeviceToHost));
  else std::memcpy(eh.data(), eps, eh.size() * sizeof(double));
  s = upload_shifts(h, count, eh.data());
  if (s) return s;
  s = copy_in(h, h->x, u, count * fe);
  if (s) return s;
  std::vector<double> chom(h->ds * count);
  for (int b = 0; b < count; ++b) {
    int np = 0;
    CK(launch_stress(g, h->ec, h->E, h->x + b * fe, 1, h->shifts + b, stress ? h->z : nullptr, h->partial, &np, h->st));
    CK(launch_reduce_partials(h->partial, np, h->ds, kMaxPartials, h->red, h->st));
    CK(cudaMemcpyAsync(h->red_h, h->red, h->ds * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    if (stress) { s = copy_out(h, stress + (size_t)b * h->ds * g.N, h->z, (size_t)h->ds * g.N * sizeof(double)); if (s) return s; }
    s = sync(h);
    if (s) return s;
    for (int c = 0; c < h->ds; ++c) chom[c * count + b] = h->red_h[c];
  }
  if (C_hom) {
    if (h->io == JFFT_MEM_DEVICE) CK(cudaMemcpy(C_hom, chom.data(), chom.size() * sizeof(double), cudaMemcpyHostToDevice));
    else std::memcpy(C_hom, chom.data(), chom.size() * sizeof(double));
  }
  return JFFT_OK;
}

// ------------------------------------------------------------- instrumentation
extern "C" int64_t jfft_launch_count(const jfft_solver* h) { return h ? h->launches : 0; }
extern "C" int64_t jfft_graph_replays(const jfft_solver* h) { return h ? h->graph_replays : 0; }

extern "C" jfft_status jfft_get_tuning(const jfft_solver* h, int* tune) {
  if (!h || !tune) return JFFT_ERR_ARG;
  for (int i = 0; i < 4; ++i) tune[i] = h->g.tune[i];
  return JFFT_OK;
}

extern "C" jfft_status jfft_set_tuning(jfft_solver* h, const int* tune) {
  if (!h || !tune) return JFFT_ERR_ARG;
  static const int allowed[4][5] = {{0, 8, 16, 32, 64}, {0, 4, 8, 16, 0}, {0, 1, 2, 4, 0}, {0, 1, 2, 4, 0}};
  for (int i = 0; i < 4; ++i) {
    bool ok = false;
    for (int j = 0; j < 5; ++j) ok = ok || (tune[i] == allowed[i][j] && (j == 0 || allowed[i][j] != 0));
    if (!ok) return fail(h, JFFT_ERR_ARG, "tuning value outside the candidate set");
  }
  CurGuard guard(h);
  jfft_status s = sync(h);
  if (s) return s;
  for (int i = 0; i < 4; ++i) h->g.tune[i] = tune[i];
  // captured graphs hold the old launch shapes
  for (auto& gr : h->graph) drop_graph(h, gr);
  for (auto& lg : h->loop) destroy_exec(lg.exec);
  return JFFT_OK;
}

extern "C" jfft_status jfft_set_profiling(jfft_solver* h, int on) {
  if (!h) return JFFT_ERR_ARG;
  CurGuard guard(h);
  jfft_status s = sync(h);
  if (s) return s;
  h->profiling = on != 0;
  if (on) h->prof.clear();
  return JFFT_OK;
}

extern "C" const char* jfft_profile_json(jfft_solver* h) {
  if (!h) return "{}";
  {
    CurGuard guard(h);
    if (sync(h)) return "{}";
  }
  std::string s = "{";
  bool first = true;
  for (auto& kv : h->prof) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s\"%s\": [%lld, %.6f]", first ? "" : ", ", kv.first.c_str(), (long long)kv.second.first,
             kv.second.second);
    s += buf;
    first = false;
  }
  s += "}";
  h->prof_json = s;
  return h->prof_json.c_str();
}

extern "C" size_t jfft_workspace_bytes(const jfft_solver* h) { return h ? h->ws_bytes : 0; }

extern "C" jfft_status jfft_workspace_estimate(const jfft_grid* grid, const jfft_options* opt, size_t* bytes) {
  if (!bytes) return JFFT_ERR_ARG;
  *bytes = 0;
  Grid g;
  if (make_grid(grid, g)) return grid && (grid->dim == 2 || grid->dim == 3) ? JFFT_ERR_UNSUPPORTED : JFFT_ERR_ARG;
  jfft_options o;
  jfft_default_options(&o);
  if (opt) o = *opt;
  int nbmax = o.max_loads <= 0 ? 6 : o.max_loads;
  if (nbmax < g.d) nbmax = g.d;
  if (nbmax > kMaxLoads) return JFFT_ERR_ARG;
  if (o.precision != JFFT_PREC_FP64 && o.precision != JFFT_PREC_MIXED) return JFFT_ERR_ARG;
  *bytes = plan_bytes(g, g.d * (g.d + 1) / 2, nbmax, o.precision, o.element, o.material_bf16);
  return JFFT_OK;
}

extern "C" jfft_status jfft_set_stream(jfft_solver* h, void* stream) {
  if (!h) return JFFT_ERR_ARG;
  CurGuard guard(nullptr);
  cudaSetDevice(h->device);
  CK(cudaStreamSynchronize(h->st));
  if (h->own_stream) {
    if (stream) {
      cudaStreamDestroy(h->st);
      cudaEventDestroy(h->ev_in);
      cudaEventDestroy(h->ev_out);
      h->ev_in = h->ev_out = nullptr;
      h->own_stream = false;
      h->st = (cudaStream_t)stream;
    }
    return JFFT_OK;
  }
  if (stream) {
    h->st = (cudaStream_t)stream;
    return JFFT_OK;
  }
  cudaStream_t st = nullptr;
  CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
  h->st = st;
  h->own_stream = true;
  return JFFT_OK;
}
