/*
 * jfft.h -- C ABI of the GB300 J-FFT solver.
 *
 * Solves the periodic small-strain linear-elastic cell problem on a regular grid
 * (Ladecky et al., arXiv 2508.02613, Sec. 2) with preconditioned conjugate
 * gradients (Sec. 2.3) and the Green (Sec. 3.1, Eq. prec_lin_systemG_FFT), Jacobi
 * (Sec. 3.2, Eq. prec_lin_systemJ) or Green-Jacobi preconditioner (Sec. 3.3,
 * Eq. prec_lin_systemJG_2). The discretisation is Q1 (bilinear quads with 2x2 Gauss
 * points in 2D, plane strain; trilinear hexes with 2x2x2 Gauss points in 3D) on the
 * unit cell with n_a nodal points per axis, periodic, h_a = 1 / n_a (Sec. 2.1).
 *
 * Conventions shared by every call:
 *  - Node I = (i_1, .., i_d) has flat index ((i_1 n_2) + i_2) n_3 + i_3 (C order,
 *    last axis contiguous); N = n_1 ... n_d. Voxel (element) e has its lowest
 *    corner at node e and couples nodes (e + o) mod n, o in {0,1}^d.
 *  - A displacement-like field is an array [d][N] of doubles (component-major,
 *    the [d, N_1, .., N_d] layout of the paper's Alg. 1). Several fields are
 *    stacked as [count][d][N].
 *  - Strain and stress use Mandel notation: 2D (11, 22, sqrt2*12); 3D
 *    (11, 22, 33, sqrt2*23, sqrt2*13, sqrt2*12) (Sec. 2; sqrt2 as in Sec. 4.5).
 *  - Material: C_e = E_e * C_unit(nu), isotropic, unit Young's modulus, plane
 *    strain in 2D (the paper's sigma = rho C^0 eps of Sec. 4 has this form).
 *  - Data pointers passed to any call other than jfft_create are host pointers
 *    when the handle's io memory is JFFT_MEM_HOST (default) and device pointers
 *    (on the handle's device) when it is JFFT_MEM_DEVICE; this includes the
 *    material field given to jfft_set_material. The field given to jfft_create is
 *    always a host pointer. The caller owns
 *    every buffer it passes; inputs are read during the call only, outputs are
 *    written before the call returns (device outputs: ordered on the handle's
 *    stream, complete when the call returns because each call synchronises it).
 *  - Every call returns a jfft_status; on failure jfft_last_error() returns a
 *    message. A handle is not thread safe; distinct handles are independent.
 *  - The library allocates its device workspace with the CUDA runtime inside
 *    jfft_create and frees it in jfft_destroy.
 */
#ifndef JFFT_H
#define JFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define JFFT_API_VERSION 1

typedef struct jfft_solver jfft_solver; /* opaque; owns all device memory */

typedef enum {
  JFFT_OK = 0,
  JFFT_ERR_ARG = 1,          /* invalid argument (message says which) */
  JFFT_ERR_OOM = 2,          /* workspace does not fit the device or the hbm_budget */
  JFFT_ERR_CUDA = 3,         /* a CUDA runtime call failed */
  JFFT_ERR_NOCONV = 4,       /* max_iter reached; outputs hold the last iterate */
  JFFT_ERR_BREAKDOWN = 5,    /* p.Kp <= 0 or a non-finite CG scalar; outputs hold the last iterate */
  JFFT_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up */
  JFFT_ERR_UNSUPPORTED = 7   /* valid request outside what this build implements */
} jfft_status;

typedef enum {
  JFFT_PC_NONE = -1,         /* plain CG (M = I), for testing */
  JFFT_PC_GREEN = 0,         /* M^-1 = F^-1 G_hat F (Eq. prec_lin_systemG_FFT) */
  JFFT_PC_GREEN_JACOBI = 1,  /* M^-1 = J^1/2 F^-1 G_hat F J^1/2 (Eq. prec_lin_systemJG_2) */
  JFFT_PC_JACOBI = 2         /* M^-1 = diag(K)^-1 (Eq. prec_lin_systemJ) */
} jfft_precond;

typedef enum {
  JFFT_MAT_YOUNG = 0,        /* field = E per voxel (>= 0, finite) */
  JFFT_MAT_DENSITY = 1       /* field = rho per voxel; E = e_min + (e_max - e_min) rho^exponent, on the device */
} jfft_material_kind;

typedef enum {
  JFFT_ELEM_Q1 = 0,          /* bilinear (2D) / trilinear (3D) voxel, full 2^d Gauss rule */
  JFFT_ELEM_P1 = 1           /* 2D: two linear triangles per voxel (the paper's Sec. 4 discretisation) */
} jfft_element;

typedef enum {
  JFFT_PREC_FP64 = 0,        /* every step in FP64 */
  JFFT_PREC_MIXED = 1        /* FP64 iterative refinement around an FP32 PCG: operator, FFT, preconditioner and
                                vectors of the inner solve in FP32, CG scalars and every reduction above the
                                thread in FP64, residual f - K u and the solution u in FP64 */
} jfft_precision;

typedef enum {
  JFFT_STOP_REL = 0,         /* ||r_k||_2 <= tol ||f||_2 (r the recursively updated residual) */
  JFFT_STOP_ABS_SQ = 1       /* ||r_k||_2^2 <= tol (the paper's rule, Sec. 4 "Termination criteria") */
} jfft_stop_mode;

typedef enum { JFFT_MEM_HOST = 0, JFFT_MEM_DEVICE = 1 } jfft_memory;

typedef enum {
  JFFT_DIAG_CLOSED_FORM = 0, /* diag(K)_{aI} = kappa_a * sum of E over the 2^d voxels at node I */
  JFFT_DIAG_COMBS = 1        /* Alg. 2: d 2^d operator applications to impulse combs (even n only) */
} jfft_diag_method;

typedef struct {
  int dim;                   /* 2 or 3 */
  int64_t n[3];              /* nodal points (= voxels) per axis; each a power of two, 4..2048 (2D), 4..1024 (3D) */
} jfft_grid;

typedef struct {
  int kind;                  /* jfft_material_kind */
  const double* field;       /* array [N] in node order (voxel e at its lowest-corner node) */
  double nu;                 /* Poisson ratio, -1 < nu < 0.5 */
  double e_min, e_max;       /* JFFT_MAT_DENSITY only */
  double exponent;           /* JFFT_MAT_DENSITY only (> 0) */
} jfft_material;

typedef struct {
  int precision;             /* jfft_precision (FP64) */
  int max_iter;              /* PCG iteration cap per load case (default 100000) */
  int stop_mode;             /* jfft_stop_mode (default JFFT_STOP_REL) */
  void* stream;              /* cudaStream_t to run on; NULL = a stream the solver creates, ordered
                                after earlier and before later work on the legacy default stream */
  size_t hbm_budget;         /* bytes the workspace may take; 0 = no limit beyond free memory */
  int check_every;           /* PCG iterations launched between host convergence checks (default 8) */
  int io_memory;             /* jfft_memory for the data pointers of later calls (default HOST) */
  int max_loads;             /* largest n_loads / count accepted by later calls (default 6) */
  double void_value;         /* replaces zero diagonal entries of K before J = diag^-1 (default 1, Sec. 3.2) */
  int device;                /* CUDA device ordinal (default 0) */
  double inner_tol;          /* MIXED: relative residual of each FP32 inner solve (default 1e-3) */
  int max_refine;            /* MIXED: largest number of inner solves per load (default 30) */
  int graphs;                /* 1 (default): the check_every-iteration PCG chunk is captured once as a
                                CUDA graph and replayed; 0: every kernel is launched from the host.
                                Results are identical; graphs are not used while profiling is on. */
  int element;               /* voxel discretisation: JFFT_ELEM_Q1 (default, bilinear / trilinear, full
                                Gauss rule) or JFFT_ELEM_P1 (2D only: each voxel split along its
                                (0,0)-(1,1) diagonal into two linear triangles, Sec. 4) */
  int autotune;              /* 1: at creation, time the candidate launch shapes of the operator and
                                FFT passes (working precision, max_loads right-hand sides) and keep
                                the fastest (jfft_get_tuning). 0 (default): built-in shapes. Shapes
                                change only the block split: results differ at most by the rounding
                                of the partial-sum reductions. */
  int reliable;              /* MIXED: 0 (default): every refinement step restarts CG on the new
                                residual (classic iterative refinement). 1: reliable updates: the
                                FP64 residual f - K u replaces the FP32 recurrence residual and,
                                for each load whose recurrence residual is within 10 % of it, the
                                search direction is kept (beta from the last r.z) instead of
                                restarting. */
  int material_bf16;         /* MIXED: 1: the FP32 operator reads E from a BF16 copy (E rounded to 8
                                significant bits, half the bytes of the FP32 copy); the FP64 residual
                                of the refinement keeps the FP64 E, so the solve still meets its
                                tolerance on the true operator. 0 (default): FP32 copy. Requires
                                precision MIXED. */
} jfft_options;

typedef struct {
  double* u;                 /* [n_loads][d][N] zero-mean fluctuation displacement, or NULL */
  double* stress;            /* [n_loads][d*][N] element-averaged Mandel stress, or NULL */
  double* C_hom;             /* [d*][n_loads]: column g = cell-averaged stress for eps_bar[g], or NULL */
  int* iters;                /* [n_loads] PCG iterations (operator applications in the loop; MIXED: summed
                                over the inner solves), or NULL */
  double* rel_res;           /* [n_loads] true ||f - K u||_2 / ||f||_2 recomputed at exit (0 if f = 0), or NULL */
  int* refine_steps;         /* [n_loads] MIXED: FP32 inner solves run (FP64: 1), or NULL */
} jfft_result;

/* Fill *opt with the defaults listed above. */
void jfft_default_options(jfft_options* opt);

/*
 * Create a solver for one grid and material (paper Sec. 2-3; setup steps of
 * Alg. 1 and Alg. 2). Uploads the field, computes E (Sec. 4 "Constitutive law"),
 * the reference symbol G_hat by Alg. 1 on the device (impulse responses of K_ref,
 * forward FFT, d x d inversion, zero frequency pinned to 0) and J^1/2 with the
 * void rule (Sec. 3.2). C_ref: NULL selects mean(E) C_unit(nu) (the mean
 * material); otherwise a host [d*][d*] Mandel matrix that must be isotropic
 * (lambda, mu with mu > 0, lambda + 2 mu / d > 0), else JFFT_ERR_UNSUPPORTED.
 * opt may be NULL (defaults). On success *out is a new handle; on failure *out
 * is NULL and the returned status says why.
 */
jfft_status jfft_create(jfft_solver** out, const jfft_grid* grid, const jfft_material* mat,
                        const double* C_ref, const jfft_options* opt);

/* Replace the material field (same grid and C_ref choice; nu may change when C_ref
 * was NULL); recomputes E, J^1/2 and, when C_ref was NULL, G_hat for the new mean
 * (Alg. 1). No reallocation. The field pointer follows the handle's io memory; a
 * device field is validated on the device (JFFT_ERR_ARG if any entry is negative or
 * not finite). */
jfft_status jfft_set_material(jfft_solver* h, const jfft_material* mat);

/* The same for a geometry G_p of pixels[a] (powers of two, <= n[a]) pixels per axis
 * discretised on this grid T_n (Sec. 4 "Material data sampling", "Discretization and
 * grid refinement": n >= p, pixel-wise constant data). mat->field holds one value
 * per pixel, [p0][p1]([p2]) C order; every voxel takes the value of the pixel that
 * contains it. JFFT_ERR_ARG for other pixel counts. */
jfft_status jfft_set_material_coarse(jfft_solver* h, const jfft_material* mat, const int64_t* pixels);

/*
 * Solve for n_loads macroscopic strains eps_bar [n_loads][d*] (Mandel): for each,
 * f = -B^T W C eps_bar (Eq. lin_system_exp), PCG from u_0 = 0 (Sec. 4 "Initial
 * solution") until the stop rule with tolerance tol, then the post-processing of
 * Sec. 5.3 / Eq. aim_fun (mean removal, stresses, homogenised stiffness) and the
 * true relative residual. The load cases run as one batch with per-load
 * convergence. JFFT_ERR_NOCONV / JFFT_ERR_BREAKDOWN still fill the outputs.
 */
jfft_status jfft_solve(jfft_solver* h, int n_loads, const double* eps_bar, double tol,
                       int precond, jfft_result* res);

/* Free the handle and its device memory. NULL is ignored. */
void jfft_destroy(jfft_solver* h);

const char* jfft_status_string(jfft_status s);
/* Message of the last failure on h; with h == NULL, the message of the last
 * failed jfft_create on the calling thread. Valid until the next call. */
const char* jfft_last_error(const jfft_solver* h);

/* Per-handle settings. */
jfft_status jfft_set_io_memory(jfft_solver* h, int io_memory);
jfft_status jfft_set_max_iter(jfft_solver* h, int max_iter);
/* Moves the handle to another stream (NULL: a stream the handle creates and owns),
 * after finishing the work queued on the current one. Captured CUDA graphs stay valid. */
jfft_status jfft_set_stream(jfft_solver* h, void* stream);

/* Device workspace in bytes that jfft_create would allocate for this grid and these
 * options (NULL options: defaults), without allocating. JFFT_ERR_ARG /
 * JFFT_ERR_UNSUPPORTED for grids jfft_create would reject. */
jfft_status jfft_workspace_estimate(const jfft_grid* grid, const jfft_options* opt, size_t* bytes);

/* ---- building blocks of the path (same handle, same pointer rules) ---- */

/* S1: the per-voxel Young's modulus E [N] as used by the solver. */
jfft_status jfft_get_material(jfft_solver* h, double* E);

/* S2: f = -B^T W C eps_bar for count strains [count][d*] -> f [count][d][N] (Eq. lin_system_exp). */
jfft_status jfft_rhs(jfft_solver* h, int count, const double* eps_bar, double* f);

/* S3: y = K x for count fields [count][d][N], K = B^T W C B matrix free (Sec. 3.1 "Matrix-free assembly").
 * With JFFT_PREC_MIXED this and jfft_apply_precond run the FP32 kernels of the
 * inner solve (inputs rounded to FP32, outputs widened to FP64). */
jfft_status jfft_apply_K(jfft_solver* h, int count, const double* x, double* y);

/* S5: diag(K) [d][N] before the void rule, by the closed form or by Alg. 2. */
jfft_status jfft_get_diag(jfft_solver* h, int method, double* diag);

/*
 * S9: the Green symbol G_hat of Alg. 1 on the half spectrum. Output [F][d][d]
 * (row-major d x d block per frequency), frequencies ordered with k_1 fastest:
 * 2D index (k_2 * n_1 + k_1), 3D ((k_3 * n_2 + k_2) * n_1 + k_1), with
 * 0 <= k_d <= n_d / 2 on the last (contiguous) axis and 0 <= k_a < n_a elsewhere;
 * F = n_1 .. n_{d-1} (n_d / 2 + 1). Values are the inverse of K_hat_ref (the
 * unnormalised DFT of the impulse responses), zero at k = 0.
 */
jfft_status jfft_get_green(jfft_solver* h, double* G);

/* S5 + S6: z = M^-1 r for count fields [count][d][N] and the given preconditioner. */
jfft_status jfft_apply_precond(jfft_solver* h, int precond, int count, const double* r, double* z);

/*
 * S4 + S7: PCG for count arbitrary right-hand sides f [count][d][N] from u_0 = 0.
 * u [count][d][N] receives the raw iterate (no mean removal), iters [count] the
 * iteration counts. With tol = 0 exactly max_iter iterations run (same-k tests,
 * FP64 handles). With JFFT_PREC_MIXED the result is the refined FP64 solution.
 */
jfft_status jfft_solve_rhs(jfft_solver* h, int count, const double* f, double tol, int precond,
                           double* u, int* iters);

/* S8: for count strains and displacements u [count][d][N] (used as given), the
 * element-averaged stress [count][d*][N] and C_hom [d*][count]; either may be NULL. */
jfft_status jfft_postprocess(jfft_solver* h, int count, const double* eps_bar, const double* u,
                             double* stress, double* C_hom);

/*
 * Allocation-free operator step (the paper has no counterpart: this exists for
 * callers that cannot allocate device memory, e.g. code inside a framework that
 * has already reserved the device memory for its own pool, or a latency-critical
 * loop that must not take the implicit device synchronisation that cudaMalloc or
 * cudaFree can cause).
 *
 * Computes y = K x and xy = x . y for one field with K = B^T W C B, C = E_e
 * C_unit(nu), on the given grid, without a handle and without allocating: no
 * cudaMalloc, cudaFree or allocating library call. All pointers are device
 * pointers on the current device, owned by the caller: E [N] Young's modulus per
 * voxel, x [d][N] input, y [d][N] output, xy one double (output). stream is a
 * cudaStream_t or NULL; the call only enqueues work on it and returns.
 *
 * Scratch: the per-block partial sums of x . y live in a library-owned static
 * device array of 8192 doubles (64 KiB), held on every GPU that loads the library
 * until the process exits. The first call on a device looks up that array's
 * address with that device current (make this first call before any stream
 * capture). All calls share the array and each call overwrites the part it uses,
 * so calls that may overlap on the GPU (other streams, other host threads) race
 * and must be serialised by the caller.
 *
 * y must not overlap x or E (the kernel writes y while other blocks still read
 * the halo layers of x), and xy must not overlap any of them: an in-place or
 * overlapping call is refused with JFFT_ERR_ARG.
 *
 * Errors: JFFT_ERR_ARG for NULL or overlapping pointers, nu outside (-1, 0.5) or
 * dim not 2/3; JFFT_ERR_UNSUPPORTED (nothing launched) for axis lengths that are
 * not powers of two in 4..2048 (2D) / 4..1024 (3D) or a launch that would need
 * more than 8192 partial sums; JFFT_ERR_CUDA if one of this call's own CUDA calls
 * fails (an error left pending on the thread by earlier work is not read or
 * cleared).
 */
jfft_status jfft_apply_K_dot_noalloc(const jfft_grid* grid, double nu, const double* E, const double* x,
                                     double* y, double* xy, void* stream);

/* ---- small-cell batches (many cells in one launch) ----
 *
 * Many independent periodic cells of one small 2D grid, each with its own material
 * field, Poisson ratio and lower Young's modulus, all solved for the same
 * macroscopic strains (paper Sec. 2 cell problem, Green or Green-Jacobi PCG of
 * Sec. 3, Alg. 1 symbol with each cell's mean material as reference). One CUDA
 * block per (cell, load case) runs the whole solve in shared memory, FP64, with
 * the stopping rule, iteration cap and void value of the options.
 */
typedef struct jfft_cells jfft_cells;

/* grid: dim 2, n[0], n[1] powers of two in [4, 32]; max_cells: largest batch;
 * opt: as for jfft_create (precision must be FP64; max_loads bounds n_loads;
 * io_memory applies to the field and result arrays of jfft_cells_solve).
 * JFFT_ERR_UNSUPPORTED for other grids or precisions, JFFT_ERR_OOM if the
 * workspace does not fit. The message of a failed call: jfft_cells_last_error(NULL). */
jfft_status jfft_cells_create(jfft_cells** out, const jfft_grid* grid, int max_cells, const jfft_options* opt);

/* mat->field: [n_cells][N] material fields (host or device memory per io_memory),
 * mapped by mat->kind with mat->e_max and mat->exponent; nu_cells and e_min_cells:
 * [n_cells] per-cell values in host memory, or NULL for mat->nu / mat->e_min.
 * eps_bar: [n_loads][3] Mandel strains (host memory).
 * Results (NULL entries skipped): res->u [n_cells][n_loads][2][N] zero-mean
 * displacement; res->C_hom [n_cells][3][n_loads]; res->iters and res->rel_res
 * [n_cells][n_loads] (true ||f - K u|| / ||f||). res->stress and
 * res->refine_steps are not written.
 * Returns JFFT_ERR_NOCONV / JFFT_ERR_BREAKDOWN if any (cell, load) did not
 * converge / broke down (all results are still written), JFFT_ERR_ARG for bad
 * arguments, JFFT_ERR_UNSUPPORTED for other preconditioners. */
jfft_status jfft_cells_solve(jfft_cells* h, int n_cells, const jfft_material* mat, const double* nu_cells,
                             const double* e_min_cells, int n_loads, const double* eps_bar, double tol,
                             jfft_precond pc, jfft_result* res);

void jfft_cells_destroy(jfft_cells* h);
const char* jfft_cells_last_error(const jfft_cells* h);
/* Kernel launches of this handle (one per jfft_cells_solve). */
int64_t jfft_cells_launch_count(const jfft_cells* h);

/* ---- request server with continuous batching ----
 *
 * Requests (grid, material field, load cases, tolerance, preconditioner and
 * precision; each one a jfft_solve of the paper's cell problem) are queued on
 * submission and run by max_active worker threads, each on its own CUDA stream, so
 * the GPU overlaps the work of every running request. A queued request starts when
 * a worker is free and its solver fits the device-memory budget: the workspace of
 * every live solver (running or idle) counts; idle solvers of the same grid shape
 * and precision are reused (material, Poisson ratio, Jacobi scaling and symbol are
 * re-set); idle solvers of other shapes are evicted, least recently used first.
 * Later requests that fit may start before an earlier one that does not. A result
 * is the same as the request's solve alone (same kernel sequence, deterministic).
 * The reference material is the mean material; max_loads is d(d+1)/2.
 */
typedef struct jfft_server jfft_server;

typedef struct {
  int max_active;            /* concurrent requests (worker threads / streams), 1..64 (default 4) */
  size_t hbm_budget;         /* device bytes the solvers may hold; 0 = 80 % of the free memory at creation */
  int device;                /* CUDA device ordinal (default 0) */
} jfft_server_options;

typedef struct {
  jfft_grid grid;
  jfft_material material;    /* field in host memory, copied at submission */
  int n_loads;               /* 1..d(d+1)/2 */
  const double* eps_bar;     /* [n_loads][d*] Mandel strains (host, copied) */
  double tol;
  int precond;               /* jfft_precond */
  int precision;             /* jfft_precision */
  int want_u;                /* 1: keep the displacement for jfft_server_wait */
} jfft_request;

typedef struct {
  int64_t submitted, finished, queued, running;
  size_t budget, used, peak_used;  /* bytes */
  int64_t solvers_created, solvers_reused, solvers_evicted;
} jfft_server_counters;

void jfft_server_default_options(jfft_server_options* opt);
jfft_status jfft_server_create(jfft_server** out, const jfft_server_options* opt);
/* Queues a request (inputs copied); *id receives its id. JFFT_ERR_OOM if its
 * solver can never fit the budget; JFFT_ERR_ARG / JFFT_ERR_UNSUPPORTED for bad
 * requests. Does not wait for the GPU. */
jfft_status jfft_server_submit(jfft_server* s, const jfft_request* req, int64_t* id);
/* 0 queued, 1 running, 2 finished, -1 unknown id. */
int jfft_server_poll(jfft_server* s, int64_t id);
/* Waits for request id, copies its results into res (host arrays with the layout of
 * jfft_solve; NULL entries skipped; u only if want_u), releases it and returns the
 * solve's status. timing (may be NULL): [4] = seconds queued, seconds running,
 * seconds from submission to completion, 1 if an idle solver was reused. */
jfft_status jfft_server_wait(jfft_server* s, int64_t id, jfft_result* res, double* timing);
jfft_status jfft_server_stats(jfft_server* s, jfft_server_counters* out);
const char* jfft_server_last_error(jfft_server* s);
/* Finishes the running requests, drops queued ones, frees every solver. */
void jfft_server_destroy(jfft_server* s);

/* ---- instrumentation ---- */

/* Number of kernels this handle has launched since creation (kernels inside a
 * replayed CUDA graph count once per replay). */
int64_t jfft_launch_count(const jfft_solver* h);

/* Number of PCG chunks this handle has run as a CUDA graph replay (options.graphs). */
int64_t jfft_graph_replays(const jfft_solver* h);

/* Launch shapes in use, tune[4] (0 = built-in default): node rows per warp segment of
 * the 2D operator {8, 16, 32, 64}; planes per segment of the 3D FP32 operator {4, 8, 16};
 * divisor of the lines per block of the forward row / inverse column FFT pass {1, 2, 4}.
 * jfft_set_tuning applies a saved choice (for example one found with options.autotune)
 * and drops captured graphs; JFFT_ERR_ARG for values outside those sets. */
jfft_status jfft_get_tuning(const jfft_solver* h, int* tune);
jfft_status jfft_set_tuning(jfft_solver* h, const int* tune);

/* When on, every kernel launch is bracketed by CUDA events on the handle's stream
 * and accumulated per kernel name; jfft_profile_json returns
 * {"kernel": [launches, total_ms], ...} (valid until the next call on h). */
jfft_status jfft_set_profiling(jfft_solver* h, int on);
const char* jfft_profile_json(jfft_solver* h);

/* Bytes of device workspace this handle holds. */
size_t jfft_workspace_bytes(const jfft_solver* h);

#ifdef __cplusplus
}
#endif
#endif /* JFFT_H */
