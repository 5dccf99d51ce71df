// Allocation-free variant of the CG operator step: y = K x and x . y for one field,
// with the per-CTA partial sums kept in a file-scope device array instead of a
// workspace allocated by jfft_create.
//
// Who needs it: callers that cannot call cudaMalloc / cudaFree, for example code
// that runs inside a framework which has already reserved the device memory for
// its own pool, or a latency-critical loop that must not take the implicit device
// synchronisation an allocation or a free can cause. They pass their own inputs
// and outputs and get the operator with no allocation at all.
#include "jfft.h"
#include "element.cuh"

#include <cmath>
#include <cstdint>
#include <mutex>

namespace {

// Partial sums of x . y, one per CTA of the operator launch. Every GPU that loads
// the library holds this array until the process exits.
constexpr int kNoAllocPartials = 8192;
static __device__ __align__(256) double g_noalloc_partials[kNoAllocPartials];

// Device address of g_noalloc_partials per device ordinal, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_ptr[kMaxDevices] = {};

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

// True if the byte ranges [a, a + na) and [b, b + nb) share any byte.
bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
  return pa < pb + nb && pb < pa + na;
}

}  // namespace

extern "C" jfft_status jfft_apply_K_dot_noalloc(const jfft_grid* grid, double nu, const double* E, const double* x,
                                                double* y, double* xy, void* stream) {
  using namespace jfft;
  if (!grid || !E || !x || !y || !xy) return JFFT_ERR_ARG;
  if (!(nu > -1.0 && nu < 0.5)) return JFFT_ERR_ARG;
  const int d = grid->dim;
  if (d != 2 && d != 3) return JFFT_ERR_ARG;
  const int nmax = d == 2 ? 2048 : 1024;
  Grid g = {};
  g.d = d;
  g.N = 1;
  double h[3];
  for (int a = 0; a < d; ++a) {
    const int64_t n = grid->n[a];
    if (!is_pow2(n) || n < 4 || n > nmax) return JFFT_ERR_UNSUPPORTED;
    g.n[a] = (int)n;
    int l = 0;
    while ((int64_t(1) << l) < n) ++l;
    g.log2n[a] = l;
    g.N *= n;
    h[a] = 1.0 / (double)n;
  }
  g.M = g.n[d - 1] / 2;
  g.F = g.N / g.n[d - 1] * (g.M + 1);
  // y is written while neighbouring blocks still read x (halo layers) and E, and the
  // kernel takes all three as non-aliasing: an in-place or overlapping call would be
  // silently wrong, so it is refused.
  const size_t field_bytes = sizeof(double) * (size_t)d * (size_t)g.N;
  const size_t e_bytes = sizeof(double) * (size_t)g.N;
  if (overlaps(y, field_bytes, x, field_bytes) || overlaps(y, field_bytes, E, e_bytes) ||
      overlaps(xy, sizeof(double), y, field_bytes) || overlaps(xy, sizeof(double), x, field_bytes) ||
      overlaps(xy, sizeof(double), E, e_bytes))
    return JFFT_ERR_ARG;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return JFFT_ERR_CUDA;
  double* partial = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
      // The current device is `dev`: its copy of the array is the one looked up.
      if (cudaGetSymbolAddress((void**)&g_ptr[dev], g_noalloc_partials) != cudaSuccess || !g_ptr[dev]) {
        g_ptr[dev] = nullptr;
        return JFFT_ERR_CUDA;
      }
    }
    partial = g_ptr[dev];
  }

  const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu = 1.0 / (2.0 * (1.0 + nu));
  const ElemConst ec = make_elem_const(d, h, lam, mu);
  cudaStream_t st = (cudaStream_t)stream;
  // Both launches report their own status; an error that earlier, unrelated work left
  // pending on this thread is neither read nor cleared here.
  int nparts = 0;
  cudaError_t e = launch_apply_K_dot_capped(g, ec, E, x, y, partial, kNoAllocPartials, &nparts, st);
  if (e != cudaSuccess) return JFFT_ERR_CUDA;
  if (nparts < 0) return JFFT_ERR_UNSUPPORTED;  // needs more partial sums than the array holds; nothing ran
  // Every slot the reduction reads was written by this call's operator launch, so
  // nothing in the shared array needs clearing first.
  e = launch_reduce_partials_own_status(partial, nparts, 1, kMaxPartials, xy, st);
  if (e != cudaSuccess) return JFFT_ERR_CUDA;
  return JFFT_OK;
}
