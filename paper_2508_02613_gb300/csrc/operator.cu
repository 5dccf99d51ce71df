// Operator-side kernels of the J-FFT solver: material (S1), matrix-free stiffness
// K = B^T W C B and the macro-strain load (S2, S3; paper Sec. 3.1 "Matrix-free
// assembly", Eq. lin_system_exp), element stress (S8), the Jacobi diagonal and
// Alg. 2 combs (S5), and the Alg. 1 impulse / inversion steps (S9).
#include "element.cuh"
#include "reduce.cuh"
#include <cuda_bf16.h>
#include <map>
#include <mutex>

namespace jfft {

// ------------------------------------------------------------------ S1
__global__ void k_material(const double* __restrict__ field, double* __restrict__ E, int64_t N, int kind,
                           double e_min, double e_max, double expo) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double v = field[i];
    E[i] = kind == 1 ? e_min + (e_max - e_min) * pow(v, expo) : v;
  }
}

// Counts entries that are negative or not finite (device-side validation of a
// material field given in device memory).
__global__ void k_check_field(const double* __restrict__ f, int64_t N, int* __restrict__ bad) {
  int local = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = f[i];
    local += (!isfinite(v) || v < 0.0) ? 1 : 0;
  }
  if (local) atomicAdd(bad, local);
}

cudaError_t launch_check_field(const double* f, int64_t N, int* bad, cudaStream_t st) {
  int blocks = (int)std::min<int64_t>((N + 255) / 256, 152 * 8);
  JFFT_K("check_field", st, k_check_field<<<blocks, 256, 0, st>>>(f, N, bad));
  return cudaGetLastError();
}

// Geometry G_p on the grid T_n (Sec. 4 "Discretization and grid refinement", n >= p):
// fine voxel I takes the value of the coarse pixel that contains it, index i_a >> s_a
// with s_a = log2(n_a / p_a) per axis.
__global__ void k_upsample(Grid g, int s0, int s1, int s2, const double* __restrict__ coarse, double* __restrict__ fine) {
  const int p1 = g.n[1] >> s1, p2 = g.d == 3 ? (g.n[2] >> s2) : 1;
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < g.N; I += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = I;
    int i2 = 0;
    if (g.d == 3) {
      i2 = (int)(r % g.n[2]);
      r /= g.n[2];
    }
    const int i1 = (int)(r % g.n[1]);
    const int i0 = (int)(r / g.n[1]);
    const int64_t c = ((int64_t)(i0 >> s0) * p1 + (i1 >> s1)) * p2 + (g.d == 3 ? (i2 >> s2) : 0);
    fine[I] = coarse[c];
  }
}

cudaError_t launch_upsample(const Grid& g, const int* shift, const double* coarse, double* fine, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((g.N + 255) / 256, 152 * 16);
  JFFT_K("upsample", st, k_upsample<<<blocks, 256, 0, st>>>(g, shift[0], shift[1], shift[2], coarse, fine));
  return cudaGetLastError();
}

cudaError_t launch_material(const double* field, double* E, int64_t N, int kind, double e_min, double e_max,
                            double expo, cudaStream_t st) {
  int blocks = (int)std::min<int64_t>((N + 255) / 256, 152 * 16);
  JFFT_K("material", st, k_material<<<blocks, 256, 0, st>>>(field, E, N, kind, e_min, e_max, expo));
  return cudaGetLastError();
}

// ------------------------------------------------------------------ S3 / S2
// Marching tile. The CTA owns an in-plane tile of P1 x P2 nodes (axes 1..d-1; P2 = 1
// in 2D) and walks `seg` node layers along axis 0. For element layer e0 it needs
// node layers e0 and e0 + 1 (a two-slot ring in shared memory, with a one-node halo
// on the low in-plane side and the high side), computes the (P1+1) x (P2+1) elements
// of the layer once each, scatters their corner forces through shared memory, and
// completes node layer e0 from the o0 = 0 corners plus the o0 = 1 corners of layer
// e0 - 1 carried in registers.
struct MarchGeom {
  int P1, P2;        // in-plane node tile (P2 = 1 in 2D)
  int seg;           // node layers per CTA
  int tiles1, tiles2;
};

template <int D> __host__ __device__ inline int plane_nodes(const MarchGeom& m) { return (m.P1 + 2) * (D == 3 ? m.P2 + 2 : 1); }
template <int D> __host__ __device__ inline int plane_elems(const MarchGeom& m) { return (m.P1 + 1) * (D == 3 ? m.P2 + 1 : 1); }

template <int D, typename T = double> static size_t march_smem(const MarchGeom& m) {
  const int pn = plane_nodes<D>(m), pe = plane_elems<D>(m);
  return sizeof(T) * (size_t(2) * D * pn + pe + size_t(D) * (1 << D) * pe);
}

// T: working precision of fields, material and constants (double or float); the
// dot partial is accumulated per thread in T and across the block in double.
// DOT: 0 none, 1 sum x.y, 2 sum y.y
// E in the working precision T, read from its stored type TE (T, or BF16 for the
// mixed-precision operator with a BF16 material copy).
template <typename T, typename TE> __device__ __forceinline__ T eload(const TE* __restrict__ E, int64_t i) {
  if constexpr (std::is_same<TE, __nv_bfloat16>::value) return (T)__bfloat162float(E[i]);
  else return (T)E[i];
}

template <typename T, int D, int DOT, bool HAS_X, bool HAS_E, bool SHIFT, typename TE = T>
__global__ void __launch_bounds__(384) k_apply_K(Grid g, MarchGeom mg, ElemConstT<T> ec, const TE* __restrict__ E,
                                                 T e_uniform, const T* __restrict__ x, T* __restrict__ y,
                                                 int64_t fstride, const StrainShift* __restrict__ shifts, T sgn,
                                                 double* __restrict__ partial, CgState* __restrict__ cg,
                                                 StageCtl sc) {
  constexpr int NC = 1 << D;
  constexpr int NCP = NC / 2;  // in-plane corners
  const int b = blockIdx.z;
  if (cg && cg[b].done) return;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm = reinterpret_cast<T*>(sm_raw);
  const int pn = plane_nodes<D>(mg), pe = plane_elems<D>(mg);
  T* ring = sm;                            // [2][D][pn]
  T* Es = ring + 2 * D * pn;               // [pe]
  T* Fs = Es + pe;                         // [D][2][NCP][pe]

  const int n0 = g.n[0], n1 = g.n[1], n2 = (D == 3 ? g.n[2] : 1);
  const int64_t plane = (int64_t)n1 * n2;
  const int t1 = blockIdx.x % mg.tiles1, t2 = blockIdx.x / mg.tiles1;
  const int i1s = t1 * mg.P1, i2s = (D == 3 ? t2 * mg.P2 : 0);
  const int L0 = blockIdx.y * mg.seg;
  const int W2 = (D == 3 ? mg.P2 + 2 : 1);   // halo tile width along axis 2 (nodes)
  const int E2 = (D == 3 ? mg.P2 + 1 : 1);   // element tile width along axis 2
  const T* xb = HAS_X ? x + (int64_t)b * fstride : nullptr;
  T* yb = y + (int64_t)b * fstride;
  StrainShift sh;
  if (SHIFT) sh = shifts[b];

  // thread -> owned in-plane node
  const int tid = threadIdx.x;
  const int own1 = (D == 3 ? tid / mg.P2 : tid), own2 = (D == 3 ? tid % mg.P2 : 0);
  const bool owner = tid < mg.P1 * (D == 3 ? mg.P2 : 1);

  auto load_layer = [&](int layer, int slot) {
    const int l = ((layer % n0) + n0) % n0;
    for (int idx = tid; idx < pn; idx += blockDim.x) {
      const int h1 = idx / W2, h2 = idx % W2;
      const int gi1 = (i1s - 1 + h1 + n1) % n1;
      const int gi2 = (D == 3 ? (i2s - 1 + h2 + n2) % n2 : 0);
      const int64_t node = (int64_t)l * plane + (int64_t)gi1 * n2 + gi2;
#pragma unroll
      for (int a = 0; a < D; ++a) ring[(slot * D + a) * pn + idx] = HAS_X ? xb[a * g.N + node] : T(0);
    }
  };

  T carry[D];
#pragma unroll
  for (int a = 0; a < D; ++a) carry[a] = T(0);
  T dot = T(0);

  if (HAS_X) load_layer(L0 - 1, (L0 - 1) & 1);
  for (int e0 = L0 - 1; e0 < L0 + mg.seg; ++e0) {
    if (HAS_X) load_layer(e0 + 1, (e0 + 1) & 1);
    if (HAS_E) {
      const int l = ((e0 % n0) + n0) % n0;
      for (int idx = tid; idx < pe; idx += blockDim.x) {
        const int h1 = idx / E2, h2 = idx % E2;
        const int gi1 = (i1s - 1 + h1 + n1) % n1;
        const int gi2 = (D == 3 ? (i2s - 1 + h2 + n2) % n2 : 0);
        Es[idx] = eload<T>(E, (int64_t)l * plane + (int64_t)gi1 * n2 + gi2);
      }
    }
    __syncthreads();
    const int s0 = e0 & 1, s1 = (e0 + 1) & 1;
    for (int idx = tid; idx < pe; idx += blockDim.x) {
      const int h1 = idx / E2, h2 = idx % E2;
      T u[D][NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int o0 = (c >> (D - 1)) & 1;
        const int o1 = (c >> (D - 2)) & 1;
        const int o2 = (D == 3 ? c & 1 : 0);
        const int node = (h1 + o1) * W2 + (h2 + o2);
#pragma unroll
        for (int a = 0; a < D; ++a) u[a][c] = HAS_X ? ring[((o0 ? s1 : s0) * D + a) * pn + node] : T(0);
      }
      const T Ee = HAS_E ? Es[idx] : e_uniform;
      element_force<D, T, SHIFT>(ec, &sh, u, Ee);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int o0 = (c >> (D - 1)) & 1;
        const int cin = c & (NCP - 1);
#pragma unroll
        for (int a = 0; a < D; ++a) Fs[((a * 2 + o0) * NCP + cin) * pe + idx] = u[a][c];
      }
    }
    __syncthreads();
    if (owner) {
#pragma unroll
      for (int a = 0; a < D; ++a) {
        T add0 = T(0), add1 = T(0);
#pragma unroll
        for (int cin = 0; cin < NCP; ++cin) {
          const int o1 = (D == 3 ? (cin >> 1) & 1 : cin & 1);
          const int o2 = (D == 3 ? cin & 1 : 0);
          const int el = (own1 + 1 - o1) * E2 + (D == 3 ? own2 + 1 - o2 : 0);
          add0 += Fs[((a * 2 + 0) * NCP + cin) * pe + el];
          add1 += Fs[((a * 2 + 1) * NCP + cin) * pe + el];
        }
        if (e0 >= L0) {
          const T q = sgn * (carry[a] + add0);
          const int l = e0;  // < n0 by construction
          const int64_t node = (int64_t)l * plane + (int64_t)(i1s + own1) * n2 + (D == 3 ? i2s + own2 : 0);
          yb[a * g.N + node] = q;
          if (DOT == 1) dot += ring[(s0 * D + a) * pn + (own1 + 1) * W2 + (D == 3 ? own2 + 1 : 0)] * q;
          if (DOT == 2) dot += q * q;
        }
        carry[a] = add1;
      }
    }
    __syncthreads();
  }
  if (DOT) {
    const double s = block_sum((double)dot);
    if (threadIdx.x == 0) partial[(int64_t)b * kMaxPartials + blockIdx.x + (int64_t)gridDim.x * blockIdx.y] = s;
    fused_stage_tail(sc, cg, b, partial + (int64_t)b * kMaxPartials, gridDim.x * gridDim.y);
  }
}

// Node layers [seg_begin(i, S, n0), seg_begin(i + 1, S, n0)) along axis 0 form segment i
// of S for the marching kernels (lengths n0 / S rounded down or up).
__host__ __device__ inline int seg_begin(int i, int S, int n0) { return (int)((int64_t)i * n0 / S); }

// Resident blocks per SM of a kernel launched with `threads` threads and no dynamic shared
// memory: the occupancy calculator's arithmetic (registers allocated per warp in units of
// 256, the SM's register, thread, block and shared-memory limits) from attribute queries
// only, the queries the FFT pass launchers also issue while a stream is being captured
// into a graph (a kernel's first use is often inside such a capture). 0 if a query fails.
static int resident_blocks_per_sm(const void* kern, int threads, int dev) {
  cudaFuncAttributes fa = {};
  int regs_sm = 0, thr_sm = 0, blk_sm = 0, smem_sm = 0;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int warps = (threads + 31) / 32;
  const int regs_warp = ((std::max(fa.numRegs, 1) * 32 + 255) / 256) * 256;
  int per_sm = std::min(blk_sm, thr_sm / (warps * 32));
  per_sm = std::min(per_sm, regs_sm / (regs_warp * warps));
  if (fa.sharedSizeBytes > 0) per_sm = std::min(per_sm, smem_sm / (int)fa.sharedSizeBytes);
  return std::max(per_sm, 0);
}

// Segments per (column group, load) of a marching launch: n0 / seg for the requested
// length; where the launch spans more than one wave of resident blocks, the count that
// fills a whole number of waves instead (the nearest, rounded down so that no block starts
// a last, nearly empty wave: a launch of 1.14 waves left most SMs idle for its tail); never
// more partial-sum slots than kMaxPartials. Resident blocks per (kernel, device) cached.
template <typename K> static int march_segments(K* kern, int threads, int ctas_x, int nb, int n0, int seg) {
  int S = std::max(1, n0 / seg);
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int64_t> cap_cache;
    int64_t cap = 0;
    {
      std::lock_guard<std::mutex> lock(mu);
      auto it = cap_cache.find({(const void*)kern, dev});
      if (it != cap_cache.end()) {
        cap = it->second;
      } else {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
          cap = (int64_t)sms * resident_blocks_per_sm((const void*)kern, threads, dev);
        cudaGetLastError();
        cap_cache[{(const void*)kern, dev}] = cap;
      }
    }
    const int64_t per_seg = (int64_t)ctas_x * nb;
    if (cap > 0 && per_seg * S > cap) {
      const int64_t waves = (per_seg * S + cap / 2) / cap;
      const int64_t s2 = waves * cap / per_seg;
      if (s2 >= 1) S = (int)std::min<int64_t>(s2, n0);
    }
  }
  if ((int64_t)ctas_x * S > kMaxPartials) S = std::max(1, kMaxPartials / ctas_x);
  return S;
}

// 2D operator, warp-marching form (no shared memory, no block barriers). Lane l of
// a warp owns node column c = c0 + l (mod n1, the contiguous axis) and walks `seg`
// node rows along axis 0. Per element row e0 it holds the node values of rows e0
// and e0 + 1 in registers, takes column c + 1 from lane l + 1 by a shuffle (lane 31
// loads that halo column itself), computes the element whose lowest corner is
// (e0, c), keeps the two corner forces of its own column and hands the two of
// column c + 1 to lane l + 1 by a shuffle. Node (e0, c) is then complete for lanes
// 1..31, so warps overlap by one column (stride 31): outputs o = 31 w + l, l >= 1.
constexpr int kWarpStride = 31;
// Warps per block: FP32 runs four-warp blocks; FP64 (bound by FP64 issue) runs one-warp
// blocks, whose finer grid spreads the work evenly over the SMs (with four-warp blocks
// the 1024^2 launch left the SMs idle for 12 % of its cycles; measured 367 -> 338 us per
// 3-load launch).
template <typename T> constexpr int k2d_warps() { return sizeof(T) == 8 ? 1 : 4; }

// HAS_X = false: x = 0 (right-hand side); SHIFT: the load's macroscopic strain is added
// to the element modes; the output is sgn * (K x + K_shift).
// P1: the voxel is two linear triangles (tri_pair_force) instead of the Q1 element.
template <typename T, int DOT, bool HAS_E, bool HAS_X, bool SHIFT, bool P1, typename TE = T>
__global__ void __launch_bounds__(32 * k2d_warps<T>())
    k_apply_K2d(Grid g, ElemConstT<T> ec, const TE* __restrict__ E, T e_uniform, const T* __restrict__ x,
                T* __restrict__ y, int64_t fstride, int groups, const StrainShift* __restrict__ shifts,
                T sgn, double* __restrict__ partial, CgState* __restrict__ cg, StageCtl sc) {
  const int b = blockIdx.z;
  if (cg && cg[b].done) return;
  StrainShift sh;
  if (SHIFT) sh = shifts[b];
  const int n0 = g.n[0], n1 = g.n[1];
  const int lane = threadIdx.x & 31;
  const int grp = blockIdx.x * k2d_warps<T>() + (threadIdx.x >> 5);
  const bool active_warp = grp < groups;
  const int o = grp * kWarpStride + lane;                  // output index before wrapping
  const int c = o % n1, cr = (o + 1) % n1;                 // own column, halo column (lane 31)
  const bool writer = active_warp && lane >= 1 && o <= n1;
  const int ocol = o % n1;
  const T* xb = x + (int64_t)b * fstride;
  T* yb = y + (int64_t)b * fstride;
  const int L0 = seg_begin(blockIdx.y, gridDim.y, n0), L1 = seg_begin(blockIdx.y + 1, gridDim.y, n0);
  T dot = T(0);
  if (active_warp) {
    T lo[2], hi[2], rlo[2], rhi[2], carry[2];
    T nx[2], nh[2];  // node row e0 + 2 (own column, halo column), loaded one step ahead
    T En = T(0);     // element row e0 + 1, loaded one step ahead
    {
      const int row = (L0 - 1 + n0) % n0;
      const int rown = L0 % n0;
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        lo[a] = HAS_X ? xb[a * g.N + (int64_t)row * n1 + c] : T(0);
        const T hlo = (HAS_X && lane == 31) ? xb[a * g.N + (int64_t)row * n1 + cr] : T(0);
        rlo[a] = __shfl_down_sync(0xffffffffu, lo[a], 1);
        if (lane == 31) rlo[a] = hlo;
        nx[a] = HAS_X ? xb[a * g.N + (int64_t)rown * n1 + c] : T(0);
        nh[a] = (HAS_X && lane == 31) ? xb[a * g.N + (int64_t)rown * n1 + cr] : T(0);
        carry[a] = T(0);
      }
      if (HAS_E) En = eload<T>(E, (int64_t)row * n1 + c);
    }
    for (int e0 = L0 - 1; e0 < L1; ++e0) {
      const T Ee = HAS_E ? En : e_uniform;
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        hi[a] = nx[a];
        rhi[a] = __shfl_down_sync(0xffffffffu, hi[a], 1);
        if (lane == 31) rhi[a] = nh[a];
      }
      if (e0 + 1 < L1) {                 // prefetch node row e0 + 2 and element row e0 + 1
        const int rn2 = (e0 + 2) & (n0 - 1);   // n0 is a power of two
        const int re1 = (e0 + 1) & (n0 - 1);
        if (HAS_X) {
#pragma unroll
          for (int a = 0; a < 2; ++a) {
            nx[a] = xb[a * g.N + (int64_t)rn2 * n1 + c];
            nh[a] = lane == 31 ? xb[a * g.N + (int64_t)rn2 * n1 + cr] : T(0);
          }
        }
        if (HAS_E) En = eload<T>(E, (int64_t)re1 * n1 + c);
      }
      T u[2][4];
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        u[a][0] = lo[a];   // corner (0, 0): node (e0, c)
        u[a][1] = rlo[a];  // corner (0, 1): node (e0, c + 1)
        u[a][2] = hi[a];   // corner (1, 0): node (e0 + 1, c)
        u[a][3] = rhi[a];  // corner (1, 1): node (e0 + 1, c + 1)
      }
      if (P1) tri_pair_force<T, SHIFT>(ec, &sh, u, Ee);
      else element_force<2, T, SHIFT>(ec, &sh, u, Ee);
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const T from_left_lo = __shfl_up_sync(0xffffffffu, u[a][1], 1);
        const T from_left_hi = __shfl_up_sync(0xffffffffu, u[a][3], 1);
        if (e0 >= L0 && writer) {
          const T sum = carry[a] + u[a][0] + from_left_lo;
          const T q = SHIFT ? sgn * sum : sum;  // sgn is 1 for the forms without a strain shift
          yb[a * g.N + (int64_t)e0 * n1 + ocol] = q;
          if (DOT == 1) dot += lo[a] * q;
          if (DOT == 2) dot += q * q;
        }
        carry[a] = u[a][2] + from_left_hi;
        lo[a] = hi[a];
        rlo[a] = rhi[a];
      }
    }
  }
  if (DOT) {
    const double s = block_sum((double)dot);
    if (threadIdx.x == 0) partial[(int64_t)b * kMaxPartials + blockIdx.x + (int64_t)gridDim.x * blockIdx.y] = s;
    fused_stage_tail(sc, cg, b, partial + (int64_t)b * kMaxPartials, gridDim.x * gridDim.y);
  }
}

template <typename T, int DOT, bool HAS_E, bool HAS_X = true, bool SHIFT = false, typename TE = T>
static cudaError_t apply_K2d_t(const Grid& g, const ElemConstT<T>& ec, const TE* E, T e_uniform, const T* x, T* y, int nb,
                               int64_t fstride, double* partial, int* nparts, CgState* cg, cudaStream_t st,
                               StageCtl sc, const StrainShift* shifts = nullptr, T sgn = T(1)) {
  const int groups = (g.n[1] + kWarpStride - 1) / kWarpStride;
  const int ctas_x = (groups + k2d_warps<T>() - 1) / k2d_warps<T>();
  const int seg = std::min(g.n[0], g.tune[0] > 0 ? g.tune[0] : 16);
  const char* name = sizeof(T) == 4 ? (DOT == 1 ? "apply_K_f32" : "apply_K_f32_plain")
                     : DOT == 1 ? "apply_K"
                     : (!HAS_X ? "apply_K_rhs" : (SHIFT ? "apply_K_residual" : (HAS_E ? "apply_K_plain" : "apply_K_ref")));
  auto kern = ec.elem == 1 ? k_apply_K2d<T, DOT, HAS_E, HAS_X, SHIFT, true, TE>
                           : k_apply_K2d<T, DOT, HAS_E, HAS_X, SHIFT, false, TE>;
  const dim3 grid(ctas_x, march_segments(kern, 32 * k2d_warps<T>(), ctas_x, nb, g.n[0], seg), nb);
  JFFT_K(name, st, kern<<<grid, 32 * k2d_warps<T>(), 0, st>>>(g, ec, E, e_uniform, x, y, fstride, groups, shifts, sgn,
                                                               partial, cg, sc));
  if (nparts) *nparts = grid.x * grid.y;
  return cudaGetLastError();
}

// Launch shape of the 3D marching kernel below (measured on GB300 at 128^3 x 6 loads and
// 512^3: J = 4 node rows per warp, four resident blocks per SM in FP32 and two in FP64,
// 8-plane segments; the per-node summation order does not depend on these).
constexpr int kWarpsPerCta3d = 4;
#ifndef JFFT_K3S_J
#define JFFT_K3S_J 4
#endif
#ifndef JFFT_K3S_SEG
#define JFFT_K3S_SEG 8
#endif
#ifndef JFFT_K3S_MINB
#define JFFT_K3S_MINB 4
#endif
#ifndef JFFT_K3S_MINB64
#define JFFT_K3S_MINB64 2
#endif

// FP64 instances hold every value in two registers: two resident blocks per SM (255 registers).
template <typename T> constexpr int k3d_min_blocks() { return sizeof(T) == 8 ? JFFT_K3S_MINB64 : JFFT_K3S_MINB; }

// 3D operator, separable warp-marching form. The element transform of element_force
// (corner values -> Walsh-Hadamard modes -> mode forces -> corner forces) is split by
// axis so that the butterfly stages shared by neighbouring elements run once:
//   forward: the plane stage (axis 0: u(e0+1) +- u(e0)) once per node, the row stage
//   (axis 1) once per (row pair, column), the column stage (axis 2) per element with the
//   right column's row-stage values from lane l + 1;
//   backward: the column stage per element, the right column's half sent to lane l + 1
//   and added there (the node-column sum), the row stage per (row pair, column), the
//   node-row sum over the two element rows, then the plane stage once per node, whose
//   e0 + 1 half is carried to the next plane step.
// Lane l of warp w owns node column c = 30 w + l (columns wrap periodically); lanes 0..30
// compute the elements whose corner columns are c and c + 1, lanes 1..30 write node
// column c (stride 30: every element a warp needs has both columns inside the warp, no
// halo loads). A warp covers node rows j0 .. j0 + J - 1 along axis 1 (element rows j0 - 1
// .. j0 + J - 1) and marches planes e0 = L0 - 1 .. L0 + seg - 1 along axis 0; the values of
// plane e0 + 1 stay in registers for the next step, so each node is loaded once per
// segment. Same mode arithmetic as element_force (mode_forces, E scaling with the
// force-free mode 0 left out, the optional strain shift), different association order.
constexpr int kColsPerWarp3s = 30;

template <typename T, int J, int DOT, bool HAS_E, bool HAS_X, bool SHIFT, typename TE = T>
__global__ void __launch_bounds__(32 * kWarpsPerCta3d, k3d_min_blocks<T>())
    k_apply_K3s(Grid g, ElemConstT<T> ec, const TE* __restrict__ E, T e_uniform, const T* __restrict__ x,
                T* __restrict__ y, int64_t fstride, int groups2, int rowblocks,
                const StrainShift* __restrict__ shifts, T sgn, double* __restrict__ partial,
                CgState* __restrict__ cg, StageCtl sc) {
  const int b = blockIdx.z;
  if (cg && cg[b].done) return;
  StrainShift sh;
  if (SHIFT) sh = shifts[b];
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const int64_t N = g.N;
  const int lane = threadIdx.x & 31;
  const int wid = blockIdx.x * kWarpsPerCta3d + (threadIdx.x >> 5);
  const bool active_warp = wid < groups2 * rowblocks;
  const int g2 = active_warp ? wid % groups2 : 0;
  const int j0 = active_warp ? (wid / groups2) * J : 0;
  const int cu = g2 * kColsPerWarp3s + lane;  // column before wrapping
  const int c = cu & (n2 - 1);
  const bool writer = active_warp && lane >= 1 && lane <= kColsPerWarp3s && cu <= n2;
  const T* xb = x + (int64_t)b * fstride;
  T* yb = y + (int64_t)b * fstride;
  const int L0 = seg_begin(blockIdx.y, gridDim.y, n0), L1 = seg_begin(blockIdx.y + 1, gridDim.y, n0);
  constexpr int R = J + 2;  // node rows j0 - 1 .. j0 + J
  T dot = T(0);
  if (active_warp) {
    int roff[R];  // offset of node row j0 - 1 + i within a plane, own column (a plane has < 2^31 nodes)
#pragma unroll
    for (int i = 0; i < R; ++i) roff[i] = ((j0 - 1 + i) & (n1 - 1)) * n2 + c;
    T A[R][3];  // plane e0, own column
    {
      const int64_t pb = (int64_t)((L0 - 1) & (n0 - 1)) * n1 * n2;
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int a = 0; a < 3; ++a) A[i][a] = HAS_X ? xb[a * N + pb + roff[i]] : T(0);
    }
    T carry[J][3];
#pragma unroll
    for (int i = 0; i < J; ++i)
#pragma unroll
      for (int a = 0; a < 3; ++a) carry[i][a] = T(0);
    for (int e0 = L0 - 1; e0 < L1; ++e0) {
      const int64_t pb0 = (int64_t)(e0 & (n0 - 1)) * n1 * n2;
      const int64_t pb1 = (int64_t)((e0 + 1) & (n0 - 1)) * n1 * n2;
      // node row 0 of the sweep (j0 - 1): plane stage
      T Sb[3], Db[3], Xb[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const T v1 = HAS_X ? xb[a * N + pb1 + roff[0]] : T(0);
        Sb[a] = v1 + A[0][a];
        Db[a] = v1 - A[0][a];
        Xb[a] = A[0][a];
        A[0][a] = v1;
      }
      T racc[3][2];  // node row being summed: plane-stage modes (sum, difference)
#pragma unroll
      for (int k = 0; k <= J; ++k) {  // element row e1 = j0 - 1 + k: node rows k (bottom), k + 1 (top)
        T St[3], Dt[3], Xt[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const T v1 = HAS_X ? xb[a * N + pb1 + roff[k + 1]] : T(0);
          St[a] = v1 + A[k + 1][a];
          Dt[a] = v1 - A[k + 1][a];
          Xt[a] = A[k + 1][a];
          A[k + 1][a] = v1;
        }
        // row stage, then column stage with lane l + 1: modes W[a][m], m bits (axis0 4, axis1 2, axis2 1)
        T W[3][8];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const T v0 = St[a] + Sb[a], v2 = St[a] - Sb[a], v4 = Dt[a] + Db[a], v6 = Dt[a] - Db[a];
          const T r0 = __shfl_down_sync(0xffffffffu, v0, 1), r2 = __shfl_down_sync(0xffffffffu, v2, 1);
          const T r4 = __shfl_down_sync(0xffffffffu, v4, 1), r6 = __shfl_down_sync(0xffffffffu, v6, 1);
          W[a][0] = r0 + v0; W[a][1] = r0 - v0;
          W[a][2] = r2 + v2; W[a][3] = r2 - v2;
          W[a][4] = r4 + v4; W[a][5] = r4 - v4;
          W[a][6] = r6 + v6; W[a][7] = r6 - v6;
        }
        if (SHIFT) {
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int bb = 0; bb < 3; ++bb) W[a][mbit<3>(bb)] += T(sh.s[a][bb]);
        }
        const int e1 = j0 - 1 + k;
        const T Ee = HAS_E ? eload<T>(E, pb0 + (int64_t)(e1 & (n1 - 1)) * n2 + c) : e_uniform;
        T F[3][8];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int m = 0; m < 8; ++m) F[a][m] = T(0);
        mode_forces<3>(ec, W, F);
        // backward: column stage (own half o2 = 0, right half o2 = 1 to lane l + 1), then row stage
        T top[3][2];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          T Q[4];  // modes over (axis0, axis1): index (m >> 1)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int m = 2 * q;
            const T y0 = m == 0 ? T(0) : F[a][m] * Ee, y1 = F[a][m | 1] * Ee;
            const T own = y0 - y1, right = y0 + y1;
            Q[q] = own + __shfl_up_sync(0xffffffffu, right, 1);
          }
          // row stage: bottom node row (o1 = 0) and top node row (o1 = 1), per plane mode
          const T bot0 = Q[0] - Q[1], top0 = Q[0] + Q[1];   // plane-sum mode (axis0 bit clear)
          const T bot1 = Q[2] - Q[3], top1 = Q[2] + Q[3];   // plane-difference mode
          top[a][0] = top0;
          top[a][1] = top1;
          if (k >= 1) {
            // node row j0 - 1 + k complete: plane stage -> planes e0 (o0 = 0) and e0 + 1 (o0 = 1)
            const T t0 = racc[a][0] + bot0, t1 = racc[a][1] + bot1;
            const T f0 = t0 - t1, f1 = t0 + t1;
            if (e0 >= L0 && writer) {
              const T sum = carry[k - 1][a] + f0;
              const T q = SHIFT ? sgn * sum : sum;
              yb[a * N + pb0 + roff[k]] = q;
              if (DOT == 1) dot += Xb[a] * q;
              if (DOT == 2) dot += q * q;
            }
            carry[k - 1][a] = f1;
          }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          racc[a][0] = top[a][0];
          racc[a][1] = top[a][1];
          Sb[a] = St[a];
          Db[a] = Dt[a];
          Xb[a] = Xt[a];
        }
      }
    }
  }
  if (DOT) {
    const double s = block_sum((double)dot);
    if (threadIdx.x == 0) partial[(int64_t)b * kMaxPartials + blockIdx.x + (int64_t)gridDim.x * blockIdx.y] = s;
    fused_stage_tail(sc, cg, b, partial + (int64_t)b * kMaxPartials, gridDim.x * gridDim.y);
  }
}

template <typename T, int J, int DOT, bool HAS_E, bool HAS_X = true, bool SHIFT = false, typename TE = T>
static cudaError_t apply_K3s_t(const Grid& g, const ElemConstT<T>& ec, const TE* E, T e_uniform, const T* x, T* y, int nb,
                               int64_t fstride, double* partial, int* nparts, CgState* cg, cudaStream_t st,
                               StageCtl sc, const StrainShift* shifts = nullptr, T sgn = T(1)) {
  const int groups2 = (g.n[2] + kColsPerWarp3s - 1) / kColsPerWarp3s;
  const int rowblocks = g.n[1] / J;
  const int warps = groups2 * rowblocks;
  const int ctas_x = (warps + kWarpsPerCta3d - 1) / kWarpsPerCta3d;
  const int seg = std::min(g.n[0], g.tune[1] > 0 ? g.tune[1] : JFFT_K3S_SEG);
  auto kern = k_apply_K3s<T, J, DOT, HAS_E, HAS_X, SHIFT, TE>;
  const dim3 grid(ctas_x, march_segments(kern, 32 * kWarpsPerCta3d, ctas_x, nb, g.n[0], seg), nb);
  const char* name = sizeof(T) == 4 ? (DOT == 1 ? "apply_K_f32" : "apply_K_f32_plain")
                     : DOT == 1 ? "apply_K"
                     : (!HAS_X ? "apply_K_rhs" : (SHIFT ? "apply_K_residual" : (HAS_E ? "apply_K_plain" : "apply_K_ref")));
  JFFT_K(name, st, kern<<<grid, 32 * kWarpsPerCta3d, 0, st>>>(g, ec, E, e_uniform, x, y, fstride, groups2, rowblocks,
                                                              shifts, sgn, partial, cg, sc));
  if (nparts) *nparts = grid.x * grid.y;
  return cudaGetLastError();
}

template <int D> static MarchGeom march_geom(const Grid& g) {
  MarchGeom m;
  if (D == 2) {
    m.P1 = std::min(g.n[1], 256);
    m.P2 = 1;
  } else {
    m.P2 = std::min(g.n[2], 32);
    m.P1 = std::min(g.n[1], 256 / m.P2);
  }
  m.tiles1 = g.n[1] / m.P1;
  m.tiles2 = (D == 3 ? g.n[2] / m.P2 : 1);
  const int tiles = m.tiles1 * m.tiles2;
  int seg = std::min(g.n[0], 16);
  while ((int64_t)tiles * (g.n[0] / seg) > kMaxPartials) seg *= 2;
  m.seg = seg;
  return m;
}

template <typename T, int D, int DOT, bool HAS_X, bool HAS_E, bool SHIFT, typename TE = T>
static cudaError_t apply_K_t(const Grid& g, const ElemConstT<T>& ec, const TE* E, T e_uniform, const T* x,
                             T* y, int nb, int64_t fstride, const StrainShift* shifts, T sgn, double* partial,
                             int* nparts, CgState* cg, cudaStream_t st, StageCtl sc) {
  MarchGeom m = march_geom<D>(g);
  const size_t smem = march_smem<D, T>(m);
  auto kern = k_apply_K<T, D, DOT, HAS_X, HAS_E, SHIFT, TE>;
  cudaError_t e = allow_dynamic_smem(kern, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(m.tiles1 * m.tiles2, g.n[0] / m.seg, nb);
  // one element per thread per layer; warps round up (owners are the first P1*P2)
  const int threads = ((std::max(plane_elems<D>(m), m.P1 * m.P2) + 31) / 32) * 32;
  const char* kname = sizeof(T) == 4 ? (DOT == 1 ? "apply_K_f32" : "apply_K_f32_plain") : DOT == 1 ? "apply_K"
                      : (!HAS_X ? "apply_K_rhs" : (SHIFT ? "apply_K_residual" : (HAS_E ? "apply_K_plain" : "apply_K_ref")));
  JFFT_K(kname, st, kern<<<grid, threads, smem, st>>>(g, m, ec, E, e_uniform, x, y, fstride, shifts, sgn, partial, cg, sc));
  if (nparts) *nparts = grid.x * grid.y;
  return cudaGetLastError();
}

template <int D>
static cudaError_t apply_K_d(const Grid& g, const ElemConst& ec, const double* E, double e_uniform, const double* x,
                             double* y, int nb, int64_t fstride, const StrainShift* shifts, double sgn, int dot_mode,
                             double* partial, int* nparts, CgState* cg, cudaStream_t st, StageCtl sc) {
  const bool hx = x != nullptr, he = E != nullptr, sh = shifts != nullptr;
  if (D == 2) {
    if (hx && !sh && sgn == 1.0) {
      if (dot_mode == 1 && he) return apply_K2d_t<double, 1, true>(g, ec, E, e_uniform, x, y, nb, fstride, partial, nparts, cg, st, sc);
      if (dot_mode == 0 && he) return apply_K2d_t<double, 0, true>(g, ec, E, e_uniform, x, y, nb, fstride, partial, nparts, cg, st, sc);
      if (dot_mode == 0 && !he) return apply_K2d_t<double, 0, false>(g, ec, E, e_uniform, x, y, nb, fstride, partial, nparts, cg, st, sc);
    }
    // right-hand side (x = 0) and true residual, with the strain shift, ||y||^2 or none
    if (he && sh && (dot_mode == 2 || dot_mode == 0)) {
      if (!hx && dot_mode == 2) return apply_K2d_t<double, 2, true, false, true>(g, ec, E, e_uniform, x, y, nb, fstride, partial, nparts, cg, st, sc, shifts, sgn);
      if (!hx && dot_mode == 0) return apply_K2d_t<double, 0, true, false, true>(g, ec, E, e_uniform, x, y, nb, fstride, partial, nparts, cg, st, sc, shifts, sgn);
      if (hx && dot_mode == 2) return apply_K2d_t<double, 2, true, true, true>(g, ec, E, e_uniform, x, y, nb, fstride, partial, nparts, cg, st, sc, shifts, sgn);
      if (hx && dot_mode == 0) return apply_K2d_t<double, 0, true, true, true>(g, ec, E, e_uniform, x, y, nb, fstride, partial, nparts, cg, st, sc, shifts, sgn);
    }
  }
  if (ec.elem != 0) return cudaErrorInvalidValue;  // P1 voxels run only on the 2D warp kernel
  // 3D FP64: the separable marching kernel (128^3: 6.7 against 7.8 ms per operator
  // application for the shared-memory tile kernel below, 512^3: 70 against 89 ms); the tile
  // kernel keeps the grids with fewer than JFFT_K3S_J rows and the right-hand side form
  if (D == 3 && g.n[1] >= JFFT_K3S_J) {
    if (hx && he && !sh && dot_mode == 1)
      return apply_K3s_t<double, JFFT_K3S_J, 1, true, true, false>(g, ec, E, e_uniform, x, y, nb, fstride, partial,
                                                                   nparts, cg, st, sc);
    if (hx && he && !sh && dot_mode == 0)
      return apply_K3s_t<double, JFFT_K3S_J, 0, true, true, false>(g, ec, E, e_uniform, x, y, nb, fstride, partial,
                                                                   nparts, cg, st, sc);
    if (hx && he && sh && dot_mode == 2)
      return apply_K3s_t<double, JFFT_K3S_J, 2, true, true, true>(g, ec, E, e_uniform, x, y, nb, fstride, partial,
                                                                  nparts, cg, st, sc, shifts, sgn);
  }
#define JFFT_AK(DOT, HX, HE, SH) \
  if (dot_mode == DOT && hx == HX && he == HE && sh == SH) \
    return apply_K_t<double, D, DOT, HX, HE, SH>(g, ec, E, e_uniform, x, y, nb, fstride, shifts, sgn, partial, nparts, cg, st, sc);
  JFFT_AK(1, true, true, false)   // CG: q = K p, p.q
  JFFT_AK(0, true, true, false)   // plain apply
  JFFT_AK(0, true, false, false)  // reference operator (uniform E)
  JFFT_AK(2, false, true, true)   // load: f = -B^T W C eps_bar, ||f||^2
  JFFT_AK(2, true, true, true)    // true residual, ||r||^2
  JFFT_AK(0, false, true, true)
  JFFT_AK(0, true, true, true)
#undef JFFT_AK
  return cudaErrorInvalidValue;
}

cudaError_t launch_apply_K(const Grid& g, const ElemConst& ec, const double* E, double e_uniform, const double* x,
                           double* y, int nb, int64_t field_stride, const StrainShift* shifts, double sgn, int dot_mode,
                           double* partial, int* nparts, CgState* done, cudaStream_t st, StageCtl sc) {
  if (g.d == 2)
    return apply_K_d<2>(g, ec, E, e_uniform, x, y, nb, field_stride, shifts, sgn, dot_mode, partial, nparts, done, st, sc);
  return apply_K_d<3>(g, ec, E, e_uniform, x, y, nb, field_stride, shifts, sgn, dot_mode, partial, nparts, done, st, sc);
}

// The CG operator variant (y = K x with per-CTA partial sums of x.y) for a caller
// that supplies its own partial-sum buffer with room for `cap` entries: the march
// segment is lengthened until the CTA count fits and nparts receives that count;
// if even a full-length march needs more than `cap`, nparts receives -1 and nothing
// is launched. The returned status is this call's own (cudaLaunchKernelEx reports
// the launch's error directly, so an error left pending by earlier, unrelated work
// is neither read nor cleared).
template <int D>
static cudaError_t apply_K_dot_capped_t(const Grid& g, const ElemConst& ec, const double* E, const double* x,
                                        double* y, double* partial, int cap, int* nparts, cudaStream_t st) {
  MarchGeom m = march_geom<D>(g);
  const int64_t tiles = (int64_t)m.tiles1 * m.tiles2;
  while (tiles * (g.n[0] / m.seg) > cap && m.seg < g.n[0]) m.seg *= 2;
  if (tiles * (g.n[0] / m.seg) > cap) {
    *nparts = -1;
    return cudaSuccess;
  }
  const size_t smem = march_smem<D>(m);
  auto kern = k_apply_K<double, D, 1, true, true, false>;
  cudaError_t e = allow_dynamic_smem(kern, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(m.tiles1 * m.tiles2, g.n[0] / m.seg, 1);
  cfg.blockDim = dim3(((std::max(plane_elems<D>(m), m.P1 * m.P2) + 31) / 32) * 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  const ElemConstT<double> ecd = ec;
  const StrainShift* no_shift = nullptr;
  CgState* no_cg = nullptr;
  JFFT_K("apply_K_dot_capped", st,
         e = cudaLaunchKernelEx(&cfg, kern, g, m, ecd, E, 0.0, x, y, (int64_t)0, no_shift, 1.0, partial, no_cg,
                                no_stage()));
  *nparts = (int)(cfg.gridDim.x * cfg.gridDim.y);
  return e;
}

cudaError_t launch_apply_K_dot_capped(const Grid& g, const ElemConst& ec, const double* E, const double* x, double* y,
                                      double* partial, int cap, int* nparts, cudaStream_t st) {
  if (g.d == 2) return apply_K_dot_capped_t<2>(g, ec, E, x, y, partial, cap, nparts, st);
  return apply_K_dot_capped_t<3>(g, ec, E, x, y, partial, cap, nparts, st);
}

// Working-precision FP32 operator (mixed-precision inner solve): y = K x with the
// material in FP32, optional fused x.y partials (dot_mode 1) or none (0).
template <int D, typename TE>
static cudaError_t apply_K_f32_d(const Grid& g, const ElemConstT<float>& ec, const TE* E, const float* x, float* y,
                                 int nb, int64_t fstride, int dot_mode, double* partial, int* nparts, CgState* cg,
                                 cudaStream_t st, StageCtl sc) {
  if (D == 2) {
    if (dot_mode == 1)
      return apply_K2d_t<float, 1, true, true, false, TE>(g, ec, E, 0.f, x, y, nb, fstride, partial, nparts, cg, st, sc);
    return apply_K2d_t<float, 0, true, true, false, TE>(g, ec, E, 0.f, x, y, nb, fstride, partial, nparts, cg, st, sc);
  }
  if (g.n[1] >= JFFT_K3S_J) {
    if (dot_mode == 1)
      return apply_K3s_t<float, JFFT_K3S_J, 1, true, true, false, TE>(g, ec, E, 0.f, x, y, nb, fstride, partial, nparts,
                                                                      cg, st, sc);
    return apply_K3s_t<float, JFFT_K3S_J, 0, true, true, false, TE>(g, ec, E, 0.f, x, y, nb, fstride, partial, nparts,
                                                                    cg, st, sc);
  }
  if (dot_mode == 1)
    return apply_K_t<float, D, 1, true, true, false, TE>(g, ec, E, 0.f, x, y, nb, fstride, nullptr, 1.f, partial, nparts,
                                                         cg, st, sc);
  return apply_K_t<float, D, 0, true, true, false, TE>(g, ec, E, 0.f, x, y, nb, fstride, nullptr, 1.f, partial, nparts,
                                                       cg, st, sc);
}

cudaError_t launch_apply_K_f32(const Grid& g, const ElemConst& ec, const float* E, const float* x, float* y, int nb,
                               int64_t field_stride, int dot_mode, double* partial, int* nparts, CgState* cg,
                               cudaStream_t st, StageCtl sc) {
  const ElemConstT<float> ecf = elem_const_as<float>(ec);
  if (g.d == 2) return apply_K_f32_d<2>(g, ecf, E, x, y, nb, field_stride, dot_mode, partial, nparts, cg, st, sc);
  return apply_K_f32_d<3>(g, ecf, E, x, y, nb, field_stride, dot_mode, partial, nparts, cg, st, sc);
}

cudaError_t launch_apply_K_f32_bf16(const Grid& g, const ElemConst& ec, const void* E16, const float* x, float* y,
                                    int nb, int64_t field_stride, int dot_mode, double* partial, int* nparts,
                                    CgState* cg, cudaStream_t st, StageCtl sc) {
  const ElemConstT<float> ecf = elem_const_as<float>(ec);
  const __nv_bfloat16* E = static_cast<const __nv_bfloat16*>(E16);
  if (g.d == 2) return apply_K_f32_d<2>(g, ecf, E, x, y, nb, field_stride, dot_mode, partial, nparts, cg, st, sc);
  return apply_K_f32_d<3>(g, ecf, E, x, y, nb, field_stride, dot_mode, partial, nparts, cg, st, sc);
}

// E16[i] = E[i] rounded to BF16 (round to nearest even)
__global__ void k_to_bf16(const double* __restrict__ E, __nv_bfloat16* __restrict__ E16, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    E16[i] = __double2bfloat16(E[i]);
}

cudaError_t launch_to_bf16(const double* E, void* E16, int64_t n, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  JFFT_K("to_bf16", st, k_to_bf16<<<blocks, 256, 0, st>>>(E, static_cast<__nv_bfloat16*>(E16), n));
  return cudaGetLastError();
}

// ------------------------------------------------------------------ S8
template <int D>
__global__ void __launch_bounds__(256) k_stress(Grid g, ElemConst ec, const double* __restrict__ E,
                                                const double* __restrict__ u, const StrainShift* __restrict__ shifts,
                                                double* __restrict__ stress, double* __restrict__ partial) {
  constexpr int NC = 1 << D;
  constexpr int DS = D * (D + 1) / 2;
  const int b = blockIdx.y;
  const double* ub = u + (int64_t)b * D * g.N;
  double acc[DS];
#pragma unroll
  for (int s = 0; s < DS; ++s) acc[s] = 0.0;
  const StrainShift sh = shifts[b];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < g.N; e += (int64_t)gridDim.x * blockDim.x) {
    int idx[3];
    int64_t r = e;
    for (int a = D - 1; a >= 0; --a) { idx[a] = (int)(r % g.n[a]); r /= g.n[a]; }
    double uc[D][NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      int64_t node = 0;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int o = (c >> (D - 1 - a)) & 1;
        node = node * g.n[a] + (idx[a] + o) % g.n[a];
      }
#pragma unroll
      for (int a = 0; a < D; ++a) uc[a][c] = ub[a * g.N + node];
    }
    double sig[6];
    if constexpr (D == 2) {
      if (ec.elem == 1) tri_pair_stress(ec, &sh, uc, E[e], sig);
      else element_stress<D>(ec, &sh, uc, E[e], sig);
    } else {
      element_stress<D>(ec, &sh, uc, E[e], sig);
    }
#pragma unroll
    for (int s = 0; s < DS; ++s) {
      if (stress) stress[((int64_t)b * DS + s) * g.N + e] = sig[s];
      acc[s] += sig[s];
    }
  }
#pragma unroll
  for (int s = 0; s < DS; ++s) {
    const double v = block_sum(acc[s]);
    if (threadIdx.x == 0) partial[((int64_t)b * DS + s) * kMaxPartials + blockIdx.x] = v * ec.vol;
  }
}

cudaError_t launch_stress(const Grid& g, const ElemConst& ec, const double* E, const double* u, int nb,
                          const StrainShift* shifts, double* stress, double* partial, int* nparts, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((g.N + 255) / 256, 1024);
  dim3 grid(blocks, nb);
  if (g.d == 2) JFFT_K("stress", st, k_stress<2><<<grid, 256, 0, st>>>(g, ec, E, u, shifts, stress, partial));
  else JFFT_K("stress", st, k_stress<3><<<grid, 256, 0, st>>>(g, ec, E, u, shifts, stress, partial));
  *nparts = blocks;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ S5
template <int D>
__global__ void k_node_esum(Grid g, const double* __restrict__ E, double* __restrict__ esum) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N; i += (int64_t)gridDim.x * blockDim.x) {
    int idx[3];
    int64_t r = i;
    for (int a = D - 1; a >= 0; --a) { idx[a] = (int)(r % g.n[a]); r /= g.n[a]; }
    double s = 0.0;
    for (int c = 0; c < (1 << D); ++c) {
      int64_t e = 0;
      for (int a = 0; a < D; ++a) {
        const int o = (c >> (D - 1 - a)) & 1;
        e = e * g.n[a] + (idx[a] - o + g.n[a]) % g.n[a];
      }
      s += E[e];
    }
    esum[i] = s;
  }
}

cudaError_t launch_node_esum(const Grid& g, const double* E, double* esum, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((g.N + 255) / 256, 152 * 16);
  if (g.d == 2) JFFT_K("node_esum", st, k_node_esum<2><<<blocks, 256, 0, st>>>(g, E, esum));
  else JFFT_K("node_esum", st, k_node_esum<3><<<blocks, 256, 0, st>>>(g, E, esum));
  return cudaGetLastError();
}

// Resolved J^1/2 table (Sec. 3.2, J = diag(K)^-1, zero diagonals replaced by the void
// value): for component a < comps and node i, with s the diagonal factor
// src[a src_cs + i], j = s^-1/2 (0 where s = 0) and the entry is j ka[a], or void_js
// where j = 0. Written in FP64 to js and / or in FP32 to js32 (the FP32 entry is
// float(j) float(ka[a]), the product the FP32 kernels formed before the table was
// resolved).
struct Ka3 { double k[3]; };
__global__ void k_jacobi_half(const double* __restrict__ src, int64_t src_cs, Ka3 ka, double void_js, int comps,
                              int64_t N, double* __restrict__ js, float* __restrict__ js32) {
  const int64_t n = comps * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx / N);
    const int64_t i = idx - a * N;
    const double s = src[a * src_cs + i];
    const double j = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
    if (js) js[idx] = j > 0.0 ? j * ka.k[a] : void_js;
    if (js32) {
      const float jf = (float)j;
      js32[idx] = jf > 0.f ? jf * (float)ka.k[a] : (float)void_js;
    }
  }
}

cudaError_t launch_jacobi_half(const double* src, int64_t src_cs, const double* ka, double void_js, int comps,
                               int64_t N, double* js, float* js32, cudaStream_t st) {
  Ka3 k3 = {{ka[0], ka[1], ka[2]}};
  const int blocks = (int)std::min<int64_t>((comps * N + 255) / 256, 152 * 16);
  JFFT_K("jacobi_half", st, k_jacobi_half<<<blocks, 256, 0, st>>>(src, src_cs, k3, void_js, comps, N, js, js32));
  return cudaGetLastError();
}

struct Kappa8 { double k[4][2]; };

// P1 closed-form diagonal: node I is corner o of the voxel I - o; diag[a][I] =
// sum_o E[I - o] kappa_o(a) (2D).
__global__ void k_diag_p1(Grid g, const double* __restrict__ E, Kappa8 kap, double* __restrict__ diag) {
  const int n0 = g.n[0], n1 = g.n[1];
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < g.N; I += (int64_t)gridDim.x * blockDim.x) {
    const int i0 = (int)(I / n1), i1 = (int)(I % n1);
    double s0 = 0.0, s1 = 0.0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int o0 = c >> 1, o1 = c & 1;
      const double e = E[(int64_t)((i0 - o0 + n0) % n0) * n1 + (i1 - o1 + n1) % n1];
      s0 += e * kap.k[c][0];
      s1 += e * kap.k[c][1];
    }
    diag[I] = s0;
    diag[g.N + I] = s1;
  }
}

cudaError_t launch_diag_p1(const Grid& g, const double* E, const double* kappa4, double* diag, cudaStream_t st) {
  Kappa8 k;
  for (int c = 0; c < 4; ++c)
    for (int a = 0; a < 2; ++a) k.k[c][a] = kappa4[c * 2 + a];
  const int blocks = (int)std::min<int64_t>((g.N + 255) / 256, 152 * 16);
  JFFT_K("diag_p1", st, k_diag_p1<<<blocks, 256, 0, st>>>(g, E, k, diag));
  return cudaGetLastError();
}

struct Kappa3 { double k[3]; };

__global__ void k_diag_closed(Grid g, const double* __restrict__ esum, Kappa3 kap, double* __restrict__ diag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N; i += (int64_t)gridDim.x * blockDim.x) {
    const double s = esum[i];
    for (int a = 0; a < g.d; ++a) diag[a * g.N + i] = kap.k[a] * s;
  }
}

cudaError_t launch_diag_closed(const Grid& g, const double* esum, const double* kappa3, double* diag,
                               cudaStream_t st) {
  Kappa3 k;
  for (int a = 0; a < 3; ++a) k.k[a] = kappa3[a];
  const int blocks = (int)std::min<int64_t>((g.N + 255) / 256, 152 * 16);
  JFFT_K("diag_closed", st, k_diag_closed<<<blocks, 256, 0, st>>>(g, esum, k, diag));
  return cudaGetLastError();
}

// Alg. 2: comb teeth of component `comp` sit at nodes whose 0-based index along
// every axis a has parity 1 - off_a (1-based index 2 I_a - off_a).
__device__ inline bool on_comb(const Grid& g, int64_t i, int offbits) {
  int64_t r = i;
  bool on = true;
  for (int a = g.d - 1; a >= 0; --a) {
    const int ia = (int)(r % g.n[a]);
    r /= g.n[a];
    const int off = (offbits >> (g.d - 1 - a)) & 1;
    on = on && ((ia & 1) == 1 - off);
  }
  return on;
}

__global__ void k_fill_comb(Grid g, int comp, int offbits, double* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N * g.d; i += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(i / g.N);
    const int64_t node = i % g.N;
    x[i] = (a == comp && on_comb(g, node, offbits)) ? 1.0 : 0.0;
  }
}

__global__ void k_extract_comb(Grid g, int comp, int offbits, const double* __restrict__ y, double* __restrict__ diag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N; i += (int64_t)gridDim.x * blockDim.x)
    if (on_comb(g, i, offbits)) diag[comp * g.N + i] = y[comp * g.N + i];
}

cudaError_t launch_fill_comb(const Grid& g, int comp, int offbits, double* x, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((g.N * g.d + 255) / 256, 152 * 16);
  JFFT_K("fill_comb", st, k_fill_comb<<<blocks, 256, 0, st>>>(g, comp, offbits, x));
  return cudaGetLastError();
}

cudaError_t launch_extract_comb(const Grid& g, int comp, int offbits, const double* y, double* diag, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((g.N + 255) / 256, 152 * 16);
  JFFT_K("extract_comb", st, k_extract_comb<<<blocks, 256, 0, st>>>(g, comp, offbits, y, diag));
  return cudaGetLastError();
}

// ------------------------------------------------------------------ S9 (Alg. 1)
// Field alpha of the batch [d][d][N] is the unit impulse in component alpha at node 0.
__global__ void k_impulses(Grid g, double* __restrict__ x) {
  const int64_t total = (int64_t)g.d * g.d * g.N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t field = i / ((int64_t)g.d * g.N);
    const int64_t rem = i % ((int64_t)g.d * g.N);
    x[i] = (rem == field * g.N) ? 1.0 : 0.0;
  }
}

cudaError_t launch_impulses(const Grid& g, double* x, cudaStream_t st) {
  const int64_t total = (int64_t)g.d * g.d * g.N;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  JFFT_K("impulses", st, k_impulses<<<blocks, 256, 0, st>>>(g, x));
  return cudaGetLastError();
}

// Steps 2-3 of Alg. 1 at every stored frequency of the half spectrum (k_0 fastest, the
// last axis halved): the transform of the impulse responses R[alpha][beta] of K_ref,
// then the d x d inversion, the zero frequency set to 0; the table stores
// G_hat * scale_store, upper triangle in the order (00, 01, 11) / (00, 01, 02, 11, 12, 22).
//
// Step 2 is evaluated over the support of R, the 3^D nodes that share an element with
// node 0 (offsets J in {-1, 0, 1}^D). Each R[alpha][beta] sums to zero (K_ref maps a
// rigid translation to zero), so its transform, the cosine sum over J, equals
//   K_hat(k) = -2 sum_J R(J) sin^2(pi k.J / n),
// in which every term keeps full relative accuracy at the lowest frequencies, where the
// full FFT of R would lose ~eps (n / 2 pi)^2 to cancellation. The phase k.J / n is an
// exact dyadic number; it is reduced to [-1/2, 1/2] exactly before sinpi. J and -J
// share one phase, so each pair is evaluated once with the sum R(J) + R(-J).
template <int D>
__global__ void __launch_bounds__(256) k_green_table(Grid g, const double* __restrict__ R, int64_t fstride,
                                                     double* __restrict__ G, double scale_store) {
  constexpr int NJ = D == 2 ? 9 : 27;   // offsets J in {-1, 0, 1}^D, J_0 slowest
  constexpr int NP = (NJ - 1) / 2;      // pairs {J, -J} with J != 0
  constexpr int NCMP = D * (D + 1) / 2;
  __shared__ double cp[NP][D][D];       // R(J) + R(-J) of the pair's first member J
  __shared__ int jof[NP][D];
  for (int t = threadIdx.x; t < NP * D * D; t += blockDim.x) {
    const int p = t / (D * D), a = (t / D) % D, b = t % D;
    // pair p: offset index p + NP + 1 (above the centre NP) and its mirror -J
    int rem = p + NP + 1;
    int off[D];
#pragma unroll
    for (int c = D - 1; c >= 0; --c) { off[c] = rem % 3 - 1; rem /= 3; }
    int64_t node_p = 0, node_m = 0;  // flat node index of J and of -J (periodic)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      node_p = node_p * g.n[c] + (off[c] + g.n[c]) % g.n[c];
      node_m = node_m * g.n[c] + (g.n[c] - off[c]) % g.n[c];
    }
    const double* Rab = R + (int64_t)a * fstride + (int64_t)b * g.N;
    cp[p][a][b] = Rab[node_p] + Rab[node_m];
    if (a == 0 && b == 0) {
#pragma unroll
      for (int c = 0; c < D; ++c) jof[p][c] = off[c];
    }
  }
  __syncthreads();
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < g.F; f += (int64_t)gridDim.x * blockDim.x) {
    int k[D];
    int64_t rem = f;
#pragma unroll
    for (int c = 0; c < D - 1; ++c) { k[c] = (int)(rem % g.n[c]); rem /= g.n[c]; }
    k[D - 1] = (int)rem;
    double K[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) K[a][b] = 0.0;
#pragma unroll 1
    for (int p = 0; p < NP; ++p) {
      double ph = 0.0;
#pragma unroll
      for (int c = 0; c < D; ++c) ph += (double)(k[c] * jof[p][c]) / (double)g.n[c];
      ph -= rint(ph);
      const double sn = sinpi(ph);
      const double s2 = -2.0 * sn * sn;
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) K[a][b] = fma(cp[p][a][b], s2, K[a][b]);
    }
    // symmetrise (the symbol is real symmetric; this removes rounding asymmetry)
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = a + 1; b < D; ++b) { const double sy = 0.5 * (K[a][b] + K[b][a]); K[a][b] = K[b][a] = sy; }
    double out[NCMP];
    if (f == 0) {
#pragma unroll
      for (int c = 0; c < NCMP; ++c) out[c] = 0.0;
    } else if (D == 2) {
      const double det = K[0][0] * K[1][1] - K[0][1] * K[1][0];
      out[0] = K[1][1] / det;
      out[1] = -K[0][1] / det;
      out[2] = K[0][0] / det;
    } else {
      const double c00 = K[1][1] * K[2][2] - K[1][2] * K[2][1];
      const double c01 = K[0][2] * K[2][1] - K[0][1] * K[2][2];
      const double c02 = K[0][1] * K[1][2] - K[0][2] * K[1][1];
      const double c11 = K[0][0] * K[2][2] - K[0][2] * K[2][0];
      const double c12 = K[0][2] * K[1][0] - K[0][0] * K[1][2];
      const double c22 = K[0][0] * K[1][1] - K[0][1] * K[1][0];
      const double det = K[0][0] * c00 + K[0][1] * (K[1][2] * K[2][0] - K[1][0] * K[2][2]) + K[0][2] * (K[1][0] * K[2][1] - K[1][1] * K[2][0]);
      out[0] = c00 / det; out[1] = c01 / det; out[2] = c02 / det;
      out[3] = c11 / det; out[4] = c12 / det; out[5] = c22 / det;
    }
#pragma unroll
    for (int c = 0; c < NCMP; ++c) G[f * NCMP + c] = out[c] * scale_store;
  }
}

cudaError_t launch_green_table(const Grid& g, const double* R, int64_t fstride, double* G, double scale_store,
                               cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((g.F + 255) / 256, 152 * 16);
  if (g.d == 2) JFFT_K("green_table", st, k_green_table<2><<<blocks, 256, 0, st>>>(g, R, fstride, G, scale_store));
  else JFFT_K("green_table", st, k_green_table<3><<<blocks, 256, 0, st>>>(g, R, fstride, G, scale_store));
  return cudaGetLastError();
}

template <int D>
__global__ void k_green_export(Grid g, const double* __restrict__ G, double* __restrict__ out, double inv_scale) {
  constexpr int NCMP = D * (D + 1) / 2;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < g.F; f += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) {
        const int lo = a < b ? a : b, hi = a < b ? b : a;
        const int c = (D == 2) ? (lo == 0 ? hi : 2) : (lo == 0 ? hi : (lo == 1 ? 2 + hi : 5));
        out[(f * D + a) * D + b] = G[f * NCMP + c] * inv_scale;
      }
  }
}

cudaError_t launch_green_export(const Grid& g, const double* G, double* out, double scale_store, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((g.F + 255) / 256, 152 * 16);
  if (g.d == 2) JFFT_K("green_export", st, k_green_export<2><<<blocks, 256, 0, st>>>(g, G, out, 1.0 / scale_store));
  else JFFT_K("green_export", st, k_green_export<3><<<blocks, 256, 0, st>>>(g, G, out, 1.0 / scale_store));
  return cudaGetLastError();
}

}  // namespace jfft
