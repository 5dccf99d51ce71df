// Q1 element operator in Walsh-Hadamard mode form (host + device).
//
// Element stiffness of the paper's FE discretisation (Sec. 2.1, K_e = B^T W C_e B
// with the full 2^d Gauss rule), evaluated without forming the (d 2^d)^2 matrix:
//   1. corner values -> modes W[m] = sum_o prod_{b in m} (2 o_b - 1) u(o), a d-stage
//      butterfly per component (the monomial basis 1, s_a, s_a s_b, ... of the
//      bilinear / trilinear shape functions, s_a = 2 xi_a - 1);
//   2. modes -> mode forces F = L W with the constant linear map of ElemConst
//      (the Gauss rule integrates products of distinct monomials to zero, so L
//      couples only modes that share a monomial after one derivative);
//   3. mode forces -> corner forces by the transposed butterfly, times E_e.
// Corner index c = sum_a o_a 2^(d-1-a); mode bit of axis a is 1 << (d-1-a).
#pragma once

#include "jfft_internal.cuh"

namespace jfft {

#define JFFT_HD __host__ __device__ __forceinline__

// Mode bit of axis a.
template <int D> JFFT_HD constexpr int mbit(int a) { return 1 << (D - 1 - a); }

// In-place forward butterfly over the D axes: v[c] -> W[m].
template <int D, typename V> JFFT_HD void wht_fwd(V* v) {
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int s = 1 << a;
#pragma unroll
    for (int c = 0; c < (1 << D); ++c) {
      if (!(c & s)) {
        V lo = v[c], hi = v[c | s];
        v[c] = lo + hi;
        v[c | s] = hi - lo;
      }
    }
  }
}

// In-place transposed butterfly: F[m] -> f[c] = sum_m prod_{b in m} (2 o_b - 1) F[m].
template <int D, typename V> JFFT_HD void wht_bwd(V* v) {
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int s = 1 << a;
#pragma unroll
    for (int c = 0; c < (1 << D); ++c) {
      if (!(c & s)) {
        V y0 = v[c], y1 = v[c | s];
        v[c] = y0 - y1;
        v[c | s] = y0 + y1;
      }
    }
  }
}

// wht_bwd for a vector whose entry 0 is zero (v[0] is not read).
template <int D, typename V> JFFT_HD void wht_bwd_z0(V* v) {
  {
    const V y1 = v[1];
    v[0] = -y1;
    v[1] = y1;
#pragma unroll
    for (int c = 2; c < (1 << D); c += 2) {
      const V y0 = v[c], z1 = v[c | 1];
      v[c] = y0 - z1;
      v[c | 1] = y0 + z1;
    }
  }
#pragma unroll
  for (int a = 1; a < D; ++a) {
    const int s = 1 << a;
#pragma unroll
    for (int c = 0; c < (1 << D); ++c) {
      if (!(c & s)) {
        V y0 = v[c], y1 = v[c | s];
        v[c] = y0 - y1;
        v[c | s] = y0 + y1;
      }
    }
  }
}

template <int D> JFFT_HD constexpr int popc(int m) {
  return (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1);
}

// Mode forces F[a][m] (zeroed on entry) from modes W[a][m] for unit E.
template <int D, typename V> JFFT_HD void mode_forces(const ElemConstT<V>& ec, const V (*W)[1 << D], V (*F)[1 << D]) {
  constexpr int NC = 1 << D;
#pragma unroll
  for (int mu = 0; mu < NC; ++mu) {
    const int k = popc<D>(mu);
    if (k >= D) continue;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int ba = mbit<D>(a);
      if (mu & ba) continue;
      const int ma = mu | ba;
      // normal stresses of monomial mu
#pragma unroll
      for (int b = 0; b < D; ++b) {
        const int bb = mbit<D>(b);
        if (mu & bb) continue;
        F[a][ma] += ec.nrm[k][a][b] * W[b][mu | bb];
      }
      // shear between two free axes a != b
#pragma unroll
      for (int b = 0; b < D; ++b) {
        const int bb = mbit<D>(b);
        if ((mu & bb) || b == a) continue;
        F[a][mu | bb] += ec.shr[k][b][b] * W[a][mu | bb] + ec.shr[k][a][b] * W[b][ma];
      }
      // shear between a free axis a and a locked axis c in mu
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const int bc = mbit<D>(c);
        if (!(mu & bc)) continue;
        F[c][ma] += ec.shr[k][a][a] * W[c][ma];
      }
    }
  }
}

// Corner forces f[a][c] = E * K_e-unit u, with u[a][c] corner displacements and an
// optional macroscopic strain shift added to the single-axis modes.
template <int D, typename V, bool SHIFT>
JFFT_HD void element_force(const ElemConstT<V>& ec, const StrainShift* sh, V (*u)[1 << D], V E) {
  constexpr int NC = 1 << D;
  V F[D][NC];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    wht_fwd<D>(u[a]);
#pragma unroll
    for (int m = 0; m < NC; ++m) F[a][m] = V(0);
  }
  if (SHIFT) {
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) u[a][mbit<D>(b)] += V(sh->s[a][b]);
  }
  mode_forces<D>(ec, u, F);
  // Mode 0 (rigid translation) carries no force: it is left out of the scaling and
  // of the first butterfly stage instead of being multiplied and added as a zero.
#pragma unroll
  for (int a = 0; a < D; ++a) {
#pragma unroll
    for (int m = 1; m < NC; ++m) u[a][m] = F[a][m] * E;
    wht_bwd_z0<D>(u[a]);
  }
}

// Element-averaged Mandel stress E C (eps_bar + eps_mu=0(u)) from the corner values.
template <int D> JFFT_HD void element_stress(const ElemConst& ec, const StrainShift* sh, double (*u)[1 << D],
                                             double E, double* sig) {
  double G[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    wht_fwd<D>(u[a]);
#pragma unroll
    for (int b = 0; b < D; ++b) {
      double w = u[a][mbit<D>(b)] + (sh ? sh->s[a][b] : 0.0);
      G[a][b] = ec.gs[b] * w;
    }
  }
  double tr = 0.0;
#pragma unroll
  for (int a = 0; a < D; ++a) tr += G[a][a];
  // Mandel order: normals, then (2D) 12 ; (3D) 23, 13, 12
#pragma unroll
  for (int a = 0; a < D; ++a) sig[a] = E * (ec.lam * tr + 2.0 * ec.mu * G[a][a]);
  const double r2 = 1.4142135623730951;
  if (D == 2) {
    sig[2] = E * r2 * ec.mu * (G[0][1] + G[1][0]);
  } else {
    sig[3] = E * r2 * ec.mu * (G[1][2] + G[2][1]);
    sig[4] = E * r2 * ec.mu * (G[0][2] + G[2][0]);
    sig[5] = E * r2 * ec.mu * (G[0][1] + G[1][0]);
  }
}

// P1 discretisation of a 2D voxel (Sec. 4 "Discretization": linear triangles): the voxel
// is split along the diagonal from corner (0,0) to corner (1,1) into T1 = {(0,0), (1,0),
// (1,1)} and T2 = {(0,0), (1,1), (0,1)}, each with a constant strain. Corner index
// c = o0 * 2 + o1. Stress of one triangle from its displacement gradient grad[a][b]
// = du_a / dx_b plus the macroscopic strain (tensor form eb), for unit E.
template <typename V> JFFT_HD void tri_stress(const ElemConstT<V>& ec, const V (*grad)[2], const V (*eb)[2], V (*sg)[2]) {
  const V e00 = grad[0][0] + eb[0][0], e11 = grad[1][1] + eb[1][1];
  const V e01 = V(0.5) * (grad[0][1] + grad[1][0]) + eb[0][1];
  const V tr = e00 + e11;
  sg[0][0] = ec.lam * tr + V(2) * ec.mu * e00;
  sg[1][1] = ec.lam * tr + V(2) * ec.mu * e11;
  sg[0][1] = sg[1][0] = V(2) * ec.mu * e01;
}

// Corner forces f[a][c] = E * K_voxel-unit u for the two triangles (in place), with an
// optional macroscopic strain shift (StrainShift holds eps_ab / gs_b).
template <typename V, bool SHIFT>
JFFT_HD void tri_pair_force(const ElemConstT<V>& ec, const StrainShift* sh, V (*u)[4], V E) {
  const V ih0 = V(2) * ec.gs[0], ih1 = V(2) * ec.gs[1];   // gs_a = 1 / (2 h_a) in 2D
  const V area = V(0.5) * ec.vol;
  V eb[2][2] = {{V(0), V(0)}, {V(0), V(0)}};
  if (SHIFT) {
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) eb[a][b] = V(sh->s[a][b]) * ec.gs[b];
  }
  V g1[2][2], g2[2][2], s1[2][2], s2[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    g1[a][0] = (u[a][2] - u[a][0]) * ih0;   // T1: (0,0) -> (1,0) along axis 0
    g1[a][1] = (u[a][3] - u[a][2]) * ih1;   //     (1,0) -> (1,1) along axis 1
    g2[a][1] = (u[a][1] - u[a][0]) * ih1;   // T2: (0,0) -> (0,1) along axis 1
    g2[a][0] = (u[a][3] - u[a][1]) * ih0;   //     (0,1) -> (1,1) along axis 0
  }
  tri_stress<V>(ec, g1, eb, s1);
  tri_stress<V>(ec, g2, eb, s2);
  const V w = area * E;
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    // T1 shape gradients: (0,0) (-ih0, 0), (1,0) (ih0, -ih1), (1,1) (0, ih1)
    // T2 shape gradients: (0,0) (0, -ih1), (0,1) (-ih0, ih1), (1,1) (ih0, 0)
    const V f0 = -ih0 * s1[a][0] - ih1 * s2[a][1];
    const V f1 = -ih0 * s2[a][0] + ih1 * s2[a][1];
    const V f2 = ih0 * s1[a][0] - ih1 * s1[a][1];
    const V f3 = ih1 * s1[a][1] + ih0 * s2[a][0];
    u[a][0] = w * f0;
    u[a][1] = w * f1;
    u[a][2] = w * f2;
    u[a][3] = w * f3;
  }
}

// Voxel-averaged Mandel stress E C (eps_bar + eps(u)) of the two triangles.
JFFT_HD void tri_pair_stress(const ElemConst& ec, const StrainShift* sh, double (*u)[4], double E, double* sig) {
  const double ih0 = 2.0 * ec.gs[0], ih1 = 2.0 * ec.gs[1];
  double eb[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  if (sh)
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) eb[a][b] = sh->s[a][b] * ec.gs[b];
  double g1[2][2], g2[2][2], s1[2][2], s2[2][2];
  for (int a = 0; a < 2; ++a) {
    g1[a][0] = (u[a][2] - u[a][0]) * ih0;
    g1[a][1] = (u[a][3] - u[a][2]) * ih1;
    g2[a][1] = (u[a][1] - u[a][0]) * ih1;
    g2[a][0] = (u[a][3] - u[a][1]) * ih0;
  }
  tri_stress<double>(ec, g1, eb, s1);
  tri_stress<double>(ec, g2, eb, s2);
  const double r2 = 1.4142135623730951;
  sig[0] = E * 0.5 * (s1[0][0] + s2[0][0]);
  sig[1] = E * 0.5 * (s1[1][1] + s2[1][1]);
  sig[2] = E * r2 * 0.5 * (s1[0][1] + s2[0][1]);
}

// Constants of the unit-E element for a d-dimensional box h[0..d-1] and Lame pair.
inline ElemConst make_elem_const(int d, const double* h, double lam, double mu) {
  ElemConst ec = {};
  double vol = 1.0;
  for (int a = 0; a < d; ++a) vol *= h[a];
  for (int a = 0; a < d; ++a) ec.gs[a] = (2.0 / h[a]) / double(1 << d);
  double kap = vol;
  for (int k = 0; k < 3; ++k) {
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        ec.nrm[k][a][b] = (a == b ? lam + 2.0 * mu : lam) * kap * ec.gs[a] * ec.gs[b];
        ec.shr[k][a][b] = mu * kap * ec.gs[a] * ec.gs[b];
      }
    kap /= 3.0;
  }
  ec.lam = lam;
  ec.mu = mu;
  ec.vol = vol;
  ec.elem = 0;
  return ec;
}

// Mode shift realising a macroscopic Mandel strain eps (length d(d+1)/2).
inline StrainShift make_shift(int d, const ElemConst& ec, const double* eps) {
  StrainShift s = {};
  const double ir2 = 0.70710678118654752440;
  double t[3][3] = {};
  if (d == 2) {
    t[0][0] = eps[0]; t[1][1] = eps[1]; t[0][1] = t[1][0] = eps[2] * ir2;
  } else {
    t[0][0] = eps[0]; t[1][1] = eps[1]; t[2][2] = eps[2];
    t[1][2] = t[2][1] = eps[3] * ir2;
    t[0][2] = t[2][0] = eps[4] * ir2;
    t[0][1] = t[1][0] = eps[5] * ir2;
  }
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) s.s[a][b] = t[a][b] / ec.gs[b];
  return s;
}

}  // namespace jfft
