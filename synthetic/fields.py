"""Seeded density fields and load cases on a periodic regular grid.

Conventions (shared with the solver's C interface):
  * a grid has ``n = (n_1, ..., n_d)`` nodal points per axis on the unit cell
    [0, 1)^d, C order, last axis contiguous; node ``I`` sits at ``x_I = I / n``;
  * fields are sampled at the nodal points and each sample is assigned to the
    whole voxel whose lowest corner is that node (pixel-wise constant material
    data, paper Sec. 4 "Material data sampling");
  * Mandel order is (11, 22, 12) in 2D and (11, 22, 33, 23, 13, 12) in 3D.

Nothing here computes a stiffness, a residual or a preconditioner.
"""

from __future__ import annotations

import itertools
import math

import numpy as np


def mandel_dim(d: int) -> int:
    """Number of Mandel components d* = d (d + 1) / 2 (paper Sec. 2)."""
    return d * (d + 1) // 2


def mandel_unit_loads(d: int) -> np.ndarray:
    """The canonical macroscopic load cases e_gamma, gamma = 1..d* (paper Sec. 4.3)."""
    return np.eye(mandel_dim(d))


def _nodal_coords(shape):
    return [np.arange(n, dtype=np.float64) / n for n in shape]


def _smooth_modes(d: int, n_modes: int, k_max: float, seed: int):
    """Steps 1-2 of the smooth_density recipe: wave vectors, amplitudes, phases."""
    kmax_i = int(math.floor(k_max))
    cands = [k for k in itertools.product(range(-kmax_i, kmax_i + 1), repeat=d)
             if 0 < sum(c * c for c in k) <= k_max * k_max]
    cands = np.array(cands, dtype=np.int64)
    if n_modes > len(cands):
        raise ValueError("n_modes exceeds the number of wave vectors with |k| <= k_max")
    rng = np.random.default_rng(seed)
    pick = rng.choice(len(cands), size=n_modes, replace=False)
    kvec = cands[pick]
    amp = rng.standard_normal(n_modes)
    phase = rng.uniform(0.0, 2.0 * math.pi, n_modes)
    return kvec, amp, phase


def smooth_density_device(shape, n_modes: int, k_max: float, seed: int, device="cuda"):
    """The smooth_density recipe (same wave vectors, amplitudes and phases) evaluated as a
    float64 torch tensor on ``device``: for grids whose host evaluation would take minutes
    (512^3). Equal to smooth_density up to the rounding of the sum."""
    import torch
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    kvec, amp, phase = _smooth_modes(d, n_modes, k_max, seed)
    coords = _nodal_coords(shape)
    fac = [torch.tensor(np.exp(2j * math.pi * np.outer(kvec[:, a], coords[a])), device=device) for a in range(d)]
    coef = torch.tensor(amp * np.exp(1j * phase), device=device)
    raw = torch.zeros(shape, dtype=torch.float64, device=device)
    for m in range(n_modes):
        t = coef[m] * fac[0][m]
        for a in range(1, d):
            t = t.reshape(t.shape + (1,)) * fac[a][m].reshape((1,) * a + (-1,))
        raw += t.real
        del t
    lo, hi = raw.min(), raw.max()
    return (raw - lo) / (hi - lo)


def smooth_density(shape, n_modes: int, k_max: float, seed: int) -> np.ndarray:
    """Smooth random density rho in [0, 1] from a sum of Fourier modes.

    Recipe (the paper's topology-optimisation densities are not available, so
    this stands in for smooth high-contrast data):
      1. candidate wave vectors: every integer k in Z^d with 0 < |k|_2 <= k_max,
         listed in lexicographic order;
      2. ``rng = numpy.random.default_rng(seed)``; draw ``n_modes`` distinct
         candidates (``rng.choice(..., replace=False)``), then amplitudes
         a ~ N(0, 1), then phases phi ~ U[0, 2 pi), in that order;
      3. raw(x) = sum_m a_m cos(2 pi k_m . x + phi_m) at the nodal points;
      4. rho = (raw - min raw) / (max raw - min raw).
    """
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    kvec, amp, phase = _smooth_modes(d, n_modes, k_max, seed)

    # Separable evaluation, one slab of the first axis at a time, so that large
    # 3D grids do not need an n_modes x N temporary.
    coords = _nodal_coords(shape)
    raw = np.empty(shape, dtype=np.float64)
    # per-axis phase factors exp(2 pi i k_a x_a), shape [n_modes, n_a]
    fac = [np.exp(2j * math.pi * np.outer(kvec[:, a], coords[a])) for a in range(d)]
    coef = amp * np.exp(1j * phase)
    for i0 in range(shape[0]):
        acc = np.zeros(shape[1:], dtype=np.complex128)
        for m in range(n_modes):
            term = coef[m] * fac[0][m, i0]
            t = fac[1][m]
            for a in range(2, d):
                t = np.multiply.outer(t, fac[a][m])
            acc += term * t
        raw[i0] = acc.real
    lo, hi = raw.min(), raw.max()
    return (raw - lo) / (hi - lo)


def laminate_density(shape, chi_tot: float) -> np.ndarray:
    """Laminate density of paper Sec. 4.1: linear in x_1, constant in the other axes.

    rho(x) = chi + (1 - chi) x_1 / (1 - dx_1), with dx_1 = 1 / n_1 the pixel size,
    sampled at the nodal points (geometry resolution p equal to the grid).
    """
    shape = tuple(int(s) for s in shape)
    x1 = np.arange(shape[0], dtype=np.float64) / shape[0]
    dx1 = 1.0 / shape[0]
    rho1 = chi_tot + (1.0 - chi_tot) / (1.0 - dx1) * x1
    return np.broadcast_to(rho1.reshape((-1,) + (1,) * (len(shape) - 1)), shape).copy()


def cosine_density(shape, chi_tot: float) -> np.ndarray:
    """Cosine geometry of paper Sec. 4.2 (2D), raised by 1 / chi (chi = inf gives voids).

    rho(x) = 0.5 + 0.25 (cos(2 pi (x1 - x2)) + cos(2 pi (x2 + x1))) + 1 / chi.
    """
    shape = tuple(int(s) for s in shape)
    if len(shape) != 2:
        raise ValueError("the cosine geometry is two-dimensional")
    x1, x2 = np.meshgrid(*_nodal_coords(shape), indexing="ij")
    lift = 0.0 if math.isinf(chi_tot) else 1.0 / chi_tot
    return 0.5 + 0.25 * (np.cos(2 * math.pi * (x1 - x2)) + np.cos(2 * math.pi * (x2 + x1))) + lift


def random_field(shape, seed: int, zero_mean: bool = False) -> np.ndarray:
    """Standard-normal array of the given shape (e.g. [d, n_1, ..., n_d]).

    ``zero_mean`` subtracts the mean over every axis but the first, so a [d, *n]
    field gets zero mean per component."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(tuple(int(s) for s in shape))
    if zero_mean:
        axes = tuple(range(1, a.ndim))
        a = a - a.mean(axis=axes, keepdims=True)
    return a


def circular_inclusion(shape, radius: float = 0.25, soft: float = 1e-4, hard: float = 1.0) -> np.ndarray:
    """Compliant circular (2D) or spherical (3D) inclusion of the given radius (in cell
    units, centred in the unit cell) in a stiff matrix, sampled at the nodes x = i / n:
    `soft` inside, `hard` outside (the motivating example of Sec. 1)."""
    shape = tuple(int(s) for s in shape)
    axes = np.meshgrid(*[np.arange(n) / n - 0.5 for n in shape], indexing="ij")
    r2 = sum(a * a for a in axes)
    return np.where(r2 <= radius * radius, soft, hard).astype(np.float64)


def gaussian_filter(rho: np.ndarray, times: int) -> np.ndarray:
    """`times` periodic convolutions with the separable kernel [1 2 1] / 4 on every axis
    (in 2D G = 1/16 [1 2 1]^T [1 2 1], Sec. 1)."""
    out = np.asarray(rho, dtype=np.float64).copy()
    for _ in range(int(times)):
        for ax in range(out.ndim):
            out = 0.25 * (np.roll(out, 1, ax) + 2.0 * out + np.roll(out, -1, ax))
    return out
