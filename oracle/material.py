"""Per-voxel material (paper Sec. 4 "Constitutive law" and "Material data sampling").

The paper's law is sigma = rho(x) C^0 eps with a scalar density. The benchmarks map a
density rho in [0, 1] to a Young's modulus E = E_min + (E_max - E_min) rho^p with
E_max = 1, E_min = 1 / contrast and a fixed Poisson ratio, so C_e = E_e C_unit(nu),
which has the same scaled-isotropic form. Voxel e takes the density sampled at its
lowest-corner node.
"""

from __future__ import annotations

import numpy as np


def young_from_density(rho: np.ndarray, e_min: float, e_max: float, exponent: float) -> np.ndarray:
    rho = np.asarray(rho, dtype=np.float64)
    return e_min + (e_max - e_min) * np.power(rho, exponent)


def upsample(coarse: np.ndarray, n) -> np.ndarray:
    """Geometry G_p on the grid T_n (Sec. 4 "Discretization and grid refinement", n >= p):
    pixel-wise constant data, so every voxel takes the value of the pixel containing it;
    each pixel covers (n_a / p_a) voxels along axis a."""
    coarse = np.asarray(coarse, dtype=np.float64)
    out = coarse
    for a, na in enumerate(n):
        pa = coarse.shape[a]
        if na % pa:
            raise ValueError("n must be a multiple of p on every axis")
        out = np.repeat(out, na // pa, axis=a)
    return out
