"""Post-processing of a solve (paper Sec. 4.3 Eq. aim_fun, Sec. 5.3).

* The Green-Jacobi iterates carry a constant shift (the outer J^(1/2) does not keep
  the mean at zero, Sec. 5.3); the fluctuation is reported with its mean removed
  per displacement component, which is the unique zero-mean solution.
* Stress at Gauss point q of element e: sigma_{e,q} = E_e C_unit (eps_bar + B_q u_e).
  The element-averaged stress is the mean over the 2^d Gauss points.
* Homogenised stiffness column gamma: the cell average of the stress for the load
  eps_bar_gamma, sum_e sum_q w_q sigma_{e,q} / |Y| with |Y| = 1.
"""

from __future__ import annotations

import numpy as np

from . import assemble, fe


def remove_mean(u: np.ndarray) -> np.ndarray:
    axes = tuple(range(1, u.ndim))
    return u - u.mean(axis=axes, keepdims=True)


def gauss_point_stress(n, E: np.ndarray, C: np.ndarray, eps_bar: np.ndarray, u: np.ndarray,
                       element: str = "q1"):
    """sigma[q, e, :] at every integration point q of every voxel e (Mandel: the Gauss
    points for Q1, the two triangles for P1), and the weights."""
    n = tuple(int(k) for k in n)
    d = len(n)
    h = assemble.grid_spacing(n)
    g = assemble.element_dofs(n)
    ue = u.reshape(-1)[g]  # [N_el, d 2^d]
    Bs, ws = fe.element_points(d, h, element)
    Ef = np.asarray(E, dtype=np.float64).reshape(-1)
    sig = []
    for B in Bs:
        eps = eps_bar[None, :] + ue @ B.T
        sig.append(Ef[:, None] * (eps @ C.T))
    return np.stack(sig), np.array(ws)


def element_stress(n, E, C, eps_bar, u, element: str = "q1") -> np.ndarray:
    """Voxel-averaged Mandel stress (equal-weight points), shape [d*, *n]."""
    n = tuple(int(k) for k in n)
    sig, _ = gauss_point_stress(n, E, C, eps_bar, u, element)
    return sig.mean(axis=0).T.reshape((sig.shape[2],) + n)


def homogenised_stress(n, E, C, eps_bar, u, element: str = "q1") -> np.ndarray:
    """(1/|Y|) int sigma dx by the voxel rule, |Y| = 1: Mandel vector of length d*."""
    sig, w = gauss_point_stress(n, E, C, eps_bar, u, element)
    return np.einsum("q,qes->s", w, sig)
