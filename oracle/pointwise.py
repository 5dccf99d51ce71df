"""Node-by-node evaluation of K x for sampled nodes (paper Eq. lin_system_exp).

For grids too large to assemble, (K x)_{alpha I} = sum over the 2^d voxels e with a
corner o at I of E_e (A x_e)_{(alpha, o)}, A the element matrix of ``fe``. Each
sampled node is evaluated from this definition alone.
"""

from __future__ import annotations

import numpy as np

from . import assemble, fe


def apply_K_at(n, E: np.ndarray, C: np.ndarray, x: np.ndarray, nodes: np.ndarray) -> np.ndarray:
    """Rows of K x at the flat node indices ``nodes``: array [len(nodes), d]."""
    n = tuple(int(k) for k in n)
    d = len(n)
    A = fe.element_matrix(d, assemble.grid_spacing(n), C)
    cs = fe.corners(d)
    nc = len(cs)
    Ef = np.asarray(E).reshape(-1)
    xf = np.asarray(x).reshape(d, -1)
    idx = np.stack(np.unravel_index(nodes, n), axis=1)  # [m, d]
    out = np.zeros((len(nodes), d))
    for ci, o in enumerate(cs):
        e = (idx - np.array(o)) % np.array(n)           # voxel with corner o at the node
        ue = np.zeros((len(nodes), d * nc))
        for cj, o2 in enumerate(cs):
            node2 = np.ravel_multi_index(tuple(((e + np.array(o2)) % np.array(n)).T), n)
            for b in range(d):
                ue[:, b * nc + cj] = xf[b, node2]
        eflat = np.ravel_multi_index(tuple(e.T), n)
        fe_ = ue @ A.T                                   # element forces, [m, d nc]
        for a in range(d):
            out[:, a] += Ef[eflat] * fe_[:, a * nc + ci]
    return out
