"""Assembly of the linear-elastic system on the periodic grid (paper Eq. lin_system_exp).

K(rho) = B^T W C(rho) B and f(rho) = -B^T W C(rho) E, written element by element:
element ``e`` (multi-index, the voxel whose lowest corner is node e) couples the
nodes ``(e + o) mod n`` for o in {0,1}^d and carries the material C_e = E_e C_unit.

Global DOF numbering is component-major, matching the [d, N_1, ..., N_d] array
layout of the paper's Alg. 1: dof(alpha, I) = alpha * N + flat(I), C order.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fe


def grid_spacing(n):
    return tuple(1.0 / float(k) for k in n)


def element_dofs(n) -> np.ndarray:
    """Global DOF index of every local DOF of every element: int64 [N_el, d 2^d]."""
    n = tuple(int(k) for k in n)
    d = len(n)
    N = int(np.prod(n))
    grids = np.meshgrid(*[np.arange(k) for k in n], indexing="ij")
    e_idx = [g.reshape(-1) for g in grids]  # element multi-index, C order
    node_of_corner = []
    for o in fe.corners(d):
        flat = np.zeros(N, dtype=np.int64)
        for a in range(d):
            flat = flat * n[a] + (e_idx[a] + o[a]) % n[a]
        node_of_corner.append(flat)
    node_of_corner = np.stack(node_of_corner, axis=1)  # [N_el, 2^d]
    return np.concatenate([node_of_corner + alpha * N for alpha in range(d)], axis=1)


def assemble_K(n, E: np.ndarray, C: np.ndarray, element: str = "q1") -> sp.csr_matrix:
    """Sparse K = sum_e E_e P_e^T A P_e, A the element matrix of material ``C``."""
    n = tuple(int(k) for k in n)
    d = len(n)
    A = fe.element_matrix(d, grid_spacing(n), C, element)
    g = element_dofs(n)
    ne, nl = g.shape
    rows = np.repeat(g, nl, axis=1).reshape(-1)
    cols = np.tile(g, (1, nl)).reshape(-1)
    vals = (np.asarray(E, dtype=np.float64).reshape(-1)[:, None] * A.reshape(1, -1)).reshape(-1)
    ndof = d * int(np.prod(n))
    K = sp.coo_matrix((vals, (rows, cols)), shape=(ndof, ndof)).tocsr()
    K.sum_duplicates()
    return K


def assemble_rhs(n, E: np.ndarray, C: np.ndarray, eps_bar: np.ndarray, element: str = "q1") -> np.ndarray:
    """f = -sum_e E_e P_e^T b(eps_bar), b = sum_q w_q B_q^T C eps_bar. Shape [d, *n], in the
    floating-point type of E and C (at least FP64)."""
    n = tuple(int(k) for k in n)
    d = len(n)
    dtype = np.result_type(np.asarray(E).dtype, np.asarray(C).dtype, np.float64).type
    b = fe.element_strain_load(d, grid_spacing(n), np.asarray(C, dtype=dtype), np.asarray(eps_bar, dtype=dtype),
                               element)
    g = element_dofs(n)
    vals = -(np.asarray(E, dtype=dtype).reshape(-1)[:, None] * b[None, :])
    f = np.zeros(d * int(np.prod(n)), dtype=dtype)
    np.add.at(f, g.reshape(-1), vals.reshape(-1))
    return f.reshape((d,) + n)


def apply(K: sp.csr_matrix, u: np.ndarray) -> np.ndarray:
    """K u for a field u of shape [d, *n]."""
    return (K @ u.reshape(-1)).reshape(u.shape)


def apply_matrix_free(n, E: np.ndarray, C: np.ndarray, u: np.ndarray, element: str = "q1") -> np.ndarray:
    """K u = B^T W C(rho) B u evaluated element by element (the matrix-free product of
    Sec. 3.1), for a field u of shape [d, *n].

    For every element e: the nodal values of its corners minus the value at its corner 0
    (A = sum_q w_q B_q^T C B_q annihilates a constant field, so A u_e = A (u_e - u_e[0])
    exactly), the element forces E_e A (u_e - u_e[0]), added into the nodes corner by
    corner. Equal to ``apply(assemble_K(...), u)`` in exact arithmetic; on smooth fields
    it keeps the relative accuracy that the assembled product loses by summing large
    entries of alternating sign (about eps (n / 2 pi)^2 at the lowest frequency),
    because the differences of neighbouring values are formed first."""
    n = tuple(int(k) for k in n)
    d = len(n)
    axes = tuple(range(1, d + 1))
    cs = fe.corners(d)
    nc = len(cs)
    N = int(np.prod(n))
    A = fe.element_matrix(d, grid_spacing(n), C, element)
    # ue[e, alpha * nc + c] = u[alpha][e + o_c] - u[alpha][e]
    ue = np.stack([np.roll(u, tuple(-o for o in oc), axes) for oc in cs], axis=-1)  # [d, *n, nc]
    ue = ue - ue[..., :1]
    ue = np.moveaxis(ue.reshape(d, N, nc), 1, 0).reshape(N, d * nc)
    Ef = np.asarray(E).reshape(-1)
    forces = (Ef[:, None] * (ue @ A.T)).reshape(N, d, nc)
    q = np.zeros((d,) + n, dtype=forces.dtype)
    for ci, oc in enumerate(cs):
        q += np.roll(np.moveaxis(forces[:, :, ci], 0, 1).reshape((d,) + n), tuple(oc), axes)
    return q
