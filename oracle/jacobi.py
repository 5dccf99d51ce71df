"""Jacobi diagonal diag(K), the void rule and J^(1/2) (paper Sec. 3.2, Eq. Jacobi, Alg. 2)."""

from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp


def diag_assembled(K: sp.csr_matrix, shape) -> np.ndarray:
    """diag(K) read from the assembled matrix, shape [d, *n]."""
    return K.diagonal().reshape(shape)


def diag_matrix_free(n, E: np.ndarray, C: np.ndarray, element: str = "q1") -> np.ndarray:
    """diag(K) without assembly: node I, component alpha collects E_e A[(alpha, o), (alpha, o)]
    from each of the 2^d voxels e = I - o that have I at their corner o (A the unit
    element matrix). In the floating-point type of E and C (the extended-precision oracle
    derives its Jacobi scaling this way). Shape [d, *n]."""
    from . import assemble, fe
    n = tuple(int(k) for k in n)
    d = len(n)
    A = fe.element_matrix(d, assemble.grid_spacing(n), C, element)
    E = np.asarray(E).astype(A.dtype)
    nc = 2 ** d
    out = np.zeros((d,) + n, dtype=A.dtype)
    for ci, o in enumerate(fe.corners(d)):
        Eo = np.roll(E, tuple(o), tuple(range(d)))   # E of the voxel with corner o at each node
        for a in range(d):
            out[a] += Eo * A[a * nc + ci, a * nc + ci]
    return out


def diag_alg2(apply_K, d: int, n) -> tuple[np.ndarray, int]:
    """Alg. 2: diag(K) from d 2^d operator applications to impulse combs.

    For component alpha and offset (i_1..i_d) in {0,1}^d the comb has a unit entry
    in component alpha at every node with 1-based index 2 I_a - i_a, I_a = 1..n_a/2
    (0-based: 2 I_a - 1 - i_a); the operator's response at those nodes is the
    diagonal there, since two comb teeth never share an element (even n_a). The
    paper's "N/(d 2^d) terms at once" is read as n^d / 2^d diagonal entries of one
    component per application. Returns (diag [d, *n], number of applications).
    """
    n = tuple(int(k) for k in n)
    if any(k % 2 for k in n):
        raise ValueError("Alg. 2 needs an even number of nodes per axis")
    diag = np.zeros((d,) + n)
    count = 0
    for alpha in range(d):
        for off in itertools.product((0, 1), repeat=d):
            sel = tuple(slice(1 - o, None, 2) for o in off)  # 0-based 2I-1-o
            comb = np.zeros((d,) + n)
            comb[(alpha,) + sel] = 1.0
            resp = apply_K(comb)
            count += 1
            diag[(alpha,) + sel] = resp[(alpha,) + sel]
    return diag, count


def void_rule(diag: np.ndarray) -> np.ndarray:
    """Zero diagonal entries (void regions) are replaced by 1 before inversion (Sec. 3.2)."""
    out = diag.copy()
    out[out == 0.0] = 1.0
    return out


def jacobi_half(diag: np.ndarray, replacement: float = 1.0) -> np.ndarray:
    """J^(1/2) = diag(K)^(-1/2), with zero entries replaced by ``replacement`` first."""
    dd = diag.copy()
    dd[dd == 0.0] = replacement
    return 1 / np.sqrt(dd)
