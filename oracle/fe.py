"""Q1 finite element on a regular periodic grid (paper Sec. 2.1).

Every component u_alpha of the displacement is a bilinear (2D) or trilinear (3D)
interpolation of its nodal values. The symmetrised gradient is evaluated at the
2^d Gauss points of each element, stored in Mandel notation
(11, 22, 12) / (11, 22, 33, 23, 13, 12) with the shear entries multiplied by
sqrt(2) (paper Sec. 2: d* = d(d+1)/2; sqrt(2) convention as in Sec. 4.5, where a
shear macro strain 0.05 appears as Mandel component 0.05 sqrt(2)).

Local node (corner) ordering: corner ``o`` in {0,1}^d, lexicographic with the last
axis fastest. Local DOF ordering of an element: ``alpha * 2^d + corner``.
"""

from __future__ import annotations

import itertools
import math

import numpy as np


def mandel_pairs(d: int):
    """(i, j) tensor index of each Mandel component."""
    if d == 2:
        return [(0, 0), (1, 1), (0, 1)]
    if d == 3:
        return [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    raise ValueError("d must be 2 or 3")


def corners(d: int):
    return list(itertools.product((0, 1), repeat=d))


def gauss_points(d: int, dtype=np.float64):
    """The 2^d Gauss points of the reference cell [0,1]^d and their weights (sum 1), in
    ``dtype`` (numpy.longdouble for the extended-precision oracle)."""
    half = dtype(0.5)
    r = half / np.sqrt(dtype(3))
    g = (half - r, half + r)
    pts = [tuple(g[i] for i in idx) for idx in itertools.product((0, 1), repeat=d)]
    w = [dtype(1) / dtype(2 ** d)] * len(pts)
    return pts, w


def shape_gradients(d: int, xi, h, dtype=np.float64) -> np.ndarray:
    """dphi_c / dx_beta at local point ``xi`` for each corner c: array [2^d, d].

    phi_c(xi) = prod_a (xi_a if c_a == 1 else 1 - xi_a), x_a = h_a xi_a.
    """
    out = np.zeros((2 ** d, d), dtype=dtype)
    for ci, c in enumerate(corners(d)):
        for b in range(d):
            v = dtype(1.0 if c[b] else -1.0) / dtype(h[b])
            for a in range(d):
                if a != b:
                    v *= xi[a] if c[a] else (1.0 - xi[a])
            out[ci, b] = v
    return out


def mandel_B(d: int, xi, h, dtype=np.float64) -> np.ndarray:
    """Symmetrised-gradient matrix B_q (d* x d 2^d) at local point ``xi``.

    Mandel row (i, i): du_i/dx_i. Row (i, j), i != j: sqrt(2) * 1/2 (du_i/dx_j + du_j/dx_i).
    """
    grad = shape_gradients(d, xi, h, dtype)
    nc = 2 ** d
    B = np.zeros((d * (d + 1) // 2, d * nc), dtype=dtype)
    for m, (i, j) in enumerate(mandel_pairs(d)):
        for c in range(nc):
            if i == j:
                B[m, i * nc + c] += grad[c, i]
            else:
                s = dtype(1) / np.sqrt(dtype(2))
                B[m, i * nc + c] += s * grad[c, j]
                B[m, j * nc + c] += s * grad[c, i]
    return B


def isotropic_C(d: int, lam: float, mu: float) -> np.ndarray:
    """C_ijkl = lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk) as a Mandel matrix (paper Sec. 4).

    In 2D this is the plane-strain restriction (in-plane components of the 3D tensor).
    The matrix takes the floating-point type of lam and mu (at least FP64).
    """
    pairs = mandel_pairs(d)
    ds = len(pairs)
    dtype = np.result_type(np.asarray(lam).dtype, np.asarray(mu).dtype, np.float64).type
    C = np.zeros((ds, ds), dtype=dtype)

    def cijkl(i, j, k, l):
        dl = lambda a, b: dtype(1.0 if a == b else 0.0)  # noqa: E731
        return lam * dl(i, j) * dl(k, l) + mu * (dl(i, k) * dl(j, l) + dl(i, l) * dl(j, k))

    r2 = np.sqrt(dtype(2))
    for m, (i, j) in enumerate(pairs):
        for n, (k, l) in enumerate(pairs):
            wm = dtype(1) if i == j else r2
            wn = dtype(1) if k == l else r2
            C[m, n] = wm * wn * cijkl(i, j, k, l)
    return C


def lame_from_young(E: float, nu: float):
    """Lame constants of an isotropic solid (3D formulas; used as plane strain in 2D)."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def C_unit(d: int, nu: float, dtype=np.float64) -> np.ndarray:
    """Isotropic stiffness with unit Young's modulus and Poisson ratio ``nu`` (in ``dtype``)."""
    return isotropic_C(d, *lame_from_young(dtype(1.0), dtype(nu)))


ELEMENTS = ("q1", "p1")


def _mandel_from_gradients(grad: np.ndarray) -> np.ndarray:
    """Mandel symmetrised-gradient matrix (d* x d nc) from shape gradients [nc, d]."""
    nc, d = grad.shape
    dtype = grad.dtype.type
    B = np.zeros((d * (d + 1) // 2, d * nc), dtype=dtype)
    for m, (i, j) in enumerate(mandel_pairs(d)):
        for c in range(nc):
            if i == j:
                B[m, i * nc + c] += grad[c, i]
            else:
                s = dtype(1) / np.sqrt(dtype(2))
                B[m, i * nc + c] += s * grad[c, j]
                B[m, j * nc + c] += s * grad[c, i]
    return B


def triangle_pair_B(h, dtype=np.float64):
    """The P1 discretisation of a 2D voxel (Sec. 4 "Discretization": linear triangles):
    the voxel with corners (o0, o1) in {0,1}^2 is split along the diagonal from (0, 0)
    to (1, 1) into T1 = {(0,0), (1,0), (1,1)} and T2 = {(0,0), (1,1), (0,1)}. Each
    triangle has a constant strain; returns [B_T1, B_T2] on the voxel's 4 corners (the
    corner outside the triangle has zero columns) and the two weights (area h0 h1 / 2)."""
    h0, h1 = dtype(h[0]), dtype(h[1])
    one, zero = dtype(1), dtype(0)
    # corner order of corners(2): (0,0), (0,1), (1,0), (1,1)
    g1 = np.array([[-one / h0, zero], [zero, zero], [one / h0, -one / h1], [zero, one / h1]], dtype=dtype)
    g2 = np.array([[zero, -one / h1], [-one / h0, one / h1], [zero, zero], [one / h0, zero]], dtype=dtype)
    area = dtype(0.5) * h0 * h1
    return [_mandel_from_gradients(g1), _mandel_from_gradients(g2)], [area, area]


def element_points(d: int, h, element: str = "q1", dtype=np.float64):
    """Integration points of one voxel: the matrices B_q and weights w_q (sum = voxel
    volume) with K_e = sum_q w_q B_q^T C B_q. Q1: the 2^d Gauss points; P1 (2D): the two
    constant-strain triangles. In ``dtype`` (the element's type follows the material's)."""
    if element == "q1":
        pts, w = gauss_points(d, dtype)
        vol = dtype(1)
        for hb in h:
            vol = vol * dtype(hb)
        return [mandel_B(d, xi, h, dtype) for xi in pts], [wq * vol for wq in w]
    if element == "p1":
        if d != 2:
            raise ValueError("P1 triangles are 2D")
        return triangle_pair_B(h, dtype)
    raise ValueError(element)


def _float_type(*arrays):
    return np.result_type(*[np.asarray(a).dtype for a in arrays], np.float64).type


def element_matrix(d: int, h, C: np.ndarray, element: str = "q1") -> np.ndarray:
    """A = sum_q w_q B_q^T C B_q over the voxel's integration points (element_points), in
    the floating-point type of C (at least FP64)."""
    dtype = _float_type(C)
    Bs, ws = element_points(d, h, element, dtype)
    A = np.zeros((d * 2 ** d, d * 2 ** d), dtype=dtype)
    for B, wq in zip(Bs, ws):
        A += wq * (B.T @ C @ B)
    return A


def element_strain_load(d: int, h, C: np.ndarray, eps: np.ndarray, element: str = "q1") -> np.ndarray:
    """b = sum_q w_q B_q^T C eps for a constant Mandel strain ``eps`` (element part of f)."""
    dtype = _float_type(C, eps)
    Bs, ws = element_points(d, h, element, dtype)
    b = np.zeros(d * 2 ** d, dtype=dtype)
    for B, wq in zip(Bs, ws):
        b += wq * (B.T @ (C @ eps))
    return b
