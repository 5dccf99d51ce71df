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


def gauss_points(d: int):
    """The 2^d Gauss points of the reference cell [0,1]^d and their weights (sum 1)."""
    g = (0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0))
    pts = [tuple(g[i] for i in idx) for idx in itertools.product((0, 1), repeat=d)]
    w = [1.0 / 2 ** d] * len(pts)
    return pts, w


def shape_gradients(d: int, xi, h) -> np.ndarray:
    """dphi_c / dx_beta at local point ``xi`` for each corner c: array [2^d, d].

    phi_c(xi) = prod_a (xi_a if c_a == 1 else 1 - xi_a), x_a = h_a xi_a.
    """
    out = np.zeros((2 ** d, d))
    for ci, c in enumerate(corners(d)):
        for b in range(d):
            v = (1.0 if c[b] else -1.0) / h[b]
            for a in range(d):
                if a != b:
                    v *= xi[a] if c[a] else (1.0 - xi[a])
            out[ci, b] = v
    return out


def mandel_B(d: int, xi, h) -> np.ndarray:
    """Symmetrised-gradient matrix B_q (d* x d 2^d) at local point ``xi``.

    Mandel row (i, i): du_i/dx_i. Row (i, j), i != j: sqrt(2) * 1/2 (du_i/dx_j + du_j/dx_i).
    """
    grad = shape_gradients(d, xi, h)
    nc = 2 ** d
    B = np.zeros((d * (d + 1) // 2, d * nc))
    for m, (i, j) in enumerate(mandel_pairs(d)):
        for c in range(nc):
            if i == j:
                B[m, i * nc + c] += grad[c, i]
            else:
                s = 1.0 / math.sqrt(2.0)
                B[m, i * nc + c] += s * grad[c, j]
                B[m, j * nc + c] += s * grad[c, i]
    return B


def isotropic_C(d: int, lam: float, mu: float) -> np.ndarray:
    """C_ijkl = lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk) as a Mandel matrix (paper Sec. 4).

    In 2D this is the plane-strain restriction (in-plane components of the 3D tensor).
    """
    pairs = mandel_pairs(d)
    ds = len(pairs)
    C = np.zeros((ds, ds))

    def cijkl(i, j, k, l):
        dl = lambda a, b: 1.0 if a == b else 0.0  # noqa: E731
        return lam * dl(i, j) * dl(k, l) + mu * (dl(i, k) * dl(j, l) + dl(i, l) * dl(j, k))

    for m, (i, j) in enumerate(pairs):
        for n, (k, l) in enumerate(pairs):
            wm = 1.0 if i == j else math.sqrt(2.0)
            wn = 1.0 if k == l else math.sqrt(2.0)
            C[m, n] = wm * wn * cijkl(i, j, k, l)
    return C


def lame_from_young(E: float, nu: float):
    """Lame constants of an isotropic solid (3D formulas; used as plane strain in 2D)."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def C_unit(d: int, nu: float) -> np.ndarray:
    """Isotropic stiffness with unit Young's modulus and Poisson ratio ``nu``."""
    return isotropic_C(d, *lame_from_young(1.0, nu))


ELEMENTS = ("q1", "p1")


def _mandel_from_gradients(grad: np.ndarray) -> np.ndarray:
    """Mandel symmetrised-gradient matrix (d* x d nc) from shape gradients [nc, d]."""
    nc, d = grad.shape
    B = np.zeros((d * (d + 1) // 2, d * nc))
    for m, (i, j) in enumerate(mandel_pairs(d)):
        for c in range(nc):
            if i == j:
                B[m, i * nc + c] += grad[c, i]
            else:
                s = 1.0 / math.sqrt(2.0)
                B[m, i * nc + c] += s * grad[c, j]
                B[m, j * nc + c] += s * grad[c, i]
    return B


def triangle_pair_B(h):
    """The P1 discretisation of a 2D voxel (Sec. 4 "Discretization": linear triangles):
    the voxel with corners (o0, o1) in {0,1}^2 is split along the diagonal from (0, 0)
    to (1, 1) into T1 = {(0,0), (1,0), (1,1)} and T2 = {(0,0), (1,1), (0,1)}. Each
    triangle has a constant strain; returns [B_T1, B_T2] on the voxel's 4 corners (the
    corner outside the triangle has zero columns) and the two weights (area h0 h1 / 2)."""
    h0, h1 = float(h[0]), float(h[1])
    # corner order of corners(2): (0,0), (0,1), (1,0), (1,1)
    g1 = np.array([[-1.0 / h0, 0.0], [0.0, 0.0], [1.0 / h0, -1.0 / h1], [0.0, 1.0 / h1]])
    g2 = np.array([[0.0, -1.0 / h1], [-1.0 / h0, 1.0 / h1], [0.0, 0.0], [1.0 / h0, 0.0]])
    area = 0.5 * h0 * h1
    return [_mandel_from_gradients(g1), _mandel_from_gradients(g2)], [area, area]


def element_points(d: int, h, element: str = "q1"):
    """Integration points of one voxel: the matrices B_q and weights w_q (sum = voxel
    volume) with K_e = sum_q w_q B_q^T C B_q. Q1: the 2^d Gauss points; P1 (2D): the two
    constant-strain triangles."""
    if element == "q1":
        pts, w = gauss_points(d)
        vol = float(np.prod(h))
        return [mandel_B(d, xi, h) for xi in pts], [wq * vol for wq in w]
    if element == "p1":
        if d != 2:
            raise ValueError("P1 triangles are 2D")
        return triangle_pair_B(h)
    raise ValueError(element)


def element_matrix(d: int, h, C: np.ndarray, element: str = "q1") -> np.ndarray:
    """A = sum_q w_q B_q^T C B_q over the voxel's integration points (element_points)."""
    Bs, ws = element_points(d, h, element)
    A = np.zeros((d * 2 ** d, d * 2 ** d))
    for B, wq in zip(Bs, ws):
        A += wq * (B.T @ C @ B)
    return A


def element_strain_load(d: int, h, C: np.ndarray, eps: np.ndarray, element: str = "q1") -> np.ndarray:
    """b = sum_q w_q B_q^T C eps for a constant Mandel strain ``eps`` (element part of f)."""
    Bs, ws = element_points(d, h, element)
    b = np.zeros(d * 2 ** d)
    for B, wq in zip(Bs, ws):
        b += wq * (B.T @ (C @ eps))
    return b
