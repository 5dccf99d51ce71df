"""The whole cell-problem solve, step by step (paper Secs. 2-4).

For each macroscopic load eps_bar_gamma (Mandel vector):
  1. K(rho) (applied matrix-free, B^T W C B element by element, or assembled) and
     f_gamma = -B^T W C(rho) eps_bar_gamma  (Eq. lin_system_exp);
  2. build the preconditioner: Green F^-1 G_hat F (Alg. 1, C_ref = mean(E) C_unit(nu)
     unless given), Jacobi diag(K)^-1 with the void rule, or Green-Jacobi
     J^(1/2) F^-1 G_hat F J^(1/2) (Eq. prec_lin_systemJG_2);
  3. PCG from x_0 = 0 to the stopping rule;
  4. remove the mean of the iterate per component; element-averaged stress and the
     homogenised stiffness column; true relative residual ||f - K u|| / ||f||.

The reference material only rescales the Green operator for the scaled-isotropic
material (C_ref = c C_unit): scaling M^-1 by 1/c scales z and p by 1/c and alpha
by c, so the PCG iterates are the same in exact arithmetic.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import assemble, fe, green, jacobi, pcg, post

PRECONDITIONERS = ("none", "green", "jacobi", "green_jacobi")


@dataclass
class CellProblem:
    """Assembled operator and preconditioner data for one material field."""
    n: tuple
    E: np.ndarray
    nu: float
    C: np.ndarray
    K: object
    G_hat: np.ndarray
    diag: np.ndarray
    J_half: np.ndarray
    element: str = "q1"
    operator: str = "matrix_free"

    @property
    def d(self):
        return len(self.n)

    def apply_K(self, u):
        if self.operator == "matrix_free":
            return assemble.apply_matrix_free(self.n, self.E, self.C, u, self.element)
        return assemble.apply(self.K, u)

    def minv(self, precond: str):
        if precond == "none":
            return lambda r: r.copy()
        if precond == "green":
            return lambda r: green.apply_green(self.G_hat, r)
        if precond == "jacobi":
            return lambda r: self.J_half * self.J_half * r
        if precond == "green_jacobi":
            return lambda r: green.apply_green_jacobi(self.G_hat, self.J_half, r)
        raise ValueError(precond)


def setup(n, E: np.ndarray, nu: float, C_ref: np.ndarray | None = None,
          void_replacement: float = 1.0, element: str = "q1", operator: str = "matrix_free",
          symbol: str = "support", precision: str = "fp64") -> CellProblem:
    """``element``: "q1" (bilinear / trilinear voxels, full Gauss rule) or "p1" (2D: each
    voxel split into two linear triangles, fe.triangle_pair_B).

    ``operator``: how PCG applies K. "matrix_free" (default) evaluates B^T W C B element
    by element on corner differences (assemble.apply_matrix_free, the matrix-free
    product of Sec. 3.1); "assembled" multiplies by the sparse matrix. Both are K; they
    differ only in rounding, which on the smooth fields of long solves is ~eps/theta for
    the first and ~eps/theta^2 for the second (theta the lowest grid frequency).
    ``symbol``: how step 2 of Alg. 1 transforms the impulse responses, "support"
    (default, green.support_transform) or "fft" (the full FFT, real and even part).
    ``precision``: "fp64"; "extended" (numpy.longdouble, 64-bit significand on x86) for
    everything derived from the FP64 inputs E and nu: C, the element matrix, the
    reference material, the Alg. 1 symbol, the diagonal (matrix-free, jacobi.
    diag_matrix_free), J^(1/2), and every PCG vector and scalar; or "extended_iteration",
    the FP64 setup arrays (C, symbol, J^(1/2)) cast to numpy.longdouble and only the
    iteration in extended precision. Both measure how far FP64 rounding moves the PCG
    iteration counts."""
    if operator not in ("matrix_free", "assembled"):
        raise ValueError(operator)
    if precision not in ("fp64", "extended", "extended_iteration"):
        raise ValueError(precision)
    if precision != "fp64" and (operator != "matrix_free" or symbol != "support"):
        raise ValueError("extended precision needs the matrix-free operator and the support-form symbol")
    n = tuple(int(k) for k in n)
    d = len(n)
    E = np.asarray(E, dtype=np.float64).reshape(n)
    C = fe.C_unit(d, nu)
    K = assemble.assemble_K(n, E, C, element)
    diag = jacobi.diag_assembled(K, (d,) + n)
    if precision == "extended":
        ld = np.longdouble
        E_l, C_l = E.astype(ld), fe.C_unit(d, nu, ld)
        C_ref_l = E_l.mean() * C_l if C_ref is None else np.asarray(C_ref).astype(ld)
        _, G_hat = green.green_symbol(n, C_ref_l, element=element, transform=symbol, dtype=ld)
        J_half = jacobi.jacobi_half(jacobi.diag_matrix_free(n, E_l, C_l, element), ld(void_replacement))
        return CellProblem(n, E_l, nu, C_l, K, G_hat, diag, J_half, element, operator)
    if C_ref is None:
        C_ref = float(E.mean()) * C
    _, G_hat = green.green_symbol(n, C_ref, element=element, transform=symbol)
    J_half = jacobi.jacobi_half(diag, void_replacement)
    if precision == "extended_iteration":
        ld = np.longdouble
        E, C, J_half, G_hat = E.astype(ld), C.astype(ld), J_half.astype(ld), G_hat.astype(ld)
    return CellProblem(n, E, nu, C, K, G_hat, diag, J_half, element, operator)


@dataclass
class SolveResult:
    u: np.ndarray          # [n_loads, d, *n], zero mean per component
    stress: np.ndarray     # [n_loads, d*, *n], element-averaged Mandel stress
    C_hom: np.ndarray      # [d*, n_loads]
    iters: np.ndarray      # [n_loads]
    rel_res: np.ndarray    # [n_loads] true ||f - K u|| / ||f|| (0 when f = 0)
    raw_u: np.ndarray      # [n_loads, d, *n] the PCG iterate before mean removal


def solve(prob: CellProblem, eps_bar: np.ndarray, tol: float, precond: str,
          max_iter: int = 100000, stop: str = "rel", dot_order: str = "blas",
          fixed_iters: np.ndarray | None = None) -> SolveResult:
    """Solve every load case. ``fixed_iters[g]`` runs exactly that many iterations with
    no stopping test (the same-k iterate comparison)."""
    eps_bar = np.atleast_2d(np.asarray(eps_bar, dtype=np.float64))
    nl = eps_bar.shape[0]
    us, raws, stresses, chom, its, rres = [], [], [], [], [], []
    minv = prob.minv(precond)
    for g in range(nl):
        f = assemble.assemble_rhs(prob.n, prob.E, prob.C, eps_bar[g], prob.element).astype(prob.E.dtype)
        if fixed_iters is not None:
            res = pcg.pcg(prob.apply_K, minv, f, 0.0, int(fixed_iters[g]), "rel", dot_order)
        else:
            res = pcg.pcg(prob.apply_K, minv, f, tol, max_iter, stop, dot_order)
        raw = res.x
        u = post.remove_mean(raw)
        nf = np.linalg.norm(f)
        rr = np.linalg.norm(f - prob.apply_K(u)) / nf if nf > 0 else 0.0
        us.append(u)
        raws.append(raw)
        stresses.append(post.element_stress(prob.n, prob.E, prob.C, eps_bar[g], u, prob.element))
        chom.append(post.homogenised_stress(prob.n, prob.E, prob.C, eps_bar[g], u, prob.element))
        its.append(res.iters)
        rres.append(rr)
    return SolveResult(np.stack(us), np.stack(stresses), np.stack(chom, axis=1),
                       np.array(its), np.array(rres), np.stack(raws))
