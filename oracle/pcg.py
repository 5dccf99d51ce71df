"""Textbook preconditioned conjugate gradients (paper Sec. 2.3 and footnote to Eq.
prec_lin_system_general: Saad, Iterative Methods, Alg. 9.1, symmetric form).

Start x_0 = 0 (paper Sec. 4 "Initial solution"), r_0 = f, z_0 = M^-1 r_0, p_0 = z_0,
gamma_0 = r_0 . z_0. Iteration k = 0, 1, ...:
    q = K p_k;  alpha = gamma_k / (p_k . q);  x += alpha p_k;  r -= alpha q
    stop if the residual test holds (the count is then k + 1)
    z = M^-1 r;  gamma_{k+1} = r . z;  beta = gamma_{k+1} / gamma_k;  p = z + beta p_k

Stopping rule. The paper stops on ||r_k||^2 <= eta with eta = 1e-10 (Sec. 4
"Termination criteria"); the benchmarks state a relative residual. Both are here:
``stop="rel"`` (default) tests ||r_k||_2 <= tol ||f||_2, ``stop="abs_sq"`` tests
||r_k||_2^2 <= tol. r is the recursively updated residual. ``iters`` is the number
of operator applications K p inside the loop (the test runs before each one), so a
right-hand side that already meets the test returns 0 iterations; f = 0 returns
x = 0 and 0 iterations.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def dot(a: np.ndarray, b: np.ndarray, order: str = "blas") -> float:
    """Inner product; ``order="sequential"`` sums left to right (for rounding-floor studies)."""
    a = a.reshape(-1)
    b = b.reshape(-1)
    if order == "sequential":
        return float(np.cumsum(a * b)[-1]) if a.size else 0.0
    return float(np.dot(a, b))


@dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    converged: bool
    res_norms: list = field(default_factory=list)  # ||r_k||_2, k = 0..iters


def pcg(apply_K, apply_Minv, f: np.ndarray, tol: float, max_iter: int,
        stop: str = "rel", dot_order: str = "blas") -> PCGResult:
    x = np.zeros_like(f)
    r = f.copy()
    rr = dot(r, r, dot_order)
    norm_f = np.sqrt(rr)
    hist = [norm_f]

    def done(rr_):
        if stop == "rel":
            return np.sqrt(rr_) <= tol * norm_f
        if stop == "abs_sq":
            return rr_ <= tol
        raise ValueError(stop)

    if norm_f == 0.0 or done(rr):
        return PCGResult(x, 0, True, hist)
    z = apply_Minv(r)
    p = z.copy()
    gamma = dot(r, z, dot_order)
    k = 0
    while k < max_iter:
        q = apply_K(p)
        alpha = gamma / dot(p, q, dot_order)
        x += alpha * p
        r -= alpha * q
        rr = dot(r, r, dot_order)
        hist.append(np.sqrt(rr))
        k += 1
        if done(rr):
            return PCGResult(x, k, True, hist)
        z = apply_Minv(r)
        gamma_new = dot(r, z, dot_order)
        beta = gamma_new / gamma
        gamma = gamma_new
        p = z + beta * p
    return PCGResult(x, k, False, hist)
