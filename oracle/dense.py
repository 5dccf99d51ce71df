"""Brute-force dense solve of K u = f on tiny grids (the exact target of every PCG run).

K is symmetric positive semidefinite with the rigid translations as its kernel
(paper Sec. 3.1); the solution is unique up to a constant per component, and the
zero-mean one is the minimum-norm least-squares solution (Moore-Penrose pseudo-
inverse), which ``numpy.linalg.lstsq`` returns.
"""

from __future__ import annotations

import numpy as np


def dense_solve(K, f: np.ndarray) -> np.ndarray:
    Kd = K.toarray() if hasattr(K, "toarray") else np.asarray(K)
    u, *_ = np.linalg.lstsq(Kd, f.reshape(-1), rcond=None)
    return u.reshape(f.shape)
