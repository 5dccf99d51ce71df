"""Write the oracle's PCG iteration counts for the 1024 x 1024 benchmark sweep.

Workload (2D plane strain, Q1, FP64): density from 16 Fourier modes with |k| <= 8
(seed 0), E = 1/contrast + (1 - 1/contrast) rho^2 for contrast in {1e2, 1e4, 1e6},
nu = 0.3, C_ref = mean material, the three Mandel unit loads solved separately,
Green and Green-Jacobi, relative residual 1e-8. Each solve runs the oracle's
textbook PCG to completion. Green-Jacobi rows also record the count obtained with
the plane-wave closed-form symbol (green.closed_form_symbol) in place of Alg. 1:
at this size the Green-Jacobi count reacts to the rounding of Alg. 1's
low-frequency entries (relative ~4e-11), and the two counts bracket that spread.
Output: oracle/data/iters_2d_1024.json, read by the CPU-baseline and reference
legs of bench.py to scale their bounded samples.

    python -m oracle.make_iteration_counts [--workers 8] [--gj-bracket-only]
"""

from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
OUT = os.path.join(HERE, "data", "iters_2d_1024.json")

SHAPE = (1024, 1024)
CONTRASTS = (1e2, 1e4, 1e6)
PRECONDS = ("green_jacobi", "green")
TOL = 1e-8


def _one(args):
    contrast, pc, load, symbol = args
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from oracle import assemble, green, material, pcg, solve
    from synthetic import smooth_density
    rho = smooth_density(SHAPE, 16, 8.0, 0)
    E = material.young_from_density(rho, 1.0 / contrast, 1.0, 2.0)
    prob = solve.setup(SHAPE, E, 0.3)
    eps = np.eye(3)[load]
    f = assemble.assemble_rhs(SHAPE, E, prob.C, eps)
    minv = prob.minv(pc)
    if symbol == "closed_form":
        _, G = green.closed_form_symbol(SHAPE, float(E.mean()) * prob.C)
        minv = lambda r: green.apply_green_jacobi(G, prob.J_half, r)
    t = time.time()
    res = pcg.pcg(prob.apply_K, minv, f, TOL, 100000)
    return {"contrast": contrast, "precond": pc, "load": load, "symbol": symbol, "iters": res.iters,
            "converged": bool(res.converged), "seconds": time.time() - t}


def main():
    workers = 8
    if "--workers" in sys.argv:
        workers = int(sys.argv[sys.argv.index("--workers") + 1])
    bracket = [(c, "green_jacobi", g, "closed_form") for c in CONTRASTS for g in range(3)]
    if "--gj-bracket-only" in sys.argv and os.path.exists(OUT):
        old = json.load(open(OUT))
        rows = [r for r in old["solves"] if r.get("symbol", "alg1") == "alg1"]
        for r in rows:
            r.setdefault("symbol", "alg1")
        jobs = bracket
    else:
        rows = []
        jobs = [(c, pc, g, "alg1") for c in CONTRASTS for pc in PRECONDS for g in range(3)] + bracket
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    with mp.get_context("spawn").Pool(workers) as pool:
        rows += pool.map(_one, jobs)
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    with open(OUT, "w") as fh:
        json.dump({"workload": "2D 1024x1024 Q1 plane strain, 16 modes |k|<=8 seed 0, E = 1/c + (1-1/c) rho^2, "
                               "nu 0.3, C_ref mean, Mandel unit loads, tol 1e-8 relative",
                   "symbols": {"alg1": "Alg. 1 (real, even transform of the impulse responses)",
                               "closed_form": "plane-wave closed form without low-frequency cancellation"},
                   "solves": rows}, fh, indent=1)
    print(OUT)


if __name__ == "__main__":
    main()
