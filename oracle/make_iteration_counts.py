"""Write the oracle's PCG iteration counts for the 1024 x 1024 benchmark sweep.

Workload (2D plane strain, Q1): density from 16 Fourier modes with |k| <= 8 (seed 0),
E = 1/contrast + (1 - 1/contrast) rho^2 for contrast in {1e2, 1e4, 1e6}, nu = 0.3,
C_ref = mean material, the three Mandel unit loads solved separately, Green and
Green-Jacobi, relative residual 1e-8 (Sec. 4 "Termination criteria", relative form).
Each solve runs the oracle's textbook PCG (matrix-free K, support-form Alg. 1) to
completion under several rounding variants of the same arithmetic:

  fp64/blas                 FP64, inner products by numpy.dot
  fp64/sequential           FP64, inner products summed left to right
  extended/blas             everything derived from the FP64 inputs (E, nu) in
                            numpy.longdouble (64-bit significand on x86): C, element
                            matrix, symbol, diagonal, J^(1/2), right-hand side, and the
                            whole iteration (Green-Jacobi only)
  extended_iteration/blas   the FP64 setup arrays and right-hand side, the iteration in
                            numpy.longdouble (Green-Jacobi only)

Green-Jacobi PCG at this size amplifies differences of rounding size by roughly six
per iteration once its first Ritz values settle (about iteration 12), so its count is
set by rounding: by the arithmetic (the less accurate, the later it stops) and even by
the last bit of the setup arrays (the two extended variants differ only by rounding
C, the symbol and J^(1/2) to FP64 and stop up to four iterations apart). The GPU
parity test takes the range over the variants, widened by one, as the window for a
correct implementation of the same iteration. Green PCG does not amplify rounding (its
variants agree to ~1e-13 over the whole run) and is recorded in FP64 only.

Output: oracle/data/iters_2d_1024.json, read by the GPU count test and by the
CPU-baseline and reference legs of bench.py to scale their bounded samples.

    python -m oracle.make_iteration_counts [--workers 8] [--only fp64|extended|extended_iteration ...]

``--only`` recomputes the rows of the named precisions and keeps the file's other rows.
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
    contrast, pc, load, precision, order = args
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from oracle import assemble, fe, material, pcg, solve
    from synthetic import smooth_density
    rho = smooth_density(SHAPE, 16, 8.0, 0)
    E = material.young_from_density(rho, 1.0 / contrast, 1.0, 2.0)
    prob = solve.setup(SHAPE, E, 0.3, precision=precision)
    if precision == "extended":
        f = assemble.assemble_rhs(SHAPE, prob.E, prob.C, np.eye(3)[load])   # derived in extended precision
    else:
        f = assemble.assemble_rhs(SHAPE, E, fe.C_unit(2, 0.3), np.eye(3)[load]).astype(prob.E.dtype)
    t = time.time()
    res = pcg.pcg(prob.apply_K, prob.minv(pc), f, TOL, 100000, "rel", order)
    return {"contrast": contrast, "precond": pc, "load": load, "precision": precision, "dot": order,
            "iters": res.iters, "converged": bool(res.converged), "seconds": round(time.time() - t, 1)}


def jobs():
    out = []
    for c in CONTRASTS:
        for pc in PRECONDS:
            for g in range(3):
                out.append((c, pc, g, "fp64", "blas"))
                out.append((c, pc, g, "fp64", "sequential"))
                if pc == "green_jacobi":
                    out.append((c, pc, g, "extended", "blas"))
                    out.append((c, pc, g, "extended_iteration", "blas"))
    # longest first: Green at high contrast runs thousands of iterations
    cost = lambda j: (j[1] == "green") * j[0] + (j[3] != "fp64") * 5e3  # noqa: E731
    return sorted(out, key=cost, reverse=True)


def main():
    workers = 8
    if "--workers" in sys.argv:
        workers = int(sys.argv[sys.argv.index("--workers") + 1])
    only = set()
    if "--only" in sys.argv:
        only = set(sys.argv[sys.argv.index("--only") + 1:])
    todo = [j for j in jobs() if not only or j[3] in only]
    kept = []
    if only and os.path.exists(OUT):
        kept = [r for r in json.load(open(OUT))["solves"] if r["precision"] not in only]
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    with mp.get_context("spawn").Pool(workers) as pool:
        rows = kept + pool.map(_one, todo, chunksize=1)
    rows.sort(key=lambda r: (r["contrast"], r["precond"], r["load"], r["precision"], r["dot"]))
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    with open(OUT, "w") as fh:
        json.dump({"workload": "2D 1024x1024 Q1 plane strain, 16 modes |k|<=8 seed 0, E = 1/c + (1-1/c) rho^2, "
                               "nu 0.3, C_ref mean, Mandel unit loads, tol 1e-8 relative",
                   "oracle": "matrix-free K on corner differences, Alg. 1 over the impulse responses' support",
                   "variants": {"fp64/blas": "FP64, numpy.dot inner products",
                                "fp64/sequential": "FP64, inner products summed left to right",
                                "extended/blas": "setup and iteration in numpy.longdouble (x86: 64-bit significand) "
                                                 "from the FP64 inputs",
                                "extended_iteration/blas": "FP64 setup arrays, iteration in numpy.longdouble"},
                   "solves": rows}, fh, indent=1)
    print(OUT)


if __name__ == "__main__":
    main()
