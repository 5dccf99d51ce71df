"""Write the oracle's PCG iteration counts for the 1024 x 1024 benchmark sweep.

Workload (2D plane strain, Q1): density from 16 Fourier modes with |k| <= 8 (seed 0),
E = 1/contrast + (1 - 1/contrast) rho^2 for contrast in {1e2, 1e4, 1e6}, nu = 0.3,
C_ref = mean material, the three Mandel unit loads solved separately, Green and
Green-Jacobi, relative residual 1e-8 (Sec. 4 "Termination criteria", relative form).
Each solve runs the oracle's textbook PCG (matrix-free K, support-form Alg. 1) to
completion under several rounding variants of the same arithmetic:

  fp64/blas        FP64, inner products by numpy.dot
  fp64/sequential  FP64, inner products summed left to right
  extended/blas    every vector, scalar, operator and transform in numpy.longdouble
                   (64-bit significand on x86; Green-Jacobi only)

Green-Jacobi PCG at this size amplifies rounding-level differences by roughly six per
iteration once its first Ritz values settle (about iteration 12), so its count depends
on the rounding: the less accurate the arithmetic, the later it stops. The extended
run is the least delayed; the FP64 sequential run the most. The GPU parity test takes
the range over the variants, widened by one, as the window for a correct
implementation of the same iteration. Green PCG does not amplify rounding (its
variants agree to ~1e-13 over the whole run) and is recorded in FP64 only.

Output: oracle/data/iters_2d_1024.json, read by the GPU count test and by the
CPU-baseline and reference legs of bench.py to scale their bounded samples.

    python -m oracle.make_iteration_counts [--workers 8]
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
    from oracle import assemble, material, pcg, solve
    from synthetic import smooth_density
    rho = smooth_density(SHAPE, 16, 8.0, 0)
    E = material.young_from_density(rho, 1.0 / contrast, 1.0, 2.0)
    prob = solve.setup(SHAPE, E, 0.3, precision=precision)
    f = assemble.assemble_rhs(SHAPE, E, prob.C, np.eye(3)[load]).astype(prob.E.dtype)
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
    # longest first: Green at high contrast runs thousands of iterations
    cost = lambda j: (j[1] == "green") * j[0] + (j[3] == "extended") * 5e3  # noqa: E731
    return sorted(out, key=cost, reverse=True)


def main():
    workers = 8
    if "--workers" in sys.argv:
        workers = int(sys.argv[sys.argv.index("--workers") + 1])
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    with mp.get_context("spawn").Pool(workers) as pool:
        rows = pool.map(_one, jobs(), chunksize=1)
    rows.sort(key=lambda r: (r["contrast"], r["precond"], r["load"], r["precision"], r["dot"]))
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    with open(OUT, "w") as fh:
        json.dump({"workload": "2D 1024x1024 Q1 plane strain, 16 modes |k|<=8 seed 0, E = 1/c + (1-1/c) rho^2, "
                               "nu 0.3, C_ref mean, Mandel unit loads, tol 1e-8 relative",
                   "oracle": "matrix-free K on corner differences, Alg. 1 over the impulse responses' support",
                   "variants": {"fp64/blas": "FP64, numpy.dot inner products",
                                "fp64/sequential": "FP64, inner products summed left to right",
                                "extended/blas": "numpy.longdouble throughout (x86: 64-bit significand)"},
                   "solves": rows}, fh, indent=1)
    print(OUT)


if __name__ == "__main__":
    main()
