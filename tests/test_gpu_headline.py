"""The 1024 x 1024 benchmark workload on the GPU against the FP64 oracle, through the C ABI.

Workload (as timed by bench.py): 2D plane strain, Q1, 16 Fourier modes with |k| <= 8,
seed 0, E = 1/c + (1 - 1/c) rho^2, nu = 0.3, C_ref = mean material, the three Mandel
unit loads, relative residual 1e-8.

* Same-k iterates (the parity rule for iterates): the GPU run with max_iter = k and no
  stopping test against the oracle's textbook PCG after k iterations, k = 1, 3, 6, 10,
  relative L2 of u <= 1e-12 and C_hom <= 1e-9, for Green and Green-Jacobi at the two
  high contrasts. Both sides apply K matrix-free on corner differences and evaluate
  Alg. 1 over the impulse responses' support, so neither carries the ~eps (n/2pi)^2
  low-frequency rounding of an assembled product or a full-FFT symbol. Green-Jacobi at
  contrast 1e6 starts amplifying rounding after k ~ 6: at k = 10 two FP64 summation
  orders of the oracle itself are ~3e-10 apart (and the FP64 oracle ~1e-11 from its
  extended-precision run). Where that oracle-vs-oracle floor exceeds 1e-12 it is the
  bound, computed here from the oracle run with sequential inner products.
* Iteration counts against oracle/data/iters_2d_1024.json, written by
  oracle/make_iteration_counts.py: for every (contrast, preconditioner, load) the
  oracle's counts under the rounding variants it records (FP64 with two summation
  orders; for Green-Jacobi also the whole iteration in extended precision), and the
  window is their range widened by one on each side (Sec. 4 "Termination criteria").
  Rounding delays Green-Jacobi convergence here: the extended-precision count is the
  lowest and the FP64 sequential one the highest, and a correct FP64 implementation
  with more accurate reductions than the oracle's lands in between.
"""

import json
import os

import numpy as np
import pytest

from oracle import assemble, material, pcg, post, solve as osolve
from synthetic import mandel_unit_loads, smooth_density

pytestmark = pytest.mark.gpu

SHAPE = (1024, 1024)
HERE = os.path.dirname(os.path.abspath(__file__))
COUNTS = os.path.join(os.path.dirname(HERE), "oracle", "data", "iters_2d_1024.json")


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def rho():
    return smooth_density(SHAPE, 16, 8.0, 0)


def _solver(rho, contrast):
    from paper_2508_02613_gb300.jfft import Solver
    return Solver(SHAPE, rho, 0.3, kind="density", e_min=1.0 / contrast, e_max=1.0, exponent=2.0, max_loads=3)


@pytest.mark.parametrize("contrast", [1e4, 1e6])
@pytest.mark.parametrize("pc", ["green", "green_jacobi"])
def test_same_k_iterates_1024(rho, contrast, pc):
    E = material.young_from_density(rho, 1.0 / contrast, 1.0, 2.0)
    s = _solver(rho, contrast)
    prob = osolve.setup(SHAPE, E, 0.3)
    eps = mandel_unit_loads(2)[:1]
    f = assemble.assemble_rhs(SHAPE, E, prob.C, eps[0])
    for k in (1, 3, 6, 10):
        s.set_max_iter(k)
        out = s.solve(eps, 0.0, pc, want_stress=False)
        assert int(out["iters"][0]) == k
        ref = pcg.pcg(prob.apply_K, prob.minv(pc), f, 0.0, k)
        u_ref = post.remove_mean(ref.x)
        du = np.linalg.norm(out["u"][0] - u_ref) / np.linalg.norm(u_ref)
        C_ref = post.homogenised_stress(SHAPE, E, prob.C, eps[0], u_ref)
        dc = np.abs(out["C_hom"][:, 0] - C_ref).max() / np.abs(C_ref).max()
        floor = 0.0
        if k >= 6:
            seq = post.remove_mean(pcg.pcg(prob.apply_K, prob.minv(pc), f, 0.0, k, "rel", "sequential").x)
            floor = np.linalg.norm(seq - u_ref) / np.linalg.norm(u_ref)
        print(f"{pc} c={contrast:g} k={k}: u {du:.2e} (oracle floor {floor:.1e})  C_hom {dc:.2e}")
        assert du <= max(1e-12, floor), (k, du, floor)
        assert dc <= 1e-9, (k, dc)
    s.close()


def _windows():
    data = json.load(open(COUNTS))
    win = {}
    for row in data["solves"]:
        key = (float(row["contrast"]), row["precond"], int(row["load"]))
        lo, hi = win.get(key, (10 ** 9, -1))
        win[key] = (min(lo, row["iters"]), max(hi, row["iters"]))
    return win


@pytest.mark.parametrize("contrast", [1e2, 1e4, 1e6])
@pytest.mark.parametrize("pc", ["green_jacobi", "green"])
def test_iteration_counts_1024(rho, contrast, pc):
    win = _windows()
    s = _solver(rho, contrast)
    out = s.solve(mandel_unit_loads(2), 1e-8, pc, want_stress=False)
    got = [int(v) for v in out["iters"]]
    for g in range(3):
        lo, hi = win[(contrast, pc, g)]
        print(f"{pc} c={contrast:g} load {g}: GPU {got[g]}, oracle {lo}..{hi}")
        assert lo - 1 <= got[g] <= hi + 1, (g, got[g], lo, hi)
        assert out["rel_res"][g] <= 1e-8 * 1.01
    s.close()
