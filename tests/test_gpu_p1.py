"""P1 triangles (each voxel split along its (0,0)-(1,1) diagonal, JFFT_ELEM_P1): GPU parity
with the FP64 oracle for every step of the path, with the tolerances of tests/test_gpu_parity.py."""

import numpy as np
import pytest

from oracle import assemble, dense, fe, green, jacobi, material, pcg, post, solve as osolve
from synthetic import laminate_density, mandel_unit_loads, random_field, smooth_density
from tests.test_gpu_parity import alg1_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _solver(shape, rho, contrast=1e4, **kw):
    from paper_2508_02613_gb300.jfft import Solver
    return Solver(shape, rho, 0.3, kind="density", e_min=1.0 / contrast, e_max=1.0, exponent=2.0, element="p1", **kw)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("shape", [(4, 4), (8, 16), (16, 8), (64, 128)])
def test_p1_operator_rhs_and_diagonal(shape):
    rho = smooth_density(shape, 8, 3.0, 1)
    E = material.young_from_density(rho, 1e-4, 1.0, 2.0)
    s = _solver(shape, rho)
    C = fe.C_unit(2, 0.3)
    K = assemble.assemble_K(shape, E, C, "p1")
    x = random_field((2, 2) + shape, 3)
    y = s.apply_K(x)
    want = np.stack([assemble.apply(K, x[i]) for i in range(2)])
    assert rel(y, want) <= 1e-13
    f = s.rhs(mandel_unit_loads(2))
    for g in range(3):
        assert rel(f[g], assemble.assemble_rhs(shape, E, C, mandel_unit_loads(2)[g], "p1")) <= 1e-13
    dg = jacobi.diag_assembled(K, (2,) + shape)
    assert rel(s.get_diag("closed_form"), dg) <= 1e-14
    assert rel(s.get_diag("combs"), dg) <= 1e-14


@pytest.mark.parametrize("shape", [(8, 16), (64, 128), (1024, 64), (64, 2048)])
@pytest.mark.parametrize("pc", ["green", "green_jacobi", "jacobi"])
def test_p1_preconditioners(shape, pc):
    rho = smooth_density(shape, 8, 3.0, 5)
    E = material.young_from_density(rho, 1e-4, 1.0, 2.0)
    s = _solver(shape, rho)
    prob = osolve.setup(shape, E, 0.3, element="p1")
    r = random_field((2, 2) + shape, 6)
    z = s.apply_precond(pc, r)
    want = np.stack([prob.minv(pc)(r[i]) for i in range(2)])
    assert rel(z, want) <= (alg1_tol(shape, 1e-13) if pc != "jacobi" else 1e-15)


@pytest.mark.parametrize("pc", ["green", "green_jacobi"])
def test_p1_converged_vs_dense(pc):
    shape = (8, 8)
    rho = smooth_density(shape, 6, 2.0, 9)
    E = material.young_from_density(rho, 1e-3, 1.0, 2.0)
    s = _solver(shape, rho, contrast=1e3)
    prob = osolve.setup(shape, E, 0.3, element="p1")
    eps = mandel_unit_loads(2)
    out = s.solve(eps, 1e-13, pc)
    for g in range(3):
        f = assemble.assemble_rhs(shape, E, prob.C, eps[g], "p1")
        want = dense.dense_solve(prob.K, f)
        assert np.linalg.norm(out["u"][g] - want) <= 1e-10 * np.linalg.norm(want)
        C_want = post.homogenised_stress(shape, E, prob.C, eps[g], want, "p1")
        assert rel(out["C_hom"][:, g], C_want) <= 1e-9
        assert rel(out["stress"][g], post.element_stress(shape, E, prob.C, eps[g], want, "p1")) <= 1e-9


def test_p1_laminate_closed_form():
    from tests.test_oracle_homogenisation import _laminate_C_hom
    from paper_2508_02613_gb300.jfft import Solver
    shape = (32, 8)
    rho = laminate_density(shape, 1e2)
    s = Solver(shape, rho, 0.3, element="p1")
    out = s.solve(mandel_unit_loads(2), 1e-13, "green_jacobi")
    layers = rho.reshape(shape[0], -1)[:, 0]
    want = _laminate_C_hom([e * fe.C_unit(2, 0.3) for e in layers], [0, 2], [1])
    assert rel(out["C_hom"], want) <= 1e-10


@pytest.mark.parametrize("pc", ["green", "green_jacobi"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_p1_32x32_workload(pc, precision):
    """The 32 x 32 workload on P1 triangles: iteration counts (FP64) within one of the
    oracle's range over two summation orders; mixed precision reaches the FP64 tolerance."""
    shape = (32, 32)
    rho = smooth_density(shape, 16, 4.0, 0)
    E = material.young_from_density(rho, 1e-4, 1.0, 2.0)
    s = _solver(shape, rho, precision=precision)
    eps = mandel_unit_loads(2)[:1]
    out = s.solve(eps, 1e-6, pc)
    prob = osolve.setup(shape, E, 0.3, element="p1")
    a = osolve.solve(prob, eps, 1e-6, pc)
    b = osolve.solve(prob, eps, 1e-6, pc, dot_order="sequential")
    if precision == "fp64":
        lo = min(int(a.iters[0]), int(b.iters[0])) - 1
        hi = max(int(a.iters[0]), int(b.iters[0])) + 1
        assert lo <= int(out["iters"][0]) <= hi, (int(out["iters"][0]), a.iters, b.iters)
    assert out["rel_res"][0] <= 1e-6 * 1.01
    assert np.linalg.norm(out["u"] - a.u) <= 10 * 1e-6 * np.linalg.norm(a.u)


def test_p1_is_2d_only():
    from paper_2508_02613_gb300.jfft import JfftError
    with pytest.raises(JfftError):
        _solver((8, 8, 8), np.ones((8, 8, 8)))
