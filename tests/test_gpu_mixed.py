"""Mixed precision (FP32 inner PCG inside FP64 iterative refinement) against the
FP64 oracle, through the C ABI.

Tolerances: single FP32 applications are compared at 2e-6 (operator: sums of ~10
FP32 terms; preconditioner: FP32 transforms of log2 N stages) relative to the
oracle's max; solves are judged on the true FP64 relative residual, which the
refinement drives to the requested tolerance, and on the solution's distance to the
oracle's converged one, bounded rigorously by the residuals: for zero-mean u and u*
with K u* = f, ||u - u*|| <= ||f - K u|| / lambda_min, lambda_min the smallest
nonzero eigenvalue of K (dense spectrum of the oracle's K on these small grids)."""

import numpy as np
import pytest

from oracle import assemble, fe, material, solve as osolve
from synthetic import mandel_unit_loads, random_field, smooth_density

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _solver(shape, rho, contrast=1e4, **kw):
    from paper_2508_02613_gb300.jfft import Solver
    return Solver(shape, rho, 0.3, kind="density", e_min=1.0 / contrast, e_max=1.0, exponent=2.0,
                  precision="mixed", **kw)


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()


def error_bound(prob, f, u_a, u_b):
    """Bound on ||u_a - u_b|| for two approximate zero-mean solutions of K u = f: each is
    within ||f - K u|| / lambda_min of the exact zero-mean solution (u - u* is orthogonal to
    the rigid translations, the kernel of K, and K (u* - u) = f - K u)."""
    ev = np.linalg.eigvalsh(prob.K.toarray())
    lam_min = ev[ev > 1e-9 * ev.max()].min()
    ra = np.linalg.norm(f - prob.apply_K(u_a))
    rb = np.linalg.norm(f - prob.apply_K(u_b))
    return (ra + rb) / lam_min


@pytest.mark.parametrize("shape", [(8, 16), (64, 512), (8, 4, 16), (16, 16, 64), (8, 16, 64), (4, 64, 32),
                                   (16, 8, 128), (8, 32, 4)])
def test_fp32_operator_and_preconditioners(shape):
    d = len(shape)
    rho = smooth_density(shape, 8, 3.0, 1)
    E = material.young_from_density(rho, 1e-4, 1.0, 2.0)
    s = _solver(shape, rho)
    prob = osolve.setup(shape, E, 0.3)
    x = random_field((2, d) + shape, 3)
    want = np.stack([assemble.apply(prob.K, x[i]) for i in range(2)])
    assert rel(s.apply_K(x), want) <= 2e-6
    for pc in ("green", "green_jacobi", "jacobi"):
        z = s.apply_precond(pc, x)
        zw = np.stack([prob.minv(pc)(x[i]) for i in range(2)])
        assert rel(z, zw) <= 2e-6, pc


@pytest.mark.parametrize("pc", ["green", "green_jacobi"])
@pytest.mark.parametrize("tol", [1e-8, 1e-11])
@pytest.mark.parametrize("reliable", [False, True])
def test_mixed_solve_reaches_fp64_residual(pc, tol, reliable):
    """reliable: the FP32 recurrence continues across residual replacements (inner
    tolerance 0.1, so that the recurrence stays close to the true residual and is
    continued rather than restarted)."""
    shape = (32, 32)
    rho = smooth_density(shape, 16, 4.0, 0)
    E = material.young_from_density(rho, 1e-4, 1.0, 2.0)
    s = _solver(shape, rho, reliable=reliable, inner_tol=0.1 if reliable else 1e-3)
    eps = mandel_unit_loads(2)
    out = s.solve(eps, tol, pc)
    assert out["status"] == 0
    assert np.all(out["rel_res"] <= tol * 1.01)
    assert np.all(out["refine_steps"] >= 2)
    prob = osolve.setup(shape, E, 0.3)
    ref = osolve.solve(prob, eps, 1e-13, pc)
    dc = rel(out["C_hom"], ref.C_hom)
    for g in range(3):
        f = assemble.assemble_rhs(shape, E, prob.C, eps[g])
        du = np.linalg.norm(out["u"][g] - ref.u[g])
        bound = error_bound(prob, f, out["u"][g], ref.u[g])
        print(f"mixed {pc} tol {tol:g} load {g}: rel_res {out['rel_res'][g]:.2e}, u diff "
              f"{du / np.linalg.norm(ref.u[g]):.2e} (bound {bound / np.linalg.norm(ref.u[g]):.2e}), "
              f"C_hom diff {dc:.2e}, iters {out['iters'][g]}, refine {out['refine_steps'][g]}")
        assert du <= bound, (g, du, bound)
    assert dc <= 10 * tol, dc


def test_mixed_solve_3d_and_rhs():
    shape = (8, 8, 16)
    rho = smooth_density(shape, 8, 3.0, 4)
    E = material.young_from_density(rho, 1e-3, 1.0, 3.0)
    from paper_2508_02613_gb300.jfft import Solver
    s = Solver(shape, rho, 0.3, kind="density", e_min=1e-3, e_max=1.0, exponent=3.0, precision="mixed")
    eps = mandel_unit_loads(3)
    out = s.solve(eps, 1e-9, "green_jacobi")
    assert out["status"] == 0 and np.all(out["rel_res"] <= 1e-9 * 1.01)
    prob = osolve.setup(shape, E, 0.3)
    ref = osolve.solve(prob, eps, 1e-13, "green_jacobi")
    assert rel(out["C_hom"], ref.C_hom) <= 1e-8
    f = assemble.assemble_rhs(shape, E, prob.C, eps[5])
    r = s.solve_rhs(f[None], 1e-9, "green")
    assert r["status"] == 0
    u = r["u"][0] - r["u"][0].mean(axis=(1, 2, 3), keepdims=True)
    assert np.linalg.norm(f - assemble.apply(prob.K, u)) <= 1.01e-9 * np.linalg.norm(f)


def bf16_round(x):
    """Round to the nearest BF16 value (8 significant bits, ties to even), for normal
    positive inputs: x = m 2^e with 0.5 <= m < 1, m rounded to a multiple of 2^-8."""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.round(m * 256.0) / 256.0, e)


def test_bf16_rounding_helper():
    assert bf16_round(1.0) == 1.0 and bf16_round(1.0 + 2.0 ** -8) == 1.0       # tie -> even
    assert bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2 * 2.0 ** -7               # tie -> even (up)
    assert bf16_round(1.0 + 2.0 ** -7) == 1.0 + 2.0 ** -7                        # exact
    assert bf16_round(0.3) == 0.30078125


@pytest.mark.parametrize("shape", [(64, 512), (16, 16, 64)])
def test_bf16_material_operator(shape):
    """options.material_bf16: the FP32 operator equals the oracle's operator assembled
    with E rounded to BF16 (to FP32 accuracy), and differs from the unrounded one by
    the BF16 rounding of E."""
    d = len(shape)
    rho = smooth_density(shape, 8, 3.0, 1)
    E = material.young_from_density(rho, 1e-4, 1.0, 2.0)
    s = _solver(shape, rho, material_bf16=True)
    x = random_field((2, d) + shape, 3)
    got = s.apply_K(x)
    prob16 = osolve.setup(shape, bf16_round(E), 0.3)
    want16 = np.stack([assemble.apply(prob16.K, x[i]) for i in range(2)])
    assert rel(got, want16) <= 2e-6
    prob = osolve.setup(shape, E, 0.3)
    want = np.stack([assemble.apply(prob.K, x[i]) for i in range(2)])
    assert 1e-5 <= rel(got, want) <= 1e-2


@pytest.mark.parametrize("pc", ["green", "green_jacobi"])
@pytest.mark.parametrize("shape", [(32, 32), (8, 8, 16)])
def test_bf16_material_solve_reaches_fp64_residual(pc, shape):
    """The refinement's FP64 residual uses the FP64 E: the BF16 material copy changes
    the inner solves only, and the solve meets 1e-9 on the true operator."""
    d = len(shape)
    rho = smooth_density(shape, 16 if d == 2 else 8, 4.0 if d == 2 else 3.0, 0)
    E = material.young_from_density(rho, 1e-4, 1.0, 2.0)
    s = _solver(shape, rho, material_bf16=True)
    eps = mandel_unit_loads(d)
    out = s.solve(eps, 1e-9, pc)
    assert out["status"] == 0
    assert np.all(out["rel_res"] <= 1e-9 * 1.01)
    prob = osolve.setup(shape, E, 0.3)
    ref = osolve.solve(prob, eps, 1e-13, pc)
    assert rel(out["C_hom"], ref.C_hom) <= 1e-8
    for g in range(len(eps)):
        f = assemble.assemble_rhs(shape, E, prob.C, eps[g])
        assert np.linalg.norm(out["u"][g] - ref.u[g]) <= error_bound(prob, f, out["u"][g], ref.u[g]), g


def test_bf16_material_needs_mixed():
    from paper_2508_02613_gb300.jfft import JfftError, Solver
    with pytest.raises(JfftError):
        Solver((16, 16), np.ones((16, 16)), 0.3, material_bf16=True)
