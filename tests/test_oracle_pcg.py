"""Pins for the oracle's PCG and whole solve (no GPU)."""

import numpy as np
import pytest

from oracle import assemble, dense, fe, green, jacobi, material, pcg, post, solve
from synthetic import mandel_unit_loads, random_field, smooth_density, cosine_density


@pytest.mark.parametrize("shape", [(8, 8), (4, 4, 4)])
@pytest.mark.parametrize("pc", ["green", "green_jacobi"])
def test_homogeneous_material_converges_in_one_iteration(shape, pc):
    """E = c everywhere and C_ref proportional to C_unit: M^-1 K is a multiple of the zero-mean
    projection, so PCG stops after exactly one iteration for any zero-mean f."""
    d = len(shape)
    prob = solve.setup(shape, np.full(shape, 3.7), 0.3, C_ref=0.6 * fe.C_unit(d, 0.3))
    f = random_field((d,) + shape, 11, zero_mean=True)
    res = pcg.pcg(prob.apply_K, prob.minv(pc), f, 1e-12, 50)
    assert res.iters == 1 and res.converged
    want = dense.dense_solve(prob.K, f)
    got = post.remove_mean(res.x)
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


def test_homogeneous_macro_strain_gives_zero_iterations():
    shape = (8, 8)
    prob = solve.setup(shape, np.full(shape, 2.0), 0.3)
    out = solve.solve(prob, mandel_unit_loads(2), 1e-8, "green_jacobi")
    assert np.all(out.iters == 0)
    assert np.abs(out.u).max() == 0.0
    assert np.allclose(out.C_hom, 2.0 * fe.C_unit(2, 0.3), atol=1e-14)


@pytest.mark.parametrize("shape", [(8, 8), (4, 6), (4, 4, 4)])
@pytest.mark.parametrize("pc", ["green", "green_jacobi", "jacobi", "none"])
def test_pcg_matches_dense_brute_force(shape, pc):
    """Converged PCG equals the zero-mean pseudo-inverse solution of the assembled system."""
    d = len(shape)
    E = material.young_from_density(smooth_density(shape, 6, 2.0, 5), 1e-3, 1.0, 2.0)
    prob = solve.setup(shape, E, 0.3)
    eps = mandel_unit_loads(d)[-1]
    f = assemble.assemble_rhs(shape, E, prob.C, eps)
    want = dense.dense_solve(prob.K, f)
    res = pcg.pcg(prob.apply_K, prob.minv(pc), f, 1e-14, 5000)
    assert res.converged
    got = post.remove_mean(res.x)
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)


def test_green_and_green_jacobi_agree_up_to_the_mean():
    """Sec. 5.3: both preconditioners converge to the same solution; Green iterates keep zero
    mean, Green-Jacobi iterates carry a constant shift that mean removal takes out."""
    shape = (16, 16)
    E = material.young_from_density(smooth_density(shape, 8, 3.0, 1), 1e-4, 1.0, 2.0)
    prob = solve.setup(shape, E, 0.3)
    eps = mandel_unit_loads(2)[:1]
    g = solve.solve(prob, eps, 1e-13, "green")
    gj = solve.solve(prob, eps, 1e-13, "green_jacobi")
    assert np.abs(g.raw_u.mean(axis=(2, 3))).max() < 1e-14
    assert np.abs(gj.raw_u.mean(axis=(2, 3))).max() > 1e-6
    assert np.linalg.norm(g.u - gj.u) <= 1e-9 * np.linalg.norm(g.u)
    assert np.allclose(g.C_hom, gj.C_hom, rtol=1e-10, atol=1e-14)


def test_green_jacobi_beats_green_on_smooth_high_contrast():
    """Qualitative trend of Secs. 1 and 4.4 on a smooth contrast-1e4 field (not an exact pin)."""
    shape = (32, 32)
    E = material.young_from_density(smooth_density(shape, 16, 4.0, 0), 1e-4, 1.0, 2.0)
    prob = solve.setup(shape, E, 0.3)
    eps = mandel_unit_loads(2)[:1]
    it_g = solve.solve(prob, eps, 1e-6, "green").iters[0]
    it_gj = solve.solve(prob, eps, 1e-6, "green_jacobi").iters[0]
    assert it_gj < it_g


def test_void_replacement_value_does_not_change_iterations():
    """Sec. 3.2: with void regions, the value that replaces zero diagonal entries does not
    change the iteration count (the paper checked 1e-15 ... 1e15). Geometry: the Sec. 4.2
    cosine density with infinite contrast sampled on 4 x 4 pixels, each pixel covering
    4 x 4 voxels of a 16 x 16 grid, used directly as the stiffness scale (sigma = rho C eps)."""
    coarse = cosine_density((4, 4), float("inf"))
    rho = np.kron(coarse, np.ones((4, 4)))
    assert (rho == 0).sum() >= 16
    counts = []
    for rep in (1e-15, 1.0, 1e15):
        prob = solve.setup(rho.shape, rho, 0.3, C_ref=fe.C_unit(2, 0.3) * rho.mean(), void_replacement=rep)
        assert np.sum(prob.diag == 0) > 0
        f = assemble.assemble_rhs(rho.shape, rho, prob.C, np.array([1.0, 1.0, 0.0]))
        res = pcg.pcg(prob.apply_K, prob.minv("green_jacobi"), f, 1e-8, 999)
        assert res.converged
        counts.append(res.iters)
    assert counts[0] == counts[1] == counts[2]


def test_stop_rules_and_iteration_count_convention():
    shape = (16, 16)
    E = material.young_from_density(smooth_density(shape, 8, 3.0, 2), 1e-2, 1.0, 2.0)
    prob = solve.setup(shape, E, 0.3)
    f = assemble.assemble_rhs(shape, E, prob.C, np.array([1.0, 0, 0]))
    res = pcg.pcg(prob.apply_K, prob.minv("green"), f, 1e-6, 1000)
    h = np.array(res.res_norms)
    assert len(h) == res.iters + 1
    assert h[-1] <= 1e-6 * h[0] and h[-2] > 1e-6 * h[0]
    res2 = pcg.pcg(prob.apply_K, prob.minv("green"), f, 1e-10, 1000, stop="abs_sq")
    h2 = np.array(res2.res_norms)
    assert h2[-1] ** 2 <= 1e-10 < h2[-2] ** 2
    # fixed iteration count reproduces the same iterate
    fixed = pcg.pcg(prob.apply_K, prob.minv("green"), f, 0.0, res.iters)
    assert fixed.iters == res.iters and np.array_equal(fixed.x, res.x)


def test_dot_order_rounding_floor():
    """Reading of the parity rule. Two FP64 runs that differ only in the summation order of
    the CG inner products agree to ~1e-15 in the first iterations; later the CG recurrence
    amplifies rounding until the gap is comparable to the iteration error itself. So iterate
    parity at 1e-10 is a property of early iterations or of tightly converged solves, not of
    a run stopped at 1e-6: at tolerance tau both runs sit within ~tau of the exact solution.
    Their counts are not fixed to one either: rounding delays Green-Jacobi convergence, so
    the same iteration run in extended precision stops first and the FP64 runs stop up to
    a few iterations later, the less accurate summation order last."""
    shape = (32, 32)
    E = material.young_from_density(smooth_density(shape, 16, 4.0, 0), 1e-4, 1.0, 2.0)
    prob = solve.setup(shape, E, 0.3)
    f = assemble.assemble_rhs(shape, E, prob.C, np.array([1.0, 0, 0]))
    exact = dense.dense_solve(prob.K, f)
    nrm = np.linalg.norm(exact)
    for k in (1, 5, 10):
        a = pcg.pcg(prob.apply_K, prob.minv("green_jacobi"), f, 0.0, k, dot_order="blas").x
        b = pcg.pcg(prob.apply_K, prob.minv("green_jacobi"), f, 0.0, k, dot_order="sequential").x
        assert np.linalg.norm(post.remove_mean(a) - post.remove_mean(b)) <= 1e-13 * nrm
    ext = solve.setup(shape, E, 0.3, precision="extended")
    for tol in (1e-6, 1e-12):
        a = pcg.pcg(prob.apply_K, prob.minv("green_jacobi"), f, tol, 5000, dot_order="blas")
        b = pcg.pcg(prob.apply_K, prob.minv("green_jacobi"), f, tol, 5000, dot_order="sequential")
        e = pcg.pcg(ext.apply_K, ext.minv("green_jacobi"), f.astype(ext.E.dtype), tol, 5000)
        assert e.iters - 1 <= min(a.iters, b.iters) and max(a.iters, b.iters) <= e.iters + 3
        ua, ub = post.remove_mean(a.x), post.remove_mean(b.x)
        assert np.linalg.norm(ua - exact) <= 10 * tol * nrm
        assert np.linalg.norm(ua - ub) <= 10 * tol * nrm


def test_filtered_inclusion_trend():
    """The motivating example of Sec. 1 (compliant circular inclusion, contrast 1e4,
    repeated [1 2 1]/4 filtering): with the sharp interface Green needs fewer iterations
    than Green-Jacobi; after smoothing Green needs many more and Green-Jacobi fewer.
    Qualitative (the paper plots the trend on 256^2, no counts are printed)."""
    from oracle import assemble, solve
    from synthetic import circular_inclusion, gaussian_filter
    shape = (64, 64)
    rho0 = circular_inclusion(shape)
    its = {}
    for i in (0, 8):
        rho = gaussian_filter(rho0, i)
        prob = solve.setup(shape, rho, 0.3)
        f = assemble.assemble_rhs(shape, rho, prob.C, np.eye(3)[0])
        its[i] = {pc: pcg.pcg(prob.apply_K, prob.minv(pc), f, 1e-6, 100000).iters
                  for pc in ("green", "green_jacobi")}
    assert its[0]["green"] < its[0]["green_jacobi"]
    assert its[8]["green_jacobi"] < its[8]["green"]
    assert its[8]["green"] > 5 * its[0]["green"]
    assert its[8]["green_jacobi"] < its[0]["green_jacobi"]


def test_extended_iterates_agree_with_fp64_before_amplification():
    """The extended-precision PCG (setup and iteration) and the FP64 one agree to rounding
    for the first iterations, at 64^2 Green-Jacobi, contrast 1e4."""
    if np.finfo(np.longdouble).eps > 1e-18:
        pytest.skip("no extended precision type on this platform")
    shape = (64, 64)
    E = material.young_from_density(smooth_density(shape, 16, 8.0, 0), 1e-4, 1.0, 2.0)
    a = solve.setup(shape, E, 0.3)
    b = solve.setup(shape, E, 0.3, precision="extended")
    fa = assemble.assemble_rhs(shape, a.E, a.C, np.eye(3)[0])
    fb = assemble.assemble_rhs(shape, b.E, b.C, np.eye(3)[0])
    assert fb.dtype == np.longdouble
    for k in (1, 5):
        xa = pcg.pcg(a.apply_K, a.minv("green_jacobi"), fa, 0.0, k).x
        xb = pcg.pcg(b.apply_K, b.minv("green_jacobi"), fb, 0.0, k).x.astype(np.float64)
        assert np.linalg.norm(xa - xb) <= 1e-13 * np.linalg.norm(xa)
