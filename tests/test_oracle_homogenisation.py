"""Pins for the oracle's homogenised stiffness (no GPU)."""

import numpy as np
import pytest

from oracle import fe, material, solve
from synthetic import laminate_density, mandel_unit_loads, smooth_density


def _laminate_C_hom(Cs: np.ndarray, normal_idx, tangent_idx):
    """Exact effective stiffness of a laminate with layer normal e_1 (rank-one lamination).

    Across the layers the tangential strains and the normal stresses are continuous and
    constant; averaging eps_N and sigma_T over the equally thick layers gives, with
    A = <C_NN^-1>, B = <C_NN^-1 C_NT>, P = <C_TN C_NN^-1>:
      C_NN* = A^-1,  C_NT* = A^-1 B,  C_TN* = P A^-1,
      C_TT* = <C_TT> - <C_TN C_NN^-1 C_NT> + P A^-1 B.
    ``Cs`` holds one Mandel stiffness per layer."""
    N, T = list(normal_idx), list(tangent_idx)
    inv = [np.linalg.inv(C[np.ix_(N, N)]) for C in Cs]
    A = np.mean(inv, axis=0)
    B = np.mean([iv @ C[np.ix_(N, T)] for iv, C in zip(inv, Cs)], axis=0)
    P = np.mean([C[np.ix_(T, N)] @ iv for iv, C in zip(inv, Cs)], axis=0)
    Ctt = np.mean([C[np.ix_(T, T)] - C[np.ix_(T, N)] @ iv @ C[np.ix_(N, T)] for iv, C in zip(inv, Cs)], axis=0)
    Ai = np.linalg.inv(A)
    ds = Cs[0].shape[0]
    out = np.zeros((ds, ds))
    out[np.ix_(N, N)] = Ai
    out[np.ix_(N, T)] = Ai @ B
    out[np.ix_(T, N)] = P @ Ai
    out[np.ix_(T, T)] = Ctt + P @ Ai @ B
    return out


@pytest.mark.parametrize("shape,normal,tangent", [((16, 8), [0, 2], [1]), ((8, 4, 4), [0, 4, 5], [1, 2, 3])])
@pytest.mark.parametrize("pc", ["green", "green_jacobi"])
def test_laminate_matches_closed_form(shape, normal, tangent, pc):
    """Layered material (Sec. 4.1 geometry, contrast 1e2): the Q1 space contains the exact
    piecewise-linear solution, so the FE homogenised stiffness equals the lamination formula."""
    d = len(shape)
    rho = laminate_density(shape, 1e2)
    Cu = fe.C_unit(d, 0.3)
    prob = solve.setup(shape, rho, 0.3)
    out = solve.solve(prob, mandel_unit_loads(d), 1e-13, pc)
    layers = rho.reshape(shape[0], -1)[:, 0]
    want = _laminate_C_hom([e * Cu for e in layers], normal, tangent)
    assert np.abs(out.C_hom - want).max() <= 1e-11 * np.abs(want).max()


@pytest.mark.parametrize("p,n", [(4, 16), (8, 32), (2, 8)])
def test_coarse_geometry_on_a_finer_grid(p, n):
    """Geometry G_p on T_n (Sec. 4, n >= p): every voxel takes its pixel's value, so a
    laminate of p layers keeps the lamination formula of p equally thick layers on
    every finer grid."""
    rng = np.random.default_rng(p * n)
    layers = 10.0 ** rng.uniform(-2, 0, p)
    coarse = np.repeat(layers[:, None], p, axis=1)           # G_p, layers normal to e_1
    fine = material.upsample(coarse, (n, n))
    # brute force: voxel (i, j) belongs to pixel (i // (n/p), j // (n/p))
    r = n // p
    want_fine = np.array([[coarse[i // r, j // r] for j in range(n)] for i in range(n)])
    assert np.array_equal(fine, want_fine)
    prob = solve.setup((n, n), fine, 0.3)
    out = solve.solve(prob, mandel_unit_loads(2), 1e-13, "green_jacobi")
    want = _laminate_C_hom([e * fe.C_unit(2, 0.3) for e in layers], [0, 2], [1])
    assert np.abs(out.C_hom - want).max() <= 1e-11 * np.abs(want).max()


@pytest.mark.parametrize("shape", [(16, 16), (6, 6, 6)])
def test_hill_bounds_symmetry_and_energy(shape):
    """Reuss <= C_hom <= Voigt (Loewner order), C_hom symmetric, and the macroscopic energy
    equals the cell-averaged stress power of the solved field."""
    d = len(shape)
    E = material.young_from_density(smooth_density(shape, 8, 3.0, 9), 1e-3, 1.0, 2.0)
    prob = solve.setup(shape, E, 0.3)
    out = solve.solve(prob, mandel_unit_loads(d), 1e-12, "green_jacobi")
    Ch = out.C_hom
    assert np.abs(Ch - Ch.T).max() <= 1e-9 * np.abs(Ch).max()
    Cu = fe.C_unit(d, 0.3)
    voigt = E.mean() * Cu
    reuss = Cu / np.mean(1.0 / E)
    scale = np.abs(voigt).max()
    assert np.linalg.eigvalsh(voigt - 0.5 * (Ch + Ch.T)).min() > -1e-12 * scale
    assert np.linalg.eigvalsh(0.5 * (Ch + Ch.T) - reuss).min() > -1e-12 * scale
    # strict improvement over both bounds for a non-uniform field
    assert np.linalg.eigvalsh(voigt - Ch).max() > 1e-6 * scale
    assert out.rel_res.max() < 1e-11
    # energy: eps_bar . C_hom eps_bar = <(eps_bar + B u) . E C (eps_bar + B u)>, which at
    # the solution of K u = f is eps_bar^T C_Voigt eps_bar - f . u
    from oracle import assemble
    for g, eps in enumerate(mandel_unit_loads(d)):
        f = assemble.assemble_rhs(shape, E, prob.C, eps)
        energy = eps @ voigt @ eps - float(np.sum(f * out.u[g]))
        assert abs(Ch[g, g] - energy) <= 1e-10 * abs(energy)
