"""Pins for the oracle's assembled operator, right-hand side, Green symbol (Alg. 1) and
Jacobi diagonal (Alg. 2). No GPU."""

import json
import math
import os

import numpy as np
import pytest

from oracle import assemble, fe, green, jacobi, material, solve
from synthetic import random_field, smooth_density

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _E(shape, seed=0):
    rho = smooth_density(shape, 4, 2.0, seed)
    return 1e-2 + rho


@pytest.mark.parametrize("shape", [(4, 4), (8, 8), (4, 6), (4, 4, 4)])
def test_K_symmetric_psd_with_translation_kernel(shape):
    """K is symmetric positive semidefinite; its kernel is exactly the d rigid translations (Sec. 3.1)."""
    d = len(shape)
    K = assemble.assemble_K(shape, _E(shape), fe.C_unit(d, 0.3))
    Kd = K.toarray()
    assert np.abs(Kd - Kd.T).max() <= 1e-15 * np.abs(Kd).max()
    ev = np.linalg.eigvalsh(Kd)
    tol = 1e-11 * ev.max()
    assert ev.min() > -tol
    assert np.sum(np.abs(ev) < tol) == d
    for a in range(d):
        t = np.zeros((d,) + shape)
        t[a] = 1.0
        assert np.abs(assemble.apply(K, t)).max() < 1e-13


def test_energy_is_sum_of_element_energies():
    """u^T K u equals the sum over elements of E_e u_e^T A u_e (B^T W C B built per element)."""
    shape = (6, 4)
    E = _E(shape, 1)
    C = fe.C_unit(2, 0.3)
    K = assemble.assemble_K(shape, E, C)
    u = random_field((2,) + shape, 5)
    A = fe.element_matrix(2, assemble.grid_spacing(shape), C)
    g = assemble.element_dofs(shape)
    ue = u.reshape(-1)[g]
    want = np.sum(E.reshape(-1) * np.einsum("ea,ab,eb->e", ue, A, ue))
    got = u.reshape(-1) @ (K @ u.reshape(-1))
    assert math.isclose(got, want, rel_tol=1e-13)


@pytest.mark.parametrize("shape", [(8, 8), (4, 4, 4)])
def test_rhs_consistent_and_zero_for_uniform_material(shape):
    """f is orthogonal to the translations; a uniform material has f = 0 for any macro strain."""
    d = len(shape)
    C = fe.C_unit(d, 0.3)
    ds = d * (d + 1) // 2
    eps = np.arange(1, ds + 1, dtype=float)
    f = assemble.assemble_rhs(shape, _E(shape, 2), C, eps)
    assert np.abs(f.reshape(d, -1).sum(axis=1)).max() < 1e-13
    assert np.abs(f).max() > 1e-3
    f0 = assemble.assemble_rhs(shape, np.full(shape, 3.0), C, eps)
    assert np.abs(f0).max() < 1e-13


def _closed_form_symbol(shape, lam, mu):
    """Q1 symbol derived by hand from plane waves (full Gauss rule), not from Alg. 1:
    S_a = 2 (h/3)^(d-2) ... (1 - cos t_a) prod_{b != a} (2 + cos t_b) / 3^(...)
    2D: S_1 = 2/3 (1-c1)(2+c2), K12 = (lam+mu) s1 s2.
    3D: S_1 = 2h/9 (1-c1)(2+c2)(2+c3), K12 = (lam+mu) h/3 s1 s2 (2+c3).
    K_aa = (lam+2mu) S_a + mu sum_{b!=a} S_b."""
    d = len(shape)
    th = np.meshgrid(*[2 * np.pi * np.arange(k) / k for k in shape], indexing="ij")
    c = [np.cos(t) for t in th]
    s = [np.sin(t) for t in th]
    h = 1.0 / shape[0]
    K = np.zeros((d, d) + tuple(shape))
    if d == 2:
        S = [2 / 3 * (1 - c[0]) * (2 + c[1]), 2 / 3 * (1 - c[1]) * (2 + c[0])]
        K[0, 1] = K[1, 0] = (lam + mu) * s[0] * s[1]
    else:
        S = [2 * h / 9 * (1 - c[a]) * np.prod([2 + c[b] for b in range(3) if b != a], axis=0) for a in range(3)]
        for a in range(3):
            for b in range(3):
                if a != b:
                    o = 3 - a - b
                    K[a, b] = (lam + mu) * h / 3 * s[a] * s[b] * (2 + c[o])
    for a in range(d):
        K[a, a] = (lam + 2 * mu) * S[a] + mu * sum(S[b] for b in range(d) if b != a)
    return K


@pytest.mark.parametrize("shape", [(4, 4), (8, 8), (6, 6, 6)])
def test_alg1_symbol_matches_closed_form(shape):
    d = len(shape)
    lam, mu = 0.7, 0.4
    K_hat, G_hat = green.green_symbol(shape, fe.isotropic_C(d, lam, mu))
    assert np.abs(K_hat.imag).max() < 1e-13
    want = _closed_form_symbol(shape, lam, mu)
    assert np.abs(K_hat.real - want).max() < 1e-13
    # symmetric, zero frequency pinned, inverse elsewhere
    assert np.abs(K_hat - np.swapaxes(K_hat, 0, 1)).max() < 1e-14
    assert np.abs(G_hat[(slice(None), slice(None)) + (0,) * d]).max() == 0.0
    Kb = np.moveaxis(K_hat.reshape(d, d, -1), 2, 0)[1:]
    Gb = np.moveaxis(G_hat.reshape(d, d, -1), 2, 0)[1:]
    assert np.abs(Kb @ Gb - np.eye(d)).max() < 1e-10
    # positive definite away from the zero frequency (Nyquist included)
    assert np.linalg.eigvalsh(Kb.real).min() > 0


@pytest.mark.parametrize("shape", [(8, 8), (16, 8), (4, 8, 4)])
def test_alg1_transform_is_real_and_even_up_to_rounding(shape):
    """The impulse response of the uniform Q1 operator is even in the node offset, so its
    transform is real and even; the oracle's real, even symbol removes rounding only. A
    wrong impulse position or a transposed response would leave O(1) imaginary parts."""
    d = len(shape)
    axes = tuple(range(2, 2 + d))
    C = fe.C_unit(d, 0.3)
    R = green.impulse_responses(shape, C)
    K_c = np.fft.fftn(R, axes=axes)
    scale = np.abs(R).sum(axis=axes).max()
    assert np.abs(K_c.imag).max() <= 1e-14 * scale
    reflected = np.roll(np.flip(K_c, axes), 1, axes)
    assert np.abs(K_c - reflected).max() <= 1e-14 * scale
    K_hat, G_hat = green.green_symbol(shape, C)
    assert K_hat.dtype == np.float64 and G_hat.dtype == np.float64
    assert np.abs(K_hat - K_c.real).max() <= 1e-14 * scale
    assert np.array_equal(K_hat, np.roll(np.flip(K_hat, axes), 1, axes))


@pytest.mark.parametrize("pc", ["green", "green_jacobi"])
def test_preconditioners_are_symmetric(pc):
    """M^-1 is symmetric (PCG's requirement): a . M b = b . M a for arbitrary fields."""
    shape = (32, 16)
    rho = smooth_density(shape, 16, 8.0, 0)
    E = material.young_from_density(rho, 1e-3, 1.0, 2.0)
    prob = solve.setup(shape, E, 0.3)
    M = prob.minv(pc)
    a = random_field((2,) + shape, 1)
    b = random_field((2,) + shape, 2)
    Mb, Ma = M(b), M(a)
    assert abs(np.vdot(a, Mb) - np.vdot(b, Ma)) <= 1e-15 * np.linalg.norm(a) * np.linalg.norm(Mb) * 16


@pytest.mark.parametrize("shape", [(8, 8), (32, 32), (4, 4, 4), (8, 8, 8), (4, 8), (16, 4), (4, 8, 16), (8, 4, 4)])
def test_closed_form_symbol_equals_alg1(shape):
    """The oracle's plane-wave closed form (rectangular elements h_a = 1/n_a) equals Alg. 1
    with the explicit DFT of the assembled operator's impulse responses, and, on square /
    cubic grids, the hand-derived formula of this file."""
    d = len(shape)
    C = 0.8 * fe.C_unit(d, 0.3)
    K1, G1 = green.green_symbol(shape, C, explicit_dft=True)
    K2, G2 = green.closed_form_symbol(shape, C)
    assert np.abs(K1 - K2).max() <= 1e-13 * np.abs(K1).max()
    assert np.abs(G1 - G2).max() <= 1e-12 * np.abs(G1).max()
    if len(set(shape)) == 1:
        lam, mu = float(C[0, 1]), 0.5 * float(C[0, 0] - C[0, 1])
        assert np.abs(K2 - _closed_form_symbol(shape, lam, mu)).max() <= 1e-13 * np.abs(K2).max()


def test_library_fft_equals_explicit_dft():
    """numpy.fft (used as a library step) agrees with the explicit O(N^2) DFT, both in the
    symbol and in the application of the Green operator."""
    shape = (4, 6)
    C = fe.C_unit(2, 0.3)
    K1, G1 = green.green_symbol(shape, C)
    K2, G2 = green.green_symbol(shape, C, explicit_dft=True)
    assert np.abs(K1 - K2).max() < 1e-13
    r = random_field((2,) + shape, 4)
    assert np.abs(green.apply_green(G1, r) - green.apply_green(G2, r, explicit_dft=True)).max() < 1e-12


@pytest.mark.parametrize("shape", [(8, 4), (4, 4, 2)])
def test_green_is_pseudo_inverse_of_reference_operator(shape):
    """K_ref u = F^-1 K_hat F u (block circulant), and G K_ref u = u - mean(u)."""
    d = len(shape)
    C = fe.C_unit(d, 0.3) * 2.0
    K_ref = assemble.assemble_K(shape, np.ones(shape), C)
    K_hat, G_hat = green.green_symbol(shape, C)
    u = random_field((d,) + shape, 7)
    axes = tuple(range(1, d + 1))
    Ku_fft = np.fft.ifftn(np.einsum("ab...,a...->b...", K_hat, np.fft.fftn(u, axes=axes)), axes=axes).real
    assert np.abs(Ku_fft - assemble.apply(K_ref, u)).max() < 1e-12
    z = green.apply_green(G_hat, assemble.apply(K_ref, u))
    um = u - u.mean(axis=axes, keepdims=True)
    assert np.abs(z - um).max() < 1e-11
    assert np.abs(green.apply_green(G_hat, u).mean(axis=axes)).max() < 1e-14


@pytest.mark.parametrize("shape", [(8, 8), (4, 6), (4, 4, 4)])
def test_alg2_comb_diagonal(shape):
    """Alg. 2 (d 2^d applications, count printed in Sec. 3.3) equals the assembled diagonal and
    the closed form kappa * sum of the E of the 2^d voxels around each node."""
    with open(os.path.join(GOLDEN, "paper_constants.json")) as fh:
        cost = json.load(fh)["jacobi_assembly_cost"]
    d = len(shape)
    E = _E(shape, 3)
    C = fe.C_unit(d, 0.3)
    K = assemble.assemble_K(shape, E, C)
    dg, count = jacobi.diag_alg2(lambda u: assemble.apply(K, u), d, shape)
    assert count == cost[str(d)]
    da = jacobi.diag_assembled(K, (d,) + shape)
    assert np.abs(dg - da).max() <= 1e-15 * np.abs(da).max()
    # closed form: each corner of a voxel contributes E_e * A[(a,c),(a,c)]; the diagonal of A
    # is corner independent (reflection symmetry of the element)
    A = fe.element_matrix(d, assemble.grid_spacing(shape), C)
    nc = 2 ** d
    Esum = np.zeros(shape)
    for o in fe.corners(d):
        Esum += np.roll(E, shift=o, axis=tuple(range(d)))
    for a in range(d):
        kap = A[a * nc, a * nc]
        assert np.allclose(np.diag(A)[a * nc:(a + 1) * nc], kap, rtol=1e-14)
        assert np.abs(da[a] - kap * Esum).max() <= 1e-14 * np.abs(da[a]).max()


def test_plane_strain_diag_closed_form():
    """Square Q1 element in plane strain: the diagonal entry is (lam + 3 mu) / 3 (the textbook
    plane-stress value E/(1-nu^2)(1/2 - nu/6) with lam replaced by the plane-strain lam)."""
    lam, mu = fe.lame_from_young(1.0, 0.3)
    A = fe.element_matrix(2, (1.0, 1.0), fe.isotropic_C(2, lam, mu))
    assert np.allclose(np.diag(A), (lam + 3 * mu) / 3, rtol=1e-14)


def test_void_rule():
    """Nodes whose surrounding voxels are all void get diagonal 1 (Sec. 3.2)."""
    shape = (8, 8)
    E = _E(shape, 4)
    E[2:5, 2:5] = 0.0  # node (3,3)..(4,4) is surrounded by void voxels
    K = assemble.assemble_K(shape, E, fe.C_unit(2, 0.3))
    dg = jacobi.diag_assembled(K, (2,) + shape)
    assert np.all(dg[:, 3:5, 3:5] == 0.0)
    assert np.all(jacobi.void_rule(dg)[:, 3:5, 3:5] == 1.0)
    jh = jacobi.jacobi_half(dg)
    assert np.all(np.isfinite(jh)) and np.all(jh[:, 3:5, 3:5] == 1.0)


# ---- Alg. 1 step 2 over the impulse responses' support, and the matrix-free operator


@pytest.mark.parametrize("shape,element", [((4, 4), "q1"), ((8, 4), "q1"), ((4, 8, 4), "q1"), ((8, 8), "p1"),
                                           ((4, 16), "p1")])
def test_support_transform_equals_explicit_dft(shape, element):
    """The support form of step 2 is the DFT of the impulse responses: equal to the explicit
    O(N^2) DFT (real, even part); the responses live on the 3^d nodes next to node 0."""
    d = len(shape)
    C = 0.9 * fe.C_unit(d, 0.28)
    R = green.impulse_responses(shape, C, element)
    far = np.ones(shape, dtype=bool)
    far[np.ix_(*[[0, 1, m - 1] for m in shape])] = False
    assert np.abs(R[..., far]).max() == 0.0
    K1, G1 = green.green_symbol(shape, C, element=element)
    K2, G2 = green.green_symbol(shape, C, explicit_dft=True, element=element)
    assert np.abs(K1 - K2).max() <= 1e-14 * np.abs(K2).max()
    assert np.abs(G1 - G2).max() <= 1e-13 * np.abs(G2).max()


def alg1_block_tol(shape, base=1e-14):
    """Block-relative accuracy of Alg. 1 evaluated from FP64 impulse responses. On elements
    with sides h_a = 1/n_a, the couplings along the long side are O(h_max/h_min) while
    their sums over one offset (which the low frequencies across the short side see) are
    O(h_min/h_max): the FP64 rounding of the responses alone then limits any evaluation
    of step 2 to ~eps (h_max/h_min)^2 relative there. Square / cubic grids: ``base``."""
    ratio = max(shape) / min(shape)
    return max(base, 8 * np.finfo(np.float64).eps * ratio ** 2)


@pytest.mark.parametrize("shape", [(1024, 1024), (2048, 2048), (128, 128, 128), (2048, 16), (8, 8, 1024),
                                   (128, 8, 16), (1024, 64)])
def test_support_transform_is_accurate_at_low_frequencies(shape):
    """Block by block, the support-form symbol equals the plane-wave closed form (derived
    from the element, not from the impulse responses) to a few ulps at every frequency,
    the lowest included, on square / cubic grids, and to the responses' own FP64 limit
    on stretched grids; the full FFT of the responses does not (cancellation of O(1)
    entries down to O(theta^2), a relative error ~eps (n / 2 pi)^2)."""
    d = len(shape)
    C = 0.37 * fe.C_unit(d, 0.3)
    Ks, Gs = green.green_symbol(shape, C)
    Kc, Gc = green.closed_form_symbol(shape, C)
    blocks = lambda X: np.moveaxis(X.reshape(d, d, -1), 2, 0)[1:]  # noqa: E731
    for X, Y in ((Ks, Kc), (Gs, Gc)):
        bx, by = blocks(X), blocks(Y)
        err = np.linalg.norm(bx - by, axis=(1, 2)) / np.linalg.norm(by, axis=(1, 2))
        assert err.max() <= alg1_block_tol(shape)
    if len(set(shape)) > 1:
        return
    if d == 2:
        _, Gf = green.green_symbol(shape, C, transform="fft")
        bf, bc = blocks(Gf), blocks(Gc)
        err_fft = np.linalg.norm(bf - bc, axis=(1, 2)) / np.linalg.norm(bc, axis=(1, 2))
        assert err_fft.max() > 1e-12


@pytest.mark.parametrize("shape,element", [((4, 8), "q1"), ((8, 4, 4), "q1"), ((4, 4, 2), "q1"), ((8, 16), "p1")])
def test_matrix_free_operator_equals_assembled(shape, element):
    d = len(shape)
    rng = np.random.default_rng(3)
    E = rng.uniform(0.05, 1.0, shape)
    C = fe.C_unit(d, 0.3)
    x = random_field((d,) + shape, 9)
    K = assemble.assemble_K(shape, E, C, element)
    want = assemble.apply(K, x)
    got = assemble.apply_matrix_free(shape, E, C, x, element)
    assert np.abs(got - want).max() <= 1e-14 * np.abs(want).max()
    for a in range(d):  # a rigid translation gives exactly zero (corner differences vanish)
        t = np.zeros((d,) + shape)
        t[a] = 0.7
        assert np.array_equal(assemble.apply_matrix_free(shape, E, C, t, element), np.zeros((d,) + shape))


def test_matrix_free_operator_accuracy_on_smooth_fields():
    """On a smooth field at 512^2 the matrix-free product keeps ~eps/theta relative
    accuracy, against the same product evaluated in extended precision; the assembled
    product, whose rounded entries no longer sum to zero per row, loses ~eps/theta^2."""
    if np.finfo(np.longdouble).eps > 1e-18:
        pytest.skip("no extended precision type on this platform")
    shape = (512, 512)
    E = material.young_from_density(smooth_density(shape, 16, 8.0, 0), 1e-2, 1.0, 2.0)
    C = fe.C_unit(2, 0.3)
    idx = np.indices(shape)
    x = np.stack([np.cos(2 * np.pi * idx[0] / shape[0] + 0.3), 0.5 * np.sin(2 * np.pi * idx[1] / shape[1])])
    ref = assemble.apply_matrix_free(shape, E.astype(np.longdouble), C.astype(np.longdouble), x.astype(np.longdouble))
    scale = float(np.abs(ref).max())
    mf = assemble.apply_matrix_free(shape, E, C, x)
    asm = assemble.apply(assemble.assemble_K(shape, E, C), x)
    assert float(np.abs(mf - ref).max()) <= 1e-13 * scale
    assert float(np.abs(asm - ref).max()) > 1e-12 * scale


@pytest.mark.parametrize("shape,element", [((8, 16), "q1"), ((4, 8, 4), "q1"), ((8, 8), "p1")])
def test_matrix_free_diagonal_equals_assembled(shape, element):
    d = len(shape)
    E = np.random.default_rng(5).uniform(0.1, 1.0, shape)
    C = fe.C_unit(d, 0.3)
    want = jacobi.diag_assembled(assemble.assemble_K(shape, E, C, element), (d,) + shape)
    got = jacobi.diag_matrix_free(shape, E, C, element)
    assert np.abs(got - want).max() <= 1e-15 * np.abs(want).max()


@pytest.mark.parametrize("shape", [(16, 32), (8, 8, 8)])
def test_extended_setup_agrees_with_fp64_to_rounding(shape):
    """The extended-precision oracle derives C, the element matrix, the symbol and J^(1/2)
    from the FP64 inputs in numpy.longdouble: equal to the FP64 setup to a few FP64 ulps."""
    if np.finfo(np.longdouble).eps > 1e-18:
        pytest.skip("no extended precision type on this platform")
    d = len(shape)
    E = material.young_from_density(smooth_density(shape, 8, 3.0, 2), 1e-3, 1.0, 2.0)
    a = solve.setup(shape, E, 0.3)
    b = solve.setup(shape, E, 0.3, precision="extended")
    assert b.G_hat.dtype == np.longdouble and b.J_half.dtype == np.longdouble
    assert float(np.abs(b.C - a.C).max()) <= 4e-16 * np.abs(a.C).max()
    assert float(np.abs(b.G_hat - a.G_hat).max()) <= 1e-14 * np.abs(a.G_hat).max()
    assert float(np.abs(b.J_half - a.J_half).max()) <= 4e-16 * np.abs(a.J_half).max()
    A64 = fe.element_matrix(d, assemble.grid_spacing(shape), a.C)
    Ald = fe.element_matrix(d, assemble.grid_spacing(shape), b.C)
    assert Ald.dtype == np.longdouble and float(np.abs(Ald - A64).max()) <= 1e-15 * np.abs(A64).max()
