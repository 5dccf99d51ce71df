"""Pins for the oracle's Q1 element and material (no GPU)."""

import json
import math
import os

import numpy as np
import pytest

from oracle import fe

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


@pytest.mark.parametrize("nu", [0.0, 0.3, 0.45, -0.5])
def test_q1_plane_stress_matches_textbook_element(nu):
    """Square Q1 element, plane stress: every row holds the textbook k_1..k_8 once."""
    g = _load("q1_plane_stress_element.json")
    E = 2.5
    lam_ps = E * nu / (1 - nu * nu)  # plane-stress first Lame constant
    mu = E / (2 * (1 + nu))
    A = fe.element_matrix(2, (1.0, 1.0), fe.isotropic_C(2, lam_ps, mu))
    k = np.array([a + b * nu for a, b in g["k"]]) * E / (1 - nu * nu)
    assert np.allclose(np.diag(A), k[0], rtol=0, atol=1e-13)
    for row in A:
        assert np.allclose(np.sort(row), np.sort(k), rtol=0, atol=1e-13)


def test_element_size_scaling():
    """K_e scales as h^(d-2): invariant in 2D, linear in h in 3D."""
    C = fe.C_unit(2, 0.3)
    assert np.allclose(fe.element_matrix(2, (0.25, 0.25), C), fe.element_matrix(2, (1.0, 1.0), C), atol=1e-14)
    C3 = fe.C_unit(3, 0.3)
    assert np.allclose(fe.element_matrix(3, (0.5,) * 3, C3), 0.5 * fe.element_matrix(3, (1.0,) * 3, C3), atol=1e-14)


@pytest.mark.parametrize("d", [2, 3])
def test_element_rigid_modes_and_rank(d):
    """Rigid translations and infinitesimal rotations have zero energy; nothing else does."""
    h = (0.5, 0.25, 0.125)[:d]
    A = fe.element_matrix(d, h, fe.C_unit(d, 0.3))
    assert np.allclose(A, A.T, atol=1e-15)
    ev = np.linalg.eigvalsh(A)
    n_rigid = d + d * (d - 1) // 2
    scale = ev.max()
    assert np.all(ev > -1e-12 * scale)
    assert np.sum(np.abs(ev) < 1e-12 * scale) == n_rigid


@pytest.mark.parametrize("d", [2, 3])
def test_B_reproduces_affine_fields(d):
    """Q1 interpolates affine displacements exactly: B_q u gives the Mandel strain sym(G)."""
    rng = np.random.default_rng(3)
    G = rng.standard_normal((d, d))
    h = np.array((0.5, 0.25, 0.2)[:d])
    cs = fe.corners(d)
    u = np.zeros(d * 2 ** d)
    for ci, c in enumerate(cs):
        x = np.array(c) * h
        disp = G @ x
        for a in range(d):
            u[a * 2 ** d + ci] = disp[a]
    eps_t = 0.5 * (G + G.T)
    want = np.array([eps_t[i, j] * (1 if i == j else math.sqrt(2)) for i, j in fe.mandel_pairs(d)])
    pts, _ = fe.gauss_points(d)
    for xi in pts:
        assert np.allclose(fe.mandel_B(d, xi, h) @ u, want, atol=1e-13)


def test_paper_material_constants():
    """Sec. 4: lambda0 = 2/3, mu0 = 1/2 give bulk modulus 1; Sec. 4.3: (K, mu) = (0.025, 0.15) <-> (E, nu) = (0.15, -0.5)."""
    g = _load("paper_constants.json")
    ref = g["reference_material"]
    C = fe.isotropic_C(3, ref["lambda"], ref["mu"])
    # bulk modulus: sigma_m = K tr(eps) for eps = I/3 (tr = 1)
    eps = np.array([1, 1, 1, 0, 0, 0]) / 3.0
    sig = C @ eps
    assert np.allclose(sig[:3], ref["bulk"], atol=1e-15) and np.allclose(sig[3:], 0)
    t = g["target_material"]
    lam, mu = fe.lame_from_young(t["young"], t["poisson"])
    assert math.isclose(mu, t["mu"], rel_tol=1e-14)
    assert math.isclose(lam + 2 * mu / 3, t["bulk"], rel_tol=1e-12)


def test_mandel_shear_convention():
    """Sec. 4.5: tensor shear strain 0.05 appears as Mandel component 6 = 0.05 sqrt(2), and
    the Mandel inner product equals the tensor double contraction."""
    g = _load("paper_constants.json")["mandel_shear"]
    pairs = fe.mandel_pairs(3)
    assert pairs[5] == (0, 1)
    eps_t = np.zeros((3, 3))
    eps_t[0, 1] = eps_t[1, 0] = g["tensor_eps_12"]
    m = np.array([eps_t[i, j] * (1 if i == j else math.sqrt(2)) for i, j in pairs])
    assert math.isclose(m[5], g["mandel_component_6"], rel_tol=1e-15)
    assert math.isclose(m @ m, np.sum(eps_t * eps_t), rel_tol=1e-15)


# ---- P1 triangles (each voxel split along the (0,0)-(1,1) diagonal) ----------------

def test_p1_patch_test_and_energy():
    """Both triangles reproduce the exact constant strain of any affine displacement, and
    the voxel energy equals vol * eps : C : eps (patch test)."""
    h = (0.25, 0.125)
    rng = np.random.default_rng(3)
    Gm = rng.standard_normal((2, 2))
    xs = [np.array([o[0] * h[0], o[1] * h[1]]) for o in fe.corners(2)]
    ue = np.concatenate([[(Gm @ x)[a] for x in xs] for a in range(2)])
    eps_t = 0.5 * (Gm + Gm.T)
    want = np.array([eps_t[0, 0], eps_t[1, 1], np.sqrt(2.0) * eps_t[0, 1]])
    Bs, ws = fe.element_points(2, h, "p1")
    assert len(Bs) == 2 and np.isclose(sum(ws), h[0] * h[1])
    for B in Bs:
        assert np.allclose(B @ ue, want, atol=1e-13)
    C = fe.C_unit(2, 0.3)
    A = fe.element_matrix(2, h, C, "p1")
    assert np.isclose(ue @ A @ ue, h[0] * h[1] * want @ C @ want, rtol=1e-13)


def test_p1_voxel_matrix_rigid_modes_and_rank():
    A = fe.element_matrix(2, (0.5, 0.5), fe.C_unit(2, 0.25), "p1")
    assert np.abs(A - A.T).max() < 1e-13
    w = np.linalg.eigvalsh(A)
    assert w.min() > -1e-12 * w.max()
    assert np.sum(np.abs(w) < 1e-10 * w.max()) == 3     # two translations and a rotation


@pytest.mark.parametrize("shape", [(4, 4), (8, 4)])
def test_p1_global_operator_kernel(shape):
    """The periodic P1 stiffness is symmetric PSD with exactly the d translations as kernel."""
    from oracle import assemble
    E = np.random.default_rng(1).uniform(0.5, 2.0, shape)
    K = assemble.assemble_K(shape, E, fe.C_unit(2, 0.3), "p1").toarray()
    assert np.abs(K - K.T).max() < 1e-12
    w = np.linalg.eigvalsh(K)
    assert w.min() > -1e-10 * w.max()
    assert np.sum(np.abs(w) < 1e-9 * w.max()) == 2


@pytest.mark.parametrize("pc", ["green", "green_jacobi"])
def test_p1_laminate_and_homogeneous_cell(pc):
    """Layers normal to e_1: the exact solution is piecewise linear in x_1 with kinks on
    grid lines, so P1 reproduces the lamination formula; a uniform cell under a random
    zero-mean load converges in one Green iteration."""
    from oracle import assemble, pcg, solve
    from synthetic import laminate_density, mandel_unit_loads, random_field
    from tests.test_oracle_homogenisation import _laminate_C_hom
    shape = (16, 8)
    rho = laminate_density(shape, 1e2)
    prob = solve.setup(shape, rho, 0.3, element="p1")
    out = solve.solve(prob, mandel_unit_loads(2), 1e-13, pc)
    layers = rho.reshape(shape[0], -1)[:, 0]
    want = _laminate_C_hom([e * fe.C_unit(2, 0.3) for e in layers], [0, 2], [1])
    assert np.abs(out.C_hom - want).max() <= 1e-11 * np.abs(want).max()
    uni = solve.setup((8, 8), np.full((8, 8), 2.5), 0.3, element="p1")
    f = random_field((2, 8, 8), 4, zero_mean=True)
    assert pcg.pcg(uni.apply_K, uni.minv(pc), f, 1e-12, 50).iters == 1
