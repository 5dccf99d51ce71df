"""Pins for the oracle's post-processing and its node-by-node operator (no GPU).

* ``post.element_stress`` (paper Eq. aim_fun, Sec. 5.3): against a brute force that
  uses no B matrix and no Gauss point. For a multilinear interpolant the derivative
  along axis b is constant along b and multilinear in the other coordinates, and the
  2-point Gauss rule integrates that exactly, so the Gauss-point average of the strain
  equals the element mean of the gradient: the mean over the element's edges parallel
  to axis b of the nodal difference quotient (u(end) - u(start)) / h_b. The element
  stress is then E_e C_unit (eps_bar + that mean strain).
* The same function against a closed form: in a laminate normal to e_1 the FE solution
  is exact, and the normal stress components (sigma_11, sigma_12 / sigma_11, sigma_13,
  sigma_12) are the same in every element and equal the lamination formula's normal
  rows times eps_bar.
* ``post.homogenised_stress`` against the energy identity: at the solution of
  K u = f, the cell-averaged stress power of the total strain equals
  eps_bar^T C_Voigt eps_bar - f . u (expand (eps_bar + B u)^T E C (eps_bar + B u) and
  use u^T K u = f . u), and Hill-Mandel makes it eps_bar . C_hom eps_bar.
* ``pointwise.apply_K_at`` against the assembled sparse K on every node of small grids.
"""

import math

import numpy as np
import pytest

from oracle import assemble, fe, pointwise, post, solve
from synthetic import laminate_density, mandel_unit_loads, random_field, smooth_density
from tests.test_oracle_homogenisation import _laminate_C_hom


def _mean_strain_brute_force(u: np.ndarray) -> np.ndarray:
    """Element-mean Mandel strain [d*, *n] of the multilinear interpolant of nodal u [d, *n]
    on the periodic unit cell, from nodal difference quotients only."""
    d = u.shape[0]
    n = u.shape[1:]
    grad = np.zeros((d, d) + n)  # grad[a, b] = mean d u_a / d x_b over element e
    for a in range(d):
        for b in range(d):
            # difference along b at every node, then averaged over the 2^(d-1) edges of
            # the element parallel to b (shifts by 0 / 1 along every other axis)
            diff = (np.roll(u[a], -1, axis=b) - u[a]) * n[b]
            acc = np.zeros(n)
            others = [c for c in range(d) if c != b]
            for shift in np.ndindex(*([2] * len(others))):
                t = diff
                for c, s in zip(others, shift):
                    if s:
                        t = np.roll(t, -1, axis=c)
                acc += t
            grad[a, b] = acc / 2 ** len(others)
    out = []
    for i, j in fe.mandel_pairs(d):
        out.append(grad[i, i] if i == j else (grad[i, j] + grad[j, i]) / math.sqrt(2.0))
    return np.stack(out)


@pytest.mark.parametrize("shape", [(4, 8), (8, 4), (4, 4, 8), (2, 4, 4)])
def test_element_stress_equals_brute_force(shape):
    d = len(shape)
    rng = np.random.default_rng(len(shape) * 100 + shape[0])
    E = rng.uniform(0.1, 2.0, shape)
    u = random_field((d,) + shape, 31)
    C = fe.C_unit(d, 0.27)
    eps = np.linspace(-0.7, 1.3, d * (d + 1) // 2)
    got = post.element_stress(shape, E, C, eps, u)
    strain = eps.reshape((-1,) + (1,) * d) + _mean_strain_brute_force(u)
    want = E[None] * np.einsum("st,t...->s...", C, strain)
    assert got.shape == want.shape
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("shape", [(8, 8), (4, 4, 4)])
def test_element_stress_homogeneous_no_fluctuation(shape):
    """E = c and u = 0: every element carries c C_unit eps_bar."""
    d = len(shape)
    C = fe.C_unit(d, 0.3)
    eps = np.arange(1.0, d * (d + 1) // 2 + 1.0)
    got = post.element_stress(shape, np.full(shape, 2.5), C, eps, np.zeros((d,) + shape))
    want = 2.5 * C @ eps
    assert np.abs(got - want.reshape((-1,) + (1,) * d)).max() <= 1e-15 * np.abs(want).max()


@pytest.mark.parametrize("shape,normal,tangent", [((16, 8), [0, 2], [1]), ((8, 4, 4), [0, 4, 5], [1, 2, 3])])
def test_laminate_normal_stress_is_constant_and_closed_form(shape, normal, tangent):
    d = len(shape)
    rho = laminate_density(shape, 1e2)
    Cu = fe.C_unit(d, 0.3)
    prob = solve.setup(shape, rho, 0.3)
    loads = mandel_unit_loads(d)
    out = solve.solve(prob, loads, 1e-13, "green_jacobi")
    layers = rho.reshape(shape[0], -1)[:, 0]
    C_star = _laminate_C_hom([e * Cu for e in layers], normal, tangent)
    for g in range(len(loads)):
        sig = out.stress[g].reshape(len(loads), -1)
        for s in normal:
            want = C_star[s] @ loads[g]
            scale = max(np.abs(C_star).max(), 1e-300)
            assert np.abs(sig[s] - want).max() <= 1e-10 * scale, (g, s)


@pytest.mark.parametrize("shape", [(16, 16), (6, 6, 6)])
def test_energy_identity(shape):
    d = len(shape)
    E = smooth_density(shape, 8, 3.0, 9) * (1 - 1e-3) + 1e-3
    prob = solve.setup(shape, E, 0.3)
    ds = d * (d + 1) // 2
    loads = np.vstack([mandel_unit_loads(d), np.linspace(-1.0, 0.8, ds)])
    out = solve.solve(prob, loads, 1e-13, "green_jacobi")
    C_voigt = E.mean() * prob.C
    for g in range(len(loads)):
        f = assemble.assemble_rhs(shape, E, prob.C, loads[g])
        energy = loads[g] @ C_voigt @ loads[g] - float(np.sum(f * out.u[g]))
        assert abs(loads[g] @ out.C_hom[:, g] - energy) <= 1e-10 * abs(energy)


@pytest.mark.parametrize("shape", [(4, 8), (8, 4), (4, 4, 8), (4, 2, 4)])
def test_pointwise_operator_equals_assembled(shape):
    d = len(shape)
    rng = np.random.default_rng(7 + len(shape))
    E = rng.uniform(0.01, 1.0, shape)
    C = fe.C_unit(d, 0.3)
    x = random_field((d,) + shape, 44)
    K = assemble.assemble_K(shape, E, C)
    want = assemble.apply(K, x).reshape(d, -1).T
    nodes = np.arange(int(np.prod(shape)))
    got = pointwise.apply_K_at(shape, E, C, x, nodes)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
    sub = rng.choice(nodes, 5, replace=False)
    assert np.array_equal(pointwise.apply_K_at(shape, E, C, x, sub), got[sub])
