"""The C CPU baseline (oracle/cbase: matrix-free operator, textbook radix-2 FFT, OpenMP)
against the Python oracle on small grids (no GPU): the same PCG iterates after k
steps, and converged solutions equal to the dense brute-force solve."""

import numpy as np
import pytest

from oracle import assemble, cbase, dense, material, pcg, post, solve
from synthetic import mandel_unit_loads, smooth_density


@pytest.fixture(scope="module", autouse=True)
def built():
    cbase.build()


@pytest.mark.parametrize("shape", [(16, 16), (32, 64), (8, 8, 8), (4, 8, 16)])
@pytest.mark.parametrize("pc", ["green", "green_jacobi"])
def test_same_iterates_as_oracle(shape, pc):
    d = len(shape)
    E = material.young_from_density(smooth_density(shape, 8, 3.0, 1), 1e-3, 1.0, 2.0)
    prob = solve.setup(shape, E, 0.3)
    f = assemble.assemble_rhs(shape, E, prob.C, mandel_unit_loads(d)[-1])
    for k in (1, 5):
        u, it, _ = cbase.pcg(prob, f, 0.0, pc, max_iter=k)
        ref = pcg.pcg(prob.apply_K, prob.minv(pc), f, 0.0, k)
        assert it == k
        assert np.linalg.norm(u - ref.x) <= 1e-13 * np.linalg.norm(ref.x)


@pytest.mark.parametrize("shape", [(8, 8), (4, 4, 4)])
@pytest.mark.parametrize("pc", ["green", "green_jacobi"])
def test_converged_equals_dense(shape, pc):
    d = len(shape)
    E = material.young_from_density(smooth_density(shape, 6, 2.0, 5), 1e-3, 1.0, 2.0)
    prob = solve.setup(shape, E, 0.3)
    f = assemble.assemble_rhs(shape, E, prob.C, mandel_unit_loads(d)[0])
    u, it, conv = cbase.pcg(prob, f, 1e-13, pc)
    assert conv and it > 0
    want = dense.dense_solve(prob.K, f)
    assert np.linalg.norm(post.remove_mean(u) - want) <= 1e-10 * np.linalg.norm(want)


def test_zero_rhs_and_bad_arguments():
    shape = (8, 8)
    prob = solve.setup(shape, np.ones(shape), 0.3)
    u, it, conv = cbase.pcg(prob, np.zeros((2,) + shape), 1e-8, "green")
    assert it == 0 and conv and not u.any()
    with pytest.raises(ValueError):
        cbase.pcg(prob, np.zeros((2,) + shape), 1e-8, "jacobi")
