"""GPU parity of every step of the path against the FP64 oracle, through the C ABI.

Tolerances (FP64 everywhere; the GPU uses FMA and tree reductions, the oracle
sequential NumPy/SciPy):
  * single operator / preconditioner applications: 1e-13 relative (a few ulps of
    the O(10)-term sums, amplified by at most log2 N FFT stages);
  * PCG iterates at the same iteration count k <= 10: 1e-12 (before the CG
    recurrence starts amplifying rounding, see tests/test_oracle_pcg.py);
  * converged solves: displacement 1e-10, homogenised stiffness 1e-9 relative;
  * runs stopped at tolerance tau: iteration counts within one, displacement within
    10 tau of the oracle's (the oracle-vs-oracle floor is ~tau).
Grids are powers of two (the FFT's requirement here), so "ragged" coverage comes
from the smallest grids (4 per axis), non-square grids and tile-count edge cases.
"""

import numpy as np
import pytest

from oracle import assemble, dense, fe, green, material, pcg, post, solve as osolve
from synthetic import cosine_density, laminate_density, mandel_unit_loads, random_field, smooth_density

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _solver(shape, rho, contrast=1e4, exponent=2.0, nu=0.3, **kw):
    from paper_2508_02613_gb300.jfft import Solver
    return Solver(shape, rho, nu, kind="density", e_min=1.0 / contrast, e_max=1.0, exponent=exponent, **kw)


def _problem(shape, seed=0, contrast=1e4, exponent=2.0, modes=8, kmax=3.0):
    rho = smooth_density(shape, modes, kmax, seed)
    E = material.young_from_density(rho, 1.0 / contrast, 1.0, exponent)
    return rho, E


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


SHAPES = [(4, 4), (8, 16), (16, 8), (64, 512), (4, 4, 4), (8, 4, 16), (16, 16, 64)]


@pytest.mark.parametrize("shape", SHAPES + [(1024, 64), (64, 1024), (2048, 16), (16, 2048), (8, 128, 8),
                                            (128, 8, 16), (8, 8, 1024)])
def test_material_and_operator(shape):
    d = len(shape)
    rho, E = _problem(shape, 1)
    s = _solver(shape, rho)
    assert rel(s.get_material(), E) <= 4e-16
    K = assemble.assemble_K(shape, E, fe.C_unit(d, 0.3))
    x = random_field((2, d) + shape, 3)
    y = s.apply_K(x)
    want = np.stack([assemble.apply(K, x[i]) for i in range(2)])
    assert rel(y, want) <= 1e-13


@pytest.mark.parametrize("shape", [(1024, 1024), (2048, 2048), (128, 128, 128), (512, 64, 64)])
def test_operator_sampled_nodes_full_size(shape):
    """At full size, K x on 4096 sampled nodes (every grid edge and corner among them)
    against the oracle's node-by-node evaluation (no assembly)."""
    from oracle import pointwise
    d = len(shape)
    rho, E = _problem(shape, 2)
    s = _solver(shape, rho, max_loads=d)
    x = random_field((1, d) + shape, 8)
    y = s.apply_K(x)[0]
    rng = np.random.default_rng(len(shape))
    N = int(np.prod(shape))
    edge = [np.ravel_multi_index(tuple(c), shape) for c in np.ndindex(*([2] * d))]
    edge += [np.ravel_multi_index(tuple(m - 1 - c for m, c in zip(shape, cc)), shape) for cc in np.ndindex(*([2] * d))]
    nodes = np.unique(np.concatenate([rng.choice(N, 4096, replace=False), edge]))
    want = pointwise.apply_K_at(shape, E, fe.C_unit(d, 0.3), x[0], nodes)
    got = y.reshape(d, -1)[:, nodes].T
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("shape", SHAPES)
def test_rhs(shape):
    d = len(shape)
    rho, E = _problem(shape, 2)
    s = _solver(shape, rho)
    ds = d * (d + 1) // 2
    eps = np.vstack([np.eye(ds)[:2], np.linspace(-1, 1, ds)])
    f = s.rhs(eps)
    for i in range(3):
        assert rel(f[i], assemble.assemble_rhs(shape, E, fe.C_unit(d, 0.3), eps[i])) <= 1e-13


@pytest.mark.parametrize("shape", [(8, 8), (4, 16), (8, 4, 8), (16, 16, 64)])
def test_jacobi_diagonal_closed_form_and_alg2(shape):
    d = len(shape)
    rho, E = _problem(shape, 3)
    s = _solver(shape, rho)
    K = assemble.assemble_K(shape, E, fe.C_unit(d, 0.3))
    want = K.diagonal().reshape((d,) + shape)
    assert rel(s.get_diag("closed_form"), want) <= 1e-14
    assert rel(s.get_diag("combs"), want) <= 1e-14


def _half_spectrum(G_hat, shape):
    """Oracle symbol [d][d][k_0..k_{d-1}] -> the library's order [F][d][d] (k_0 fastest,
    last axis halved)."""
    d = len(shape)
    M = shape[-1] // 2
    g = np.moveaxis(G_hat.real, (0, 1), (-2, -1))[..., : M + 1, :, :]
    axes = tuple(range(d))[::-1] + (d, d + 1)
    return np.transpose(g, axes).reshape(-1, d, d)


# Every compile-time FFT line length (64..2048) on each transformed axis: the real axis
# (last), the axis-0 pass, and in 3D the middle axis; plus the small and ragged grids.
FFT_SHAPES = [(4, 4), (8, 16), (16, 8), (64, 512), (1024, 64), (64, 1024), (2048, 16), (16, 2048), (128, 256),
              (1024, 1024), (4, 4, 4), (8, 4, 16), (16, 16, 64), (8, 8, 1024), (8, 128, 8), (128, 8, 16),
              (256, 4, 8), (4, 2048 // 4, 8), (8, 8, 256)]

def alg1_tol(shape, base):
    """Symbol tables are compared block by block, ||G_gpu(k) - G_ref(k)|| <= tol ||G_ref(k)||
    at every stored frequency k != 0. Both sides evaluate step 2 of Alg. 1 over the
    impulse responses' support, every term to a few ulps: on square / cubic grids a few
    ulps per block remain (``base``). On elements with sides h_a = 1/n_a the long-side
    couplings of the responses are O(h_max/h_min) and their sums over one offset are
    O(h_min/h_max), so the FP64 rounding of the responses limits either side to
    ~eps (h_max/h_min)^2 relative at the low frequencies across the short side (the
    oracle's own table is that far from the closed form; tests/test_oracle_operator.py)."""
    ratio = max(shape) / min(shape)
    return max(base, 8 * np.finfo(np.float64).eps * ratio ** 2)


def _block_rel(a, b):
    """Largest block-relative difference over the frequencies (blocks [F, d, d]), k = 0 skipped
    (both sides pin it to zero; checked separately)."""
    na = np.linalg.norm(a[1:] - b[1:], axis=(1, 2))
    nb = np.linalg.norm(b[1:], axis=(1, 2))
    return float((na / nb).max())


@pytest.mark.parametrize("shape", [(8, 8), (16, 4), (4, 8, 16), (8, 8, 8), (1024, 1024), (2048, 16), (16, 2048),
                                   (8, 8, 1024), (128, 8, 16)])
def test_green_symbol_alg1(shape):
    d = len(shape)
    rho, E = _problem(shape, 4)
    s = _solver(shape, rho)
    _, G_hat = green.green_symbol(shape, E.mean() * fe.C_unit(d, 0.3))
    got = s.get_green()
    want = _half_spectrum(G_hat, shape)
    assert np.abs(got[0]).max() == 0.0
    assert _block_rel(got, want) <= alg1_tol(shape, 1e-14)


@pytest.mark.parametrize("shape", [(1024, 1024), (128, 128, 128), (2048, 16), (8, 8, 1024), (64, 512)])
def test_green_symbol_against_closed_form(shape):
    """The table against the plane-wave closed form of the uniform Q1 operator, derived from
    the element and not from impulse responses."""
    d = len(shape)
    rho, E = _problem(shape, 4)
    s = _solver(shape, rho)
    _, G_cf = green.closed_form_symbol(shape, E.mean() * fe.C_unit(d, 0.3))
    assert _block_rel(s.get_green(), _half_spectrum(G_cf, shape)) <= alg1_tol(shape, 1e-14)


@pytest.mark.parametrize("shape", FFT_SHAPES)
@pytest.mark.parametrize("pc", ["green", "green_jacobi", "jacobi"])
def test_preconditioners(shape, pc):
    """Element by element against the oracle (numpy FFT, support-form symbol): the two
    transforms round differently, ~eps log2 N relative to the output's scale; on stretched
    grids the symbols' own limit (alg1_tol) dominates."""
    d = len(shape)
    rho, E = _problem(shape, 5)
    s = _solver(shape, rho)
    prob = osolve.setup(shape, E, 0.3)
    r = random_field((2, d) + shape, 6)
    z = s.apply_precond(pc, r)
    minv = prob.minv(pc)
    want = np.stack([minv(r[i]) for i in range(2)])
    assert rel(z, want) <= (alg1_tol(shape, 1e-13) if pc != "jacobi" else 1e-15)


@pytest.mark.parametrize("shape", [(16, 16), (8, 8, 8)])
@pytest.mark.parametrize("pc", ["green", "green_jacobi"])
def test_homogeneous_one_iteration(shape, pc):
    from paper_2508_02613_gb300.jfft import Solver
    d = len(shape)
    C_ref = 0.6 * fe.C_unit(d, 0.3)
    s = Solver(shape, np.full(shape, 3.7), 0.3, C_ref=C_ref)
    f = random_field((d,) + shape, 7, zero_mean=True)[None]  # zero mean per component
    out = s.solve_rhs(f, 1e-12, pc)
    assert int(out["iters"][0]) == 1
    prob = osolve.setup(shape, np.full(shape, 3.7), 0.3, C_ref=C_ref)
    want = dense.dense_solve(prob.K, f[0]) if np.prod(shape) <= 512 else None
    if want is not None:
        assert np.linalg.norm(post.remove_mean(out["u"][0]) - want) <= 1e-11 * np.linalg.norm(want)


@pytest.mark.parametrize("shape", [(32, 32), (8, 8, 8)])
@pytest.mark.parametrize("pc", ["green", "green_jacobi"])
def test_same_k_iterates(shape, pc):
    d = len(shape)
    rho, E = _problem(shape, 8, contrast=1e4)
    s = _solver(shape, rho)
    prob = osolve.setup(shape, E, 0.3)
    f = assemble.assemble_rhs(shape, E, prob.C, mandel_unit_loads(d)[0])
    for k in (1, 3, 10):
        s.set_max_iter(k)
        out = s.solve_rhs(f[None], 0.0, pc)
        assert int(out["iters"][0]) == k
        ref = pcg.pcg(prob.apply_K, prob.minv(pc), f, 0.0, k)
        assert np.linalg.norm(out["u"][0] - ref.x) <= 1e-12 * np.linalg.norm(ref.x)


@pytest.mark.parametrize("shape", [(8, 8), (4, 4, 4)])
@pytest.mark.parametrize("pc", ["green", "green_jacobi", "jacobi", "none"])
def test_converged_vs_dense(shape, pc):
    d = len(shape)
    rho, E = _problem(shape, 9, contrast=1e3)
    s = _solver(shape, rho, contrast=1e3)
    prob = osolve.setup(shape, E, 0.3)
    eps = mandel_unit_loads(d)[-1:]
    out = s.solve(eps, 1e-13, pc)
    f = assemble.assemble_rhs(shape, E, prob.C, eps[0])
    want = dense.dense_solve(prob.K, f)
    assert np.linalg.norm(out["u"][0] - want) <= 1e-10 * np.linalg.norm(want)
    C_want = post.homogenised_stress(shape, E, prob.C, eps[0], want)
    assert rel(out["C_hom"][:, 0], C_want) <= 1e-9
    assert out["rel_res"][0] <= 1e-12


def creep_window(prob, eps, tol, pc):
    """Iteration counts at which a PCG run to `tol` may stop, from the oracle: its counts
    under two summation orders, and every iteration at which either order's relative
    residual lies within a factor `band` of the tolerance, widened by one on each side.
    `band` is how far the two orders' residual trajectories drift apart over the last
    ten iterations before they stop (twice the largest relative gap, between 1.05 and
    1.5): where the residual creeps along the threshold, rounding of that size decides
    the stopping iteration."""
    f = assemble.assemble_rhs(prob.n, prob.E, prob.C, eps, prob.element)
    hs = []
    for order in ("blas", "sequential"):
        # run past the threshold and read the stopping count off the history
        res = pcg.pcg(prob.apply_K, prob.minv(pc), f, tol / 1.5, 100000, "rel", order)
        hs.append(np.asarray(res.res_norms) / res.res_norms[0])
    counts = [int(np.argmax(h <= tol)) for h in hs]
    n = min(counts)
    gap = max(abs(hs[0][k] / hs[1][k] - 1.0) for k in range(max(0, n - 10), n + 1))
    band = min(1.5, max(1.05, 1.0 + 2.0 * gap))
    ns = list(counts)
    for h in hs:
        ns += [k for k in range(len(h)) if tol / band <= h[k] <= tol * band]
    return min(ns) - 1, max(ns) + 1


@pytest.mark.parametrize("pc", ["green", "green_jacobi"])
def test_small_workload_32x32(pc):
    """The 32 x 32 workload: 16 Fourier modes |k| <= 4, E = 1e-4 + (1 - 1e-4) rho^2,
    nu = 0.3, eps_xx = 1, tolerance 1e-6, C_ref = mean material."""
    shape = (32, 32)
    rho = smooth_density(shape, 16, 4.0, 0)
    E = material.young_from_density(rho, 1e-4, 1.0, 2.0)
    s = _solver(shape, rho)
    eps = mandel_unit_loads(2)[:1]
    out = s.solve(eps, 1e-6, pc)
    prob = osolve.setup(shape, E, 0.3)
    ref = osolve.solve(prob, eps, 1e-6, pc)
    lo, hi = creep_window(prob, eps[0], 1e-6, pc)
    assert lo <= int(out["iters"][0]) <= hi, (int(out["iters"][0]), lo, hi)
    nrm = np.linalg.norm(ref.u)
    assert np.linalg.norm(out["u"] - ref.u) <= 10 * 1e-6 * nrm
    assert rel(out["C_hom"], ref.C_hom) <= 1e-6
    assert out["rel_res"][0] <= 2e-6
    # converged parity on the same workload
    tight = s.solve(eps, 1e-12, pc)
    ref_t = osolve.solve(prob, eps, 1e-12, pc)
    assert np.linalg.norm(tight["u"] - ref_t.u) <= 1e-10 * np.linalg.norm(ref_t.u)
    assert rel(tight["C_hom"], ref_t.C_hom) <= 1e-9
    st = tight["stress"][0]
    assert rel(st, ref_t.stress[0]) <= 1e-9


@pytest.mark.parametrize("contrast,pc", [(1e2, "green_jacobi"), (1e4, "green_jacobi"), (1e2, "green")])
def test_iteration_counts_256_benchmark_density(contrast, pc):
    """The benchmark's density recipe (16 modes, |k| <= 8, seed 0) at 256 x 256, three
    Mandel loads batched, relative tolerance 1e-8, true residual below the tolerance.
    Iteration counts: within the oracle's own spread over two summation orders, widened
    on each side by that spread (at least one). Green-Jacobi counts at this size move by
    up to three between two FP64 summation orders of the same oracle."""
    shape = (256, 256)
    rho = smooth_density(shape, 16, 8.0, 0)
    E = material.young_from_density(rho, 1.0 / contrast, 1.0, 2.0)
    s = _solver(shape, rho, contrast=contrast)
    out = s.solve(mandel_unit_loads(2), 1e-8, pc, want_stress=False)
    prob = osolve.setup(shape, E, 0.3)
    for g in range(3):
        f = assemble.assemble_rhs(shape, E, prob.C, np.eye(3)[g])
        a = pcg.pcg(prob.apply_K, prob.minv(pc), f, 1e-8, 100000).iters
        b = pcg.pcg(prob.apply_K, prob.minv(pc), f, 1e-8, 100000, "rel", "sequential").iters
        lo, hi = min(a, b), max(a, b)
        w = max(1, hi - lo)
        assert lo - w <= int(out["iters"][g]) <= hi + w, (g, int(out["iters"][g]), a, b)
        assert out["rel_res"][g] <= 1e-8 * 1.01


@pytest.mark.parametrize("filt", [0, 4, 16])
@pytest.mark.parametrize("pc", ["green", "green_jacobi"])
def test_filtered_inclusion_counts(filt, pc):
    """Sec. 1 motivating example at 128^2 (circular inclusion, contrast 1e4, filtered
    `filt` times): iteration counts in the oracle's creep window (creep_window), true
    residual below the tolerance."""
    from synthetic import circular_inclusion, gaussian_filter
    from paper_2508_02613_gb300.jfft import Solver
    shape = (128, 128)
    rho = gaussian_filter(circular_inclusion(shape), filt)
    s = Solver(shape, rho, 0.3)
    out = s.solve(mandel_unit_loads(2)[:1], 1e-6, pc, want_stress=False)
    prob = osolve.setup(shape, rho, 0.3)
    lo, hi = creep_window(prob, mandel_unit_loads(2)[0], 1e-6, pc)
    assert lo <= int(out["iters"][0]) <= hi, (int(out["iters"][0]), lo, hi)
    assert out["rel_res"][0] <= 1e-6 * 1.01


@pytest.mark.parametrize("p,n", [((4, 4), (16, 16)), ((8, 2), (32, 16)), ((4, 4, 2), (8, 16, 8))])
def test_coarse_geometry_upsampling(p, n):
    """jfft_set_material_coarse (geometry G_p on T_n) equals jfft_set_material with the
    oracle's upsampled field, bit for bit."""
    from oracle import material as omat
    from paper_2508_02613_gb300.jfft import Solver
    rng = np.random.default_rng(sum(p))
    coarse = rng.uniform(0.0, 1.0, p)
    fine = omat.upsample(coarse, n)
    a = Solver(n, np.ones(n), 0.3, kind="density", e_min=1e-3, e_max=1.0, exponent=2.0)
    a.set_material_coarse(coarse)
    b = Solver(n, fine, 0.3, kind="density", e_min=1e-3, e_max=1.0, exponent=2.0)
    assert np.array_equal(a.get_material(), b.get_material())
    d = len(n)
    oa = a.solve(mandel_unit_loads(d), 1e-10, "green_jacobi")
    ob = b.solve(mandel_unit_loads(d), 1e-10, "green_jacobi")
    assert np.array_equal(oa["u"], ob["u"]) and np.array_equal(oa["iters"], ob["iters"])
    with pytest.raises(Exception):
        a.set_material_coarse(rng.uniform(0.0, 1.0, tuple(2 * k for k in n)))


@pytest.mark.parametrize("shape,normal,tangent", [((32, 8), [0, 2], [1]), ((16, 4, 4), [0, 4, 5], [1, 2, 3])])
def test_laminate_closed_form(shape, normal, tangent):
    from tests.test_oracle_homogenisation import _laminate_C_hom
    from paper_2508_02613_gb300.jfft import Solver
    d = len(shape)
    rho = laminate_density(shape, 1e2)
    s = Solver(shape, rho, 0.3)
    out = s.solve(mandel_unit_loads(d), 1e-13, "green_jacobi")
    layers = rho.reshape(shape[0], -1)[:, 0]
    want = _laminate_C_hom([e * fe.C_unit(d, 0.3) for e in layers], normal, tangent)
    assert rel(out["C_hom"], want) <= 1e-10


def test_void_replacement_value_invariance():
    from paper_2508_02613_gb300.jfft import Solver
    rho = np.kron(cosine_density((4, 4), float("inf")), np.ones((4, 4)))
    its = []
    for rep in (1e-15, 1.0, 1e15):
        s = Solver(rho.shape, rho, 0.3, void_value=rep, C_ref=fe.C_unit(2, 0.3) * rho.mean())
        out = s.solve(np.array([[1.0, 1.0, 0.0]]), 1e-8, "green_jacobi")
        assert out["status"] == 0
        its.append(int(out["iters"][0]))
    assert its[0] == its[1] == its[2]


def test_batched_loads_equal_single_loads():
    shape = (64, 64)
    rho, _ = _problem(shape, 10)
    s = _solver(shape, rho)
    eps = mandel_unit_loads(2)
    batch = s.solve(eps, 1e-8, "green_jacobi")
    for g in range(3):
        one = s.solve(eps[g:g + 1], 1e-8, "green_jacobi")
        assert int(one["iters"][0]) == int(batch["iters"][g])
        assert np.array_equal(one["u"][0], batch["u"][g])
        assert np.array_equal(one["C_hom"][:, 0], batch["C_hom"][:, g])


def test_deterministic_and_counts_launches():
    shape = (64, 32)
    rho, _ = _problem(shape, 11)
    s = _solver(shape, rho)
    a = s.solve(mandel_unit_loads(2), 1e-8, "green_jacobi")
    n0 = s.launch_count
    b = s.solve(mandel_unit_loads(2), 1e-8, "green_jacobi")
    assert s.launch_count > n0
    assert np.array_equal(a["u"], b["u"]) and np.array_equal(a["C_hom"], b["C_hom"])
    s.set_profiling(True)
    s.solve(mandel_unit_loads(2)[:1], 1e-8, "green_jacobi")
    prof = s.profile()
    assert prof["apply_K"][0] > 0 and prof["fft_rows_real_fwd_xr"][0] > 0 and prof["fft_lines"][1] > 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_matches_direct_launches(precision):
    """The PCG chunk replayed as a CUDA graph gives bit-identical results to the same
    kernels launched one by one, on the solver's own stream and on a caller stream."""
    torch = pytest.importorskip("torch")
    shape = (64, 32)
    rho, _ = _problem(shape, 13)
    outs = []
    for graphs, stream in ((False, None), (True, None), (True, "torch")):
        st = torch.cuda.Stream() if stream else None
        s = _solver(shape, rho, graphs=graphs, precision=precision,
                    stream=st.cuda_stream if st is not None else None)
        out = s.solve(mandel_unit_loads(2), 1e-8, "green_jacobi")
        assert (s.graph_replays > 0) == graphs
        outs.append(out)
    for o in outs[1:]:
        assert np.array_equal(o["iters"], outs[0]["iters"])
        assert np.array_equal(o["u"], outs[0]["u"]) and np.array_equal(o["C_hom"], outs[0]["C_hom"])


@pytest.mark.parametrize("shape,precision", [((256, 128), "fp64"), ((256, 128), "mixed"), ((32, 32, 64), "mixed")])
def test_autotuned_launch_shapes(shape, precision):
    """options.autotune picks shapes from the candidate sets; the tuned solve meets the
    tolerance (true residual) and agrees with the default-shape solve within 10 tol (the
    shapes change only the rounding of the partial-sum reductions, which can move the
    iteration count); set_tuning reproduces the tuned run bit for bit."""
    d = len(shape)
    rho, _ = _problem(shape, 15)
    tuned = _solver(shape, rho, precision=precision, autotune=True)
    t = tuned.tuning
    assert t[0] in (0, 8, 16, 32, 64) and t[1] in (0, 4, 8, 16) and t[2] in (0, 1, 2, 4) and t[3] in (0, 1, 2, 4)
    a = tuned.solve(mandel_unit_loads(d), 1e-8, "green_jacobi")
    base = _solver(shape, rho, precision=precision).solve(mandel_unit_loads(d), 1e-8, "green_jacobi")
    assert a["rel_res"].max() <= 1e-8 * 1.01
    assert np.linalg.norm(a["u"] - base["u"]) <= 10 * 1e-8 * np.linalg.norm(base["u"])
    again = _solver(shape, rho, precision=precision)
    again.set_tuning(t)
    b = again.solve(mandel_unit_loads(d), 1e-8, "green_jacobi")
    assert np.array_equal(a["u"], b["u"]) and np.array_equal(a["iters"], b["iters"])


def test_device_io_matches_host_io():
    torch = pytest.importorskip("torch")
    shape = (32, 64)
    rho, _ = _problem(shape, 12)
    s = _solver(shape, rho)
    eps = mandel_unit_loads(2)
    host = s.solve(eps, 1e-8, "green")
    s.set_io_memory("device")
    dev = s.solve(torch.tensor(eps, device="cuda"), 1e-8, "green")
    assert np.array_equal(host["u"], dev["u"].cpu().numpy())
    assert np.array_equal(host["C_hom"], dev["C_hom"].cpu().numpy())


def test_argument_errors_are_reported():
    from paper_2508_02613_gb300.jfft import JfftError, Solver
    with pytest.raises(JfftError) as ei:
        Solver((6, 8), np.ones((6, 8)), 0.3)
    assert ei.value.status == 7 and "power of two" in str(ei.value)
    bad = np.ones((8, 8))
    bad[0, 0] = -1.0
    with pytest.raises(JfftError) as ei:
        Solver((8, 8), bad, 0.3)
    assert ei.value.status == 1
    s = Solver((8, 8), np.ones((8, 8)), 0.3, max_loads=3)
    with pytest.raises(JfftError):
        s.solve(np.eye(3).repeat(2, axis=0), 1e-6)
