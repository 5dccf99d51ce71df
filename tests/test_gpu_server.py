"""Request server with continuous batching (jfft_server_*): requests of different grids,
materials, load cases, preconditioners and precisions run concurrently on their own
streams; each result must equal the same solve run alone (same kernels, deterministic),
admission must respect the memory budget, and idle solvers are reused or evicted."""

import numpy as np
import pytest

from synthetic import mandel_unit_loads, smooth_density

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _requests():
    rng = np.random.default_rng(5)
    shapes = [(32, 32), (64, 128), (128, 128), (256, 256), (16, 16, 16), (32, 32, 16), (64, 64), (128, 64)]
    out = []
    for i in range(12):
        shape = shapes[i % len(shapes)]
        d = len(shape)
        ds = d * (d + 1) // 2
        rho = smooth_density(shape, 16 if d == 2 else 24, 6.0, 100 + i)
        nl = int(rng.integers(1, ds + 1))
        eps = mandel_unit_loads(d)[rng.permutation(ds)[:nl]]
        out.append(dict(shape=shape, field=rho, nu=float(rng.uniform(0.2, 0.4)),
                        e_min=float(10.0 ** -rng.uniform(2, 5)), eps=eps,
                        precond=["green_jacobi", "green"][i % 2] if d == 2 else "green_jacobi",
                        precision=["mixed", "fp64", "mixed"][i % 3]))
    return out


def _alone(r):
    from paper_2508_02613_gb300.jfft import Solver
    d = len(r["shape"])
    s = Solver(r["shape"], r["field"], r["nu"], kind="density", e_min=r["e_min"], e_max=1.0, exponent=2.0,
               precision=r["precision"], max_loads=d * (d + 1) // 2)
    return s.solve(r["eps"], 1e-8, r["precond"], want_stress=False)


def test_results_equal_alone_and_in_the_mix():
    from paper_2508_02613_gb300.jfft import Server
    reqs = _requests()
    srv = Server(max_active=4)
    ids = [srv.submit(r["shape"], r["field"], r["nu"], r["eps"], 1e-8, r["precond"], r["precision"],
                      kind="density", e_min=r["e_min"], e_max=1.0, exponent=2.0, want_u=True) for r in reqs]
    outs = [srv.wait(i) for i in ids]
    st = srv.stats()
    assert st["submitted"] == st["finished"] == len(reqs)
    assert st["peak_used"] <= st["budget"]
    for r, o in zip(reqs, outs):
        assert o["status"] == 0
        assert o["latency_s"] >= o["run_s"] > 0.0
        one = _alone(r)
        assert np.array_equal(o["iters"], one["iters"]), (r["shape"], o["iters"], one["iters"])
        assert np.array_equal(o["u"], one["u"]) and np.array_equal(o["C_hom"], one["C_hom"])
        assert o["rel_res"].max() <= 1e-8 * 1.01
    srv.close()


def test_admission_respects_the_memory_budget_and_reuses_solvers():
    from paper_2508_02613_gb300.jfft import Server, workspace_estimate
    big = workspace_estimate((256, 256), "mixed", 3)
    small = workspace_estimate((64, 64), "mixed", 3)
    budget = int(1.5 * big)            # one 256^2 solver at a time, plus small ones
    srv = Server(max_active=3, hbm_budget=budget)
    ids = []
    for i in range(8):
        shape = (256, 256) if i % 2 == 0 else (64, 64)
        rho = smooth_density(shape, 16, 6.0, 200 + i)
        ids.append(srv.submit(shape, rho, 0.3, mandel_unit_loads(2)[:1], 1e-8, "green_jacobi", "mixed",
                              kind="density", e_min=1e-3, e_max=1.0, exponent=2.0))
    outs = [srv.wait(i) for i in ids]
    st = srv.stats()
    assert all(o["status"] == 0 for o in outs)
    assert st["peak_used"] <= budget
    assert st["solvers_reused"] >= 1
    assert st["solvers_created"] <= 1 + budget // small
    srv.close()


def test_request_larger_than_the_budget_is_rejected():
    from paper_2508_02613_gb300.jfft import JfftError, Server
    srv = Server(max_active=1, hbm_budget=1 << 20)
    with pytest.raises(JfftError):
        srv.submit((256, 256), np.ones((256, 256)), 0.3, mandel_unit_loads(2)[:1], 1e-8)
    srv.close()


def test_poisson_ratio_change_on_a_live_solver():
    """set_material with another nu (after graphs were captured) gives the result of a
    solver created with that nu."""
    from paper_2508_02613_gb300.jfft import Solver
    shape = (64, 64)
    rho = smooth_density(shape, 16, 6.0, 300)
    a = Solver(shape, rho, 0.3, kind="density", e_min=1e-3, e_max=1.0, exponent=2.0)
    a.solve(mandel_unit_loads(2), 1e-8, "green_jacobi")   # graphs captured with nu = 0.3
    a.set_material(rho, nu=0.37)
    b = Solver(shape, rho, 0.37, kind="density", e_min=1e-3, e_max=1.0, exponent=2.0)
    oa = a.solve(mandel_unit_loads(2), 1e-8, "green_jacobi")
    ob = b.solve(mandel_unit_loads(2), 1e-8, "green_jacobi")
    assert np.array_equal(oa["u"], ob["u"]) and np.array_equal(oa["iters"], ob["iters"])


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_served_results_match_the_oracle(precision):
    """Small requests (32^2, 32 x 64, 8^3, 8 x 8 x 16; different contrasts, Poisson ratios, load sets
    and preconditioners) served concurrently, against the FP64 oracle solved to 1e-13: the
    served u is within the rigorous residual bound ||f - K u|| / lambda_min of the oracle's
    (plus the oracle's own residual bound), C_hom within 10 tol."""
    from oracle import assemble, material, solve as osolve
    from paper_2508_02613_gb300.jfft import Server
    from tests.test_gpu_mixed import error_bound
    cases = [((32, 32), 1e3, 0.25, [0, 2], "green_jacobi"), ((32, 64), 1e5, 0.35, [1], "green"),
             ((8, 8, 8), 1e3, 0.3, [0, 3, 5], "green_jacobi"), ((8, 8, 16), 1e4, 0.22, [5], "green_jacobi"),
             ((32, 32), 1e2, 0.4, [0, 1, 2], "green")]
    srv = Server(max_active=4)
    subs = []
    for i, (shape, contrast, nu, loads, pc) in enumerate(cases):
        d = len(shape)
        rho = smooth_density(shape, 12 if d == 2 else 16, 4.0, 300 + i)
        eps = mandel_unit_loads(d)[loads]
        rid = srv.submit(shape, rho, nu, eps, 1e-8, pc, precision, kind="density", e_min=1.0 / contrast, e_max=1.0,
                         exponent=2.0, want_u=True)
        subs.append((rid, shape, rho, contrast, nu, eps, pc))
    for rid, shape, rho, contrast, nu, eps, pc in subs:
        o = srv.wait(rid)
        assert o["status"] == 0 and o["rel_res"].max() <= 1e-8 * 1.01
        E = material.young_from_density(rho, 1.0 / contrast, 1.0, 2.0)
        prob = osolve.setup(shape, E, nu)
        ref = osolve.solve(prob, eps, 1e-13, pc)
        assert np.abs(o["C_hom"] - ref.C_hom).max() <= 10 * 1e-8 * np.abs(ref.C_hom).max()
        for g in range(len(eps)):
            f = assemble.assemble_rhs(shape, E, prob.C, eps[g])
            assert np.linalg.norm(o["u"][g] - ref.u[g]) <= error_bound(prob, f, o["u"][g], ref.u[g]), (shape, g)
    srv.close()
