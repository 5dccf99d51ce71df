"""Row passes on a capped grid (GPU, through the C ABI).

The FFT row passes that write one partial sum per (component, block) -- the forward
real pass with the fused PCG update x += alpha p, r -= alpha q (||r||^2) and the
inverse real pass (r . z) -- launch at most kMaxPartials / d = 43690 blocks per
component; on grids with more row groups than that every block takes several groups.
512 x 512 x 256 with the row-pass tuning (0, 0, 4, 4) (a quarter of the rows per block)
has 65536 groups per component, so both passes run capped there; the default shapes
(16 rows per block in FP64) stay uncapped.

* z = M^-1 r: every row's transform is independent of how rows are grouped into blocks,
  so the capped and the uncapped runs are bit-identical.
* FP64 PCG after k = 3 iterations with no stopping test: only the summation order of
  r . z and ||r||^2 differs, relative difference of u <= 1e-12.
* Mixed precision to tol 1e-8: the capped run meets the tolerance and lies within
  10 tol of the uncapped one.
"""

import numpy as np
import pytest

from synthetic import mandel_unit_loads

pytestmark = pytest.mark.gpu

SHAPE = (512, 512, 256)
CAPPED = (0, 0, 4, 4)
DEFAULT = (0, 0, 0, 0)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def rho():
    from synthetic import smooth_density_device
    return smooth_density_device(SHAPE, 8, 3.0, 21).cpu().numpy()


def _solver(rho, precision):
    from paper_2508_02613_gb300.jfft import Solver
    return Solver(SHAPE, rho, 0.3, kind="density", e_min=1e-4, e_max=1.0, exponent=2.0, io="device",
                  max_loads=3, precision=precision)


def test_precond_capped_equals_uncapped(rho):
    torch = pytest.importorskip("torch")
    s = _solver(rho, "fp64")
    gen = torch.Generator(device="cuda").manual_seed(5)
    r = torch.randn((1, 3) + SHAPE, dtype=torch.float64, device="cuda", generator=gen)
    for pc in ("green", "green_jacobi"):
        s.set_tuning(DEFAULT)
        a = s.apply_precond(pc, r).clone()
        s.set_tuning(CAPPED)
        b = s.apply_precond(pc, r)
        assert torch.isfinite(a).all() and torch.equal(a, b), pc
    s.close()


def test_pcg_same_k_capped_fp64(rho):
    torch = pytest.importorskip("torch")
    s = _solver(rho, "fp64")
    eps = torch.tensor(mandel_unit_loads(3)[:1], dtype=torch.float64, device="cuda")
    f = s.rhs(eps)
    s.set_max_iter(3)
    for pc in ("green", "green_jacobi"):
        s.set_tuning(DEFAULT)
        ra = s.solve_rhs(f, 0.0, pc)
        a = ra["u"].clone()
        s.set_tuning(CAPPED)
        rb = s.solve_rhs(f, 0.0, pc)
        b = rb["u"]
        assert int(ra["iters"][0]) == 3 and int(rb["iters"][0]) == 3
        d = float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(a))
        print(f"{pc}: capped vs uncapped after 3 iterations {d:.1e}")
        assert d <= 1e-12, (pc, d)
    s.close()


def test_mixed_converged_capped(rho):
    torch = pytest.importorskip("torch")
    eps = torch.tensor(mandel_unit_loads(3)[:1], dtype=torch.float64, device="cuda")
    outs = []
    for tune in (DEFAULT, CAPPED):
        s = _solver(rho, "mixed")
        s.set_tuning(tune)
        out = s.solve(eps, 1e-8, "green_jacobi", want_stress=False)
        outs.append({k: (v.cpu().numpy() if hasattr(v, "cpu") else np.asarray(v)) for k, v in out.items()})
        s.close()
    a, b = outs
    print(f"iterations uncapped {a['iters']}, capped {b['iters']}")
    assert b["rel_res"].max() <= 1e-8 * 1.01
    assert np.linalg.norm(b["u"] - a["u"]) <= 10 * 1e-8 * np.linalg.norm(a["u"])
