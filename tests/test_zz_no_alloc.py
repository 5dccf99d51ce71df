"""The allocation-free operator step against the handle-based one.

jfft_apply_K_dot_noalloc serves callers that cannot allocate device memory (their
device memory already belongs to another pool, or their loop must not take the
synchronisation an allocation can cause); it keeps its partial sums in a static
device array shared by all calls. This file is collected last so that a run which
stops at the first failure has run every other test first.
"""

import numpy as np
import pytest

from synthetic import random_field, smooth_density

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(64, 512), (16, 16, 64)])
def test_noalloc_operator_matches_handle_operator_twice(shape):
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_02613_gb300.jfft import Solver, apply_K_dot_noalloc

    d = len(shape)
    rho = smooth_density(shape, 8, 3.0, 21)
    s = Solver(shape, rho, 0.3, kind="density", e_min=1e-4, e_max=1.0, exponent=2.0)
    E = torch.tensor(s.get_material(), device="cuda")
    for call in range(2):  # two calls in a row: the shared scratch must not leak state
        x_h = random_field((d,) + shape, 100 + call)
        y_ref = s.apply_K(x_h[None])[0]
        x = torch.tensor(x_h, device="cuda")
        y = torch.empty_like(x)
        xy = torch.empty(1, dtype=torch.float64, device="cuda")
        st = apply_K_dot_noalloc(shape, 0.3, E, x, y, xy, torch.cuda.current_stream().cuda_stream)
        assert st == 0
        torch.cuda.synchronize()
        y_h = y.cpu().numpy()
        assert np.abs(y_h - y_ref).max() <= 1e-13 * np.abs(y_ref).max()
        dot_ref = float(np.sum(x_h * y_ref))
        assert abs(float(xy.item()) - dot_ref) <= 1e-13 * np.sum(np.abs(x_h * y_ref))
    s.close()


def test_noalloc_rejects_unsupported_sizes():
    torch = pytest.importorskip("torch")
    from paper_2508_02613_gb300.jfft import apply_K_dot_noalloc
    E = torch.ones(6, 8, dtype=torch.float64, device="cuda")
    x = torch.zeros(2, 6, 8, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    xy = torch.empty(1, dtype=torch.float64, device="cuda")
    assert apply_K_dot_noalloc((6, 8), 0.3, E, x, y, xy) == 7          # not a power of two
    big = (4096, 4)
    assert apply_K_dot_noalloc(big, 0.3, E, x, y, xy) == 7             # beyond the largest axis
