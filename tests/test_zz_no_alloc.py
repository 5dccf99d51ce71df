"""The allocation-free operator step against the handle-based one.

jfft_apply_K_dot_noalloc serves callers that cannot allocate device memory (their
device memory already belongs to another pool, or their loop must not take the
synchronisation an allocation can cause); it keeps its partial sums in a static
device array shared by all calls. This file is collected last so that a run which
stops at the first failure has run every other test first.

Every call below passes buffers sized for the grid it names, so a regression in the
library's own checks shows up as a wrong status or a wrong result, never as an
access outside a buffer.
"""

import numpy as np
import pytest

from synthetic import random_field, smooth_density

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _compare_twice(shape, s, E, make_x, tol=1e-13):
    """Two calls in a row on fresh inputs (the shared scratch must not leak state
    between calls); y and x.y against the handle's operator."""
    torch = pytest.importorskip("torch")
    from paper_2508_02613_gb300.jfft import apply_K_dot_noalloc
    for call in range(2):
        x = make_x(call)
        y_ref = s.apply_K(x[None])[0]
        y = torch.empty_like(x)
        xy = torch.empty(1, dtype=torch.float64, device="cuda")
        st = apply_K_dot_noalloc(shape, 0.3, E, x, y, xy, torch.cuda.current_stream().cuda_stream)
        assert st == 0
        torch.cuda.synchronize()
        assert float((y - y_ref).abs().max()) <= tol * float(y_ref.abs().max())
        prod = x * y_ref
        assert abs(float(xy.item()) - float(prod.sum())) <= tol * float(prod.abs().sum())


@pytest.mark.parametrize("shape", [(64, 512), (16, 16, 64)])
def test_noalloc_operator_matches_handle_operator_twice(shape):
    torch = pytest.importorskip("torch")
    from paper_2508_02613_gb300.jfft import Solver

    d = len(shape)
    rho = smooth_density(shape, 8, 3.0, 21)
    s = Solver(shape, rho, 0.3, kind="density", e_min=1e-4, e_max=1.0, exponent=2.0)
    E = torch.tensor(s.get_material(), device="cuda")
    s.set_io_memory("device")
    _compare_twice(shape, s, E, lambda call: torch.tensor(random_field((d,) + shape, 100 + call), device="cuda"))
    s.close()


def test_noalloc_lengthened_march_segment():
    """A 3D grid of 2^26 voxels needs more than 8192 blocks at the default march segment
    (16 node layers), so the launch lengthens the segment to 32 layers to fit the
    static partial-sum array; the result must not change."""
    torch = pytest.importorskip("torch")
    from paper_2508_02613_gb300.jfft import Solver

    shape = (1024, 1024, 64)
    i0 = np.arange(shape[0])[:, None, None]
    i1 = np.arange(shape[1])[None, :, None]
    i2 = np.arange(shape[2])[None, None, :]
    E_h = 1.0 + 0.9 * np.cos(2 * np.pi * (3 * i0 / shape[0] + i1 / shape[1])) * np.sin(2 * np.pi * i2 / shape[2])
    s = Solver(shape, E_h, 0.3, max_loads=3)
    E = torch.tensor(E_h, device="cuda")
    del E_h
    s.set_io_memory("device")

    def make_x(call):
        gen = torch.Generator(device="cuda")
        gen.manual_seed(500 + call)
        return torch.randn((3,) + shape, dtype=torch.float64, device="cuda", generator=gen)

    _compare_twice(shape, s, E, make_x)
    s.close()


def test_noalloc_rejects_unsupported_sizes_and_overlap():
    torch = pytest.importorskip("torch")
    from paper_2508_02613_gb300.jfft import apply_K_dot_noalloc

    def bufs(shape):
        d = len(shape)
        E = torch.ones(shape, dtype=torch.float64, device="cuda")
        x = torch.zeros((d,) + shape, dtype=torch.float64, device="cuda")
        return E, x, torch.empty_like(x), torch.empty(1, dtype=torch.float64, device="cuda")

    E, x, y, xy = bufs((6, 8))
    assert apply_K_dot_noalloc((6, 8), 0.3, E, x, y, xy) == 7          # not a power of two
    E, x, y, xy = bufs((4096, 4))
    assert apply_K_dot_noalloc((4096, 4), 0.3, E, x, y, xy) == 7       # beyond the largest axis
    E, x, y, xy = bufs((16, 16))
    assert apply_K_dot_noalloc((16, 16), 0.3, E, x, x, xy) == 1        # in place: y is x
    assert apply_K_dot_noalloc((16, 16), 0.7, E, x, y, xy) == 1        # nu outside (-1, 0.5)
    torch.cuda.synchronize()


def test_noalloc_binding_validates_tensors():
    torch = pytest.importorskip("torch")
    from paper_2508_02613_gb300.jfft import apply_K_dot_noalloc
    shape = (16, 16)
    E = torch.ones(shape, dtype=torch.float64, device="cuda")
    x = torch.zeros((2,) + shape, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    xy = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        apply_K_dot_noalloc(shape, 0.3, E.cpu().numpy(), x, y, xy)                # host memory
    with pytest.raises(ValueError):
        apply_K_dot_noalloc(shape, 0.3, E, x.float(), y, xy)                      # float32
    with pytest.raises(ValueError):
        apply_K_dot_noalloc(shape, 0.3, E, x, y[:, :8], xy)                       # too few elements
    with pytest.raises(ValueError):
        apply_K_dot_noalloc(shape, 0.3, E.t(), x, y, xy)                          # not contiguous
