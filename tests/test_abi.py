"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/jfft.h declares. Host-only calls only (no GPU needed)."""

import ctypes

import pytest

from paper_2508_02613_gb300 import build as pbuild
from paper_2508_02613_gb300 import jfft


@pytest.fixture(scope="module")
def lib():
    pbuild.build()
    return jfft.load()


def test_every_declared_function_is_exported(lib):
    names = jfft.header_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) == set(jfft._SIGNATURES), "binding and header disagree"


def test_status_strings_and_defaults(lib):
    assert lib.jfft_status_string(0) == b"ok"
    assert b"converged" in lib.jfft_status_string(4)
    opt = jfft.JfftOptions()
    lib.jfft_default_options(ctypes.byref(opt))
    assert opt.max_iter == 100000 and opt.check_every == 8 and opt.max_loads == 6
    assert opt.void_value == 1.0 and opt.io_memory == 0 and opt.stop_mode == 0
    assert opt.precision == 0 and opt.inner_tol == 1e-3 and opt.max_refine == 30 and opt.graphs == 1
    assert opt.element == 0 and opt.autotune == 0 and opt.reliable == 0 and opt.material_bf16 == 0


def test_sources_target_sm103a_only():
    assert pbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_null_handle_calls_are_rejected(lib):
    assert lib.jfft_solve(None, 1, None, 1e-6, 0, None) == jfft.JFFT_ERR_ARG
    assert lib.jfft_apply_K(None, 1, None, None) == jfft.JFFT_ERR_ARG
    assert lib.jfft_launch_count(None) == 0
    assert lib.jfft_graph_replays(None) == 0


def test_workspace_estimate_accounts_for_tables():
    """Host-side sizing (no GPU): the BF16 material copy takes 2 bytes per voxel instead
    of 4; the resolved J^1/2 table holds one factor per node for Q1 on a grid with equal
    spacing and one per DOF for P1 voxels (FP64 table, plus its FP32 copy when mixed)."""
    from paper_2508_02613_gb300.jfft import workspace_estimate
    shape = (64, 64)
    N = 64 * 64
    assert workspace_estimate(shape, "mixed", 3) - workspace_estimate(shape, "mixed", 3, material_bf16=True) == 2 * N
    assert workspace_estimate(shape, "fp64", 3, element="p1") - workspace_estimate(shape, "fp64", 3) == N * 8
    assert workspace_estimate(shape, "mixed", 3, element="p1") - workspace_estimate(shape, "mixed", 3) == N * (8 + 4)
