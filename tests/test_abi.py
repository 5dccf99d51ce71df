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
