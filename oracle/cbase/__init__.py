"""Timed CPU baseline (TEST INFRASTRUCTURE, not the product): the oracle's PCG in plain C
with a matrix-free operator, a textbook radix-2 FFT and OpenMP on every host core
(pcg_cpu.c). Setup arrays (element matrix, Alg. 1 symbol, J^(1/2)) come from the
Python oracle; only tests/ and the CPU legs of bench.py use this module.

    build()                     compile pcg_cpu.c into libjfft_cpu.so next to it (gcc, -fopenmp)
    pcg(prob, f, tol, precond)  solve K u = f for an oracle.solve.CellProblem
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pcg_cpu.c")
LIB = os.path.join(HERE, "libjfft_cpu.so")
_lib = None


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off", SRC, "-o", tmp, "-lm"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("gcc failed:\n" + r.stdout)
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(LIB)
        P = ctypes.c_void_p
        lib.jfft_cpu_pcg.restype = ctypes.c_int
        lib.jfft_cpu_pcg.argtypes = [ctypes.c_int, P, P, P, P, P, P, ctypes.c_double, ctypes.c_int, P,
                                     ctypes.POINTER(ctypes.c_int)]
        lib.jfft_cpu_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def threads() -> int:
    return int(_load().jfft_cpu_threads())


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def pcg(prob, f, tol, precond="green_jacobi", max_iter=100000):
    """Solve K u = f (f [d, *n]) with the C baseline for the oracle problem ``prob``
    (matrix-free K from its unit element matrix, its Alg. 1 symbol and J^(1/2)).
    Returns (u, iterations, converged)."""
    from oracle import assemble, fe
    lib = _load()
    n = tuple(prob.n)
    d = len(n)
    A = np.ascontiguousarray(fe.element_matrix(d, assemble.grid_spacing(n), np.asarray(prob.C, np.float64),
                                               prob.element), dtype=np.float64)
    E = np.ascontiguousarray(prob.E, dtype=np.float64)
    G = np.ascontiguousarray(prob.G_hat, dtype=np.float64)
    J = None
    if precond == "green_jacobi":
        J = np.ascontiguousarray(np.broadcast_to(prob.J_half, (d,) + n), dtype=np.float64)
    elif precond != "green":
        raise ValueError(precond)
    f = np.ascontiguousarray(f, dtype=np.float64)
    u = np.empty_like(f)
    nn = np.array(n, dtype=np.int64)
    conv = ctypes.c_int(0)
    k = lib.jfft_cpu_pcg(d, _p(nn), _p(E), _p(A), _p(G), _p(J), _p(f), float(tol), int(max_iter), _p(u),
                         ctypes.byref(conv))
    if k < 0:
        raise RuntimeError("jfft_cpu_pcg rejected its arguments")
    return u, int(k), bool(conv.value)
