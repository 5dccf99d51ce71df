"""ctypes binding of libjfft (include/jfft.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts NumPy arrays
(host io mode) or CUDA tensor pointers (device io mode) to the C ABI and raises
``JfftError`` on failure. There is no CPU fallback: if the library is missing or
cannot be loaded, ``load()`` raises.
"""

from __future__ import annotations

import ctypes
import os
import re
from ctypes import POINTER, c_char_p, c_double, c_int, c_int64, c_size_t, c_void_p

import numpy as np

from . import build as _build

JFFT_OK, JFFT_ERR_ARG, JFFT_ERR_OOM, JFFT_ERR_CUDA = 0, 1, 2, 3
JFFT_ERR_NOCONV, JFFT_ERR_BREAKDOWN, JFFT_ERR_TIMEOUT, JFFT_ERR_UNSUPPORTED = 4, 5, 6, 7
PRECOND = {"none": -1, "green": 0, "green_jacobi": 1, "jacobi": 2}
MATERIAL = {"young": 0, "density": 1}
STOP = {"rel": 0, "abs_sq": 1}
MEM = {"host": 0, "device": 1}
PRECISION = {"fp64": 0, "mixed": 1}
ELEMENT = {"q1": 0, "p1": 1}
DIAG = {"closed_form": 0, "combs": 1}


class JfftGrid(ctypes.Structure):
    _fields_ = [("dim", c_int), ("n", c_int64 * 3)]


class JfftMaterial(ctypes.Structure):
    _fields_ = [("kind", c_int), ("field", POINTER(c_double)), ("nu", c_double), ("e_min", c_double),
                ("e_max", c_double), ("exponent", c_double)]


class JfftOptions(ctypes.Structure):
    _fields_ = [("precision", c_int), ("max_iter", c_int), ("stop_mode", c_int), ("stream", c_void_p),
                ("hbm_budget", c_size_t), ("check_every", c_int), ("io_memory", c_int), ("max_loads", c_int),
                ("void_value", c_double), ("device", c_int), ("inner_tol", c_double), ("max_refine", c_int),
                ("graphs", c_int), ("element", c_int), ("autotune", c_int), ("reliable", c_int),
                ("material_bf16", c_int)]


class JfftResult(ctypes.Structure):
    _fields_ = [("u", c_void_p), ("stress", c_void_p), ("C_hom", c_void_p), ("iters", c_void_p),
                ("rel_res", c_void_p), ("refine_steps", c_void_p)]


class JfftServerOptions(ctypes.Structure):
    _fields_ = [("max_active", c_int), ("hbm_budget", c_size_t), ("device", c_int)]


class JfftRequest(ctypes.Structure):
    _fields_ = [("grid", JfftGrid), ("material", JfftMaterial), ("n_loads", c_int), ("eps_bar", c_void_p),
                ("tol", c_double), ("precond", c_int), ("precision", c_int), ("want_u", c_int)]


class JfftServerCounters(ctypes.Structure):
    _fields_ = [("submitted", c_int64), ("finished", c_int64), ("queued", c_int64), ("running", c_int64),
                ("budget", c_size_t), ("used", c_size_t), ("peak_used", c_size_t),
                ("solvers_created", c_int64), ("solvers_reused", c_int64), ("solvers_evicted", c_int64)]


class JfftError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"jfft status {status}: {msg}")
        self.status = status


_LIB = None

_SIGNATURES = {
    "jfft_default_options": (None, [POINTER(JfftOptions)]),
    "jfft_create": (c_int, [POINTER(c_void_p), POINTER(JfftGrid), POINTER(JfftMaterial), c_void_p,
                            POINTER(JfftOptions)]),
    "jfft_set_material": (c_int, [c_void_p, POINTER(JfftMaterial)]),
    "jfft_set_material_coarse": (c_int, [c_void_p, POINTER(JfftMaterial), POINTER(c_int64)]),
    "jfft_solve": (c_int, [c_void_p, c_int, c_void_p, c_double, c_int, POINTER(JfftResult)]),
    "jfft_destroy": (None, [c_void_p]),
    "jfft_status_string": (c_char_p, [c_int]),
    "jfft_last_error": (c_char_p, [c_void_p]),
    "jfft_set_io_memory": (c_int, [c_void_p, c_int]),
    "jfft_set_max_iter": (c_int, [c_void_p, c_int]),
    "jfft_get_material": (c_int, [c_void_p, c_void_p]),
    "jfft_rhs": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "jfft_apply_K": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "jfft_get_diag": (c_int, [c_void_p, c_int, c_void_p]),
    "jfft_get_green": (c_int, [c_void_p, c_void_p]),
    "jfft_apply_precond": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "jfft_solve_rhs": (c_int, [c_void_p, c_int, c_void_p, c_double, c_int, c_void_p, c_void_p]),
    "jfft_postprocess": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "jfft_cells_create": (c_int, [POINTER(c_void_p), POINTER(JfftGrid), c_int, POINTER(JfftOptions)]),
    "jfft_cells_solve": (c_int, [c_void_p, c_int, POINTER(JfftMaterial), c_void_p, c_void_p, c_int, c_void_p,
                                 c_double, c_int, POINTER(JfftResult)]),
    "jfft_cells_destroy": (None, [c_void_p]),
    "jfft_cells_last_error": (ctypes.c_char_p, [c_void_p]),
    "jfft_cells_launch_count": (c_int64, [c_void_p]),
    "jfft_launch_count": (c_int64, [c_void_p]),
    "jfft_graph_replays": (c_int64, [c_void_p]),
    "jfft_get_tuning": (c_int, [c_void_p, POINTER(c_int)]),
    "jfft_set_tuning": (c_int, [c_void_p, POINTER(c_int)]),
    "jfft_server_default_options": (None, [POINTER(JfftServerOptions)]),
    "jfft_server_create": (c_int, [POINTER(c_void_p), POINTER(JfftServerOptions)]),
    "jfft_server_submit": (c_int, [c_void_p, POINTER(JfftRequest), POINTER(c_int64)]),
    "jfft_server_poll": (c_int, [c_void_p, c_int64]),
    "jfft_server_wait": (c_int, [c_void_p, c_int64, POINTER(JfftResult), c_void_p]),
    "jfft_server_stats": (c_int, [c_void_p, POINTER(JfftServerCounters)]),
    "jfft_server_last_error": (ctypes.c_char_p, [c_void_p]),
    "jfft_server_destroy": (None, [c_void_p]),
    "jfft_set_profiling": (c_int, [c_void_p, c_int]),
    "jfft_profile_json": (c_char_p, [c_void_p]),
    "jfft_workspace_bytes": (c_size_t, [c_void_p]),
    "jfft_workspace_estimate": (c_int, [POINTER(JfftGrid), POINTER(JfftOptions), POINTER(c_size_t)]),
    "jfft_set_stream": (c_int, [c_void_p, c_void_p]),
    "jfft_apply_K_dot_noalloc": (c_int, [POINTER(JfftGrid), c_double, c_void_p, c_void_p, c_void_p, c_void_p,
                                         c_void_p]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libjfft.so (built in-tree by ``build.build()``); raises if it is absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError(f"libjfft.so not built at {path}; run paper_2508_02613_gb300.build.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def header_functions() -> list[str]:
    """Names of the functions declared in include/jfft.h."""
    hdr = os.path.join(_build.INCLUDE, "jfft.h")
    src = open(hdr).read()
    return sorted(set(re.findall(r"^\s*(?:[\w\*]+\s+)+\**(jfft_\w+)\s*\(", src, re.M)))


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(c_void_p)
    if hasattr(a, "data_ptr"):
        return c_void_p(a.data_ptr())
    raise TypeError(type(a))


def _f64(a, shape=None):
    out = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        out = out.reshape(shape)
    return out


def _check_noalloc_tensor(name, t, numel):
    """The C call reads and writes raw device pointers with no way to check them, so the
    binding requires contiguous float64 CUDA tensors on the current device, of the size
    the grid implies, before it passes a pointer on."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name} must be a torch CUDA tensor, got {type(t).__name__}")
    if not t.is_cuda or t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} must live on the current CUDA device (cuda:{torch.cuda.current_device()}), "
                         f"not {t.device}")
    if t.dtype != torch.float64:
        raise ValueError(f"{name} must be float64, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, the grid needs {numel}")


def apply_K_dot_noalloc(shape, nu, E, x, y, xy, stream=None) -> int:
    """jfft_apply_K_dot_noalloc on CUDA tensors E [*shape], x / y [d, *shape], xy [1];
    returns the status code (no allocation happens in the library). Raises ValueError
    before the call if a tensor is not a contiguous float64 tensor on the current
    CUDA device with the element count the grid implies."""
    lib = load()
    d = len(shape)
    N = int(np.prod([int(v) for v in shape]))
    _check_noalloc_tensor("E", E, N)
    _check_noalloc_tensor("x", x, d * N)
    _check_noalloc_tensor("y", y, d * N)
    _check_noalloc_tensor("xy", xy, 1)
    g = JfftGrid(d, (c_int64 * 3)(*(list(int(s) for s in shape) + [0] * (3 - d))))
    return lib.jfft_apply_K_dot_noalloc(ctypes.byref(g), float(nu), _ptr(E), _ptr(x), _ptr(y), _ptr(xy),
                                        c_void_p(stream) if stream else None)


class Solver:
    """One grid + material; methods mirror the C calls of the same name."""

    def __init__(self, shape, field, nu, kind="young", e_min=0.0, e_max=1.0, exponent=1.0, C_ref=None,
                 max_iter=100000, stop_mode="rel", stream=None, check_every=8, io="host", max_loads=6,
                 void_value=1.0, device=0, hbm_budget=0, pinned=False, precision="fp64", inner_tol=1e-3,
                 max_refine=30, graphs=True, element="q1", autotune=False, reliable=False, material_bf16=False):
        self.lib = load()
        self.pinned = pinned
        self.shape = tuple(int(s) for s in shape)
        self.d = len(self.shape)
        self.ds = self.d * (self.d + 1) // 2
        self.N = int(np.prod(self.shape))
        self.io = io
        g = JfftGrid(self.d, (c_int64 * 3)(*(list(self.shape) + [0] * (3 - self.d))))
        self._field = _f64(field).reshape(-1)
        mat = JfftMaterial(MATERIAL[kind], self._field.ctypes.data_as(POINTER(c_double)), nu, e_min, e_max, exponent)
        self._mat_args = (kind, nu, e_min, e_max, exponent)
        opt = JfftOptions()
        self.lib.jfft_default_options(ctypes.byref(opt))
        opt.max_iter = max_iter
        opt.stop_mode = STOP[stop_mode]
        opt.stream = c_void_p(stream) if stream else None
        opt.check_every = check_every
        opt.io_memory = MEM[io]
        opt.max_loads = max_loads
        opt.void_value = void_value
        opt.device = device
        opt.hbm_budget = hbm_budget
        opt.precision = PRECISION[precision]
        opt.inner_tol = inner_tol
        opt.max_refine = max_refine
        opt.graphs = 1 if graphs else 0
        opt.element = ELEMENT[element]
        opt.autotune = 1 if autotune else 0
        opt.reliable = 1 if reliable else 0
        opt.material_bf16 = 1 if material_bf16 else 0
        self.precision = precision
        self.max_loads = max(max_loads, self.d)
        h = c_void_p()
        cref = None if C_ref is None else _f64(C_ref).reshape(-1)
        st = self.lib.jfft_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(mat), _ptr(cref), ctypes.byref(opt))
        if st != JFFT_OK:
            msg = self.lib.jfft_last_error(None) or self.lib.jfft_status_string(st)
            raise JfftError(st, msg.decode() if isinstance(msg, bytes) else msg)
        self.h = h

    # -- plumbing
    def _check(self, st, allow=()):
        if st != JFFT_OK and st not in allow:
            raise JfftError(st, self.lib.jfft_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.jfft_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _out(self, shape, dtype=np.float64):
        if self.io == "host":
            if self.pinned:
                import torch
                tdt = torch.float64 if dtype == np.float64 else torch.int32
                return torch.empty(shape, dtype=tdt, pin_memory=True).numpy()
            return np.empty(shape, dtype=dtype)
        import torch
        tdt = torch.float64 if dtype == np.float64 else torch.int32
        return torch.empty(shape, dtype=tdt, device="cuda")

    def _in(self, a, shape):
        if self.io == "host":
            return _f64(a, shape)
        return a

    # -- calls
    def set_material(self, field, e_min=None, e_max=None, exponent=None, nu=None):
        """New material field (host array, or a CUDA tensor in device io mode); the
        density map parameters and nu (with the mean reference material) may change,
        the kind may not."""
        kind, nu0, e_min0, e_max0, exponent0 = self._mat_args
        nu = nu0 if nu is None else nu
        e_min = e_min0 if e_min is None else e_min
        e_max = e_max0 if e_max is None else e_max
        exponent = exponent0 if exponent is None else exponent
        self._mat_args = (kind, nu, e_min, e_max, exponent)
        if self.io == "host":
            self._field = _f64(field).reshape(-1)
            fptr = self._field.ctypes.data_as(POINTER(c_double))
        else:
            self._field = field
            fptr = ctypes.cast(c_void_p(field.data_ptr()), POINTER(c_double))
        mat = JfftMaterial(MATERIAL[kind], fptr, nu, e_min, e_max, exponent)
        self._check(self.lib.jfft_set_material(self.h, ctypes.byref(mat)))

    def set_material_coarse(self, field, e_min=None, e_max=None, exponent=None, nu=None):
        """Geometry G_p: field has p_a pixels per axis (powers of two, p_a <= n_a); every
        voxel takes the value of its pixel (host array, or a CUDA tensor in device io)."""
        kind, nu0, e_min0, e_max0, exponent0 = self._mat_args
        nu = nu0 if nu is None else nu
        e_min = e_min0 if e_min is None else e_min
        e_max = e_max0 if e_max is None else e_max
        exponent = exponent0 if exponent is None else exponent
        self._mat_args = (kind, nu, e_min, e_max, exponent)
        pix = (c_int64 * 3)(*(list(field.shape) + [0] * (3 - len(field.shape))))
        if self.io == "host":
            self._field = _f64(field).reshape(-1)
            fptr = self._field.ctypes.data_as(POINTER(c_double))
        else:
            self._field = field
            fptr = ctypes.cast(c_void_p(field.data_ptr()), POINTER(c_double))
        mat = JfftMaterial(MATERIAL[kind], fptr, nu, e_min, e_max, exponent)
        self._check(self.lib.jfft_set_material_coarse(self.h, ctypes.byref(mat), pix))

    def set_io_memory(self, io):
        self._check(self.lib.jfft_set_io_memory(self.h, MEM[io]))
        self.io = io

    def set_max_iter(self, m):
        self._check(self.lib.jfft_set_max_iter(self.h, int(m)))

    def set_stream(self, stream):
        self._check(self.lib.jfft_set_stream(self.h, c_void_p(stream) if stream else None))

    def solve(self, eps_bar, tol, precond="green_jacobi", want_u=True, want_stress=True):
        eps = np.atleast_2d(_f64(eps_bar)) if self.io == "host" else eps_bar
        nl = int(eps.shape[0])
        u = self._out((nl, self.d) + self.shape) if want_u else None
        stress = self._out((nl, self.ds) + self.shape) if want_stress else None
        chom = self._out((self.ds, nl))
        its = self._out((nl,), np.int32)
        rel = self._out((nl,))
        ref = self._out((nl,), np.int32)
        res = JfftResult(_ptr(u), _ptr(stress), _ptr(chom), _ptr(its), _ptr(rel), _ptr(ref))
        st = self._check(self.lib.jfft_solve(self.h, nl, _ptr(eps), float(tol), PRECOND[precond], ctypes.byref(res)),
                         allow=(JFFT_ERR_NOCONV, JFFT_ERR_BREAKDOWN))
        return {"u": u, "stress": stress, "C_hom": chom, "iters": its, "rel_res": rel, "refine_steps": ref,
                "status": st}

    def get_material(self):
        E = self._out(self.shape)
        self._check(self.lib.jfft_get_material(self.h, _ptr(E)))
        return E

    def rhs(self, eps_bar):
        eps = np.atleast_2d(_f64(eps_bar)) if self.io == "host" else eps_bar
        f = self._out((int(eps.shape[0]), self.d) + self.shape)
        self._check(self.lib.jfft_rhs(self.h, int(eps.shape[0]), _ptr(eps), _ptr(f)))
        return f

    def apply_K(self, x):
        x = self._in(x, (-1, self.d) + self.shape)
        y = self._out(tuple(x.shape))
        self._check(self.lib.jfft_apply_K(self.h, int(x.shape[0]), _ptr(x), _ptr(y)))
        return y

    def get_diag(self, method="closed_form"):
        out = self._out((self.d,) + self.shape)
        self._check(self.lib.jfft_get_diag(self.h, DIAG[method], _ptr(out)))
        return out

    def get_green(self):
        F = self.N // self.shape[-1] * (self.shape[-1] // 2 + 1)
        out = self._out((F, self.d, self.d))
        self._check(self.lib.jfft_get_green(self.h, _ptr(out)))
        return out

    def apply_precond(self, precond, r):
        r = self._in(r, (-1, self.d) + self.shape)
        z = self._out(tuple(r.shape))
        self._check(self.lib.jfft_apply_precond(self.h, PRECOND[precond], int(r.shape[0]), _ptr(r), _ptr(z)))
        return z

    def solve_rhs(self, f, tol, precond="green_jacobi"):
        f = self._in(f, (-1, self.d) + self.shape)
        nb = int(f.shape[0])
        u = self._out(tuple(f.shape))
        its = self._out((nb,), np.int32)
        st = self._check(self.lib.jfft_solve_rhs(self.h, nb, _ptr(f), float(tol), PRECOND[precond], _ptr(u), _ptr(its)),
                         allow=(JFFT_ERR_NOCONV, JFFT_ERR_BREAKDOWN))
        return {"u": u, "iters": its, "status": st}

    def postprocess(self, eps_bar, u):
        eps = np.atleast_2d(_f64(eps_bar)) if self.io == "host" else eps_bar
        nl = int(eps.shape[0])
        u = self._in(u, (nl, self.d) + self.shape)
        stress = self._out((nl, self.ds) + self.shape)
        chom = self._out((self.ds, nl))
        self._check(self.lib.jfft_postprocess(self.h, nl, _ptr(eps), _ptr(u), _ptr(stress), _ptr(chom)))
        return {"stress": stress, "C_hom": chom}

    @property
    def launch_count(self) -> int:
        return int(self.lib.jfft_launch_count(self.h))

    @property
    def graph_replays(self) -> int:
        return int(self.lib.jfft_graph_replays(self.h))

    @property
    def tuning(self) -> list:
        t = (c_int * 4)()
        self._check(self.lib.jfft_get_tuning(self.h, t))
        return list(t)

    def set_tuning(self, tune):
        self._check(self.lib.jfft_set_tuning(self.h, (c_int * 4)(*tune)))

    @property
    def workspace_bytes(self) -> int:
        return int(self.lib.jfft_workspace_bytes(self.h))

    def set_profiling(self, on: bool):
        self._check(self.lib.jfft_set_profiling(self.h, 1 if on else 0))

    def profile(self) -> dict:
        import json
        return json.loads(self.lib.jfft_profile_json(self.h).decode())


class Cells:
    """Batch of small 2D cells solved in one launch (jfft_cells_*): one grid shape
    (n0, n1 powers of two in [4, 32]), per-cell material fields, Poisson ratios and
    lower moduli, shared macroscopic strains."""

    def __init__(self, shape, max_cells, max_loads=3, max_iter=100000, stop_mode="rel", stream=None,
                 io="host", void_value=1.0, device=0):
        self.lib = load()
        self.shape = tuple(int(s) for s in shape)
        self.N = int(np.prod(self.shape))
        self.io = io
        g = JfftGrid(len(self.shape), (c_int64 * 3)(*(list(self.shape) + [0] * (3 - len(self.shape)))))
        opt = JfftOptions()
        self.lib.jfft_default_options(ctypes.byref(opt))
        opt.max_iter = max_iter
        opt.stop_mode = STOP[stop_mode]
        opt.stream = c_void_p(stream) if stream else None
        opt.io_memory = MEM[io]
        opt.max_loads = max_loads
        opt.void_value = void_value
        opt.device = device
        h = c_void_p()
        st = self.lib.jfft_cells_create(ctypes.byref(h), ctypes.byref(g), int(max_cells), ctypes.byref(opt))
        if st != JFFT_OK:
            raise JfftError(st, self.lib.jfft_cells_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.jfft_cells_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _out(self, shape, dtype=np.float64):
        if self.io == "host":
            return np.empty(shape, dtype=dtype)
        import torch
        return torch.empty(shape, dtype=torch.float64 if dtype == np.float64 else torch.int32, device="cuda")

    @property
    def launch_count(self) -> int:
        return int(self.lib.jfft_cells_launch_count(self.h))

    def solve(self, fields, nu, eps_bar, tol, precond="green_jacobi", kind="young", e_min=0.0, e_max=1.0,
              exponent=1.0, want_u=True):
        """fields [n_cells, *shape]; nu and e_min scalars or [n_cells] arrays."""
        n_cells = int(fields.shape[0])
        nu_a = np.broadcast_to(np.asarray(nu, dtype=np.float64), (n_cells,)).copy()
        em_a = np.broadcast_to(np.asarray(e_min, dtype=np.float64), (n_cells,)).copy()
        eps = _f64(np.atleast_2d(eps_bar))
        nl = int(eps.shape[0])
        if self.io == "host":
            self._fields = _f64(fields).reshape(n_cells, -1)
            fptr = self._fields.ctypes.data_as(POINTER(c_double))
        else:
            self._fields = fields
            fptr = ctypes.cast(c_void_p(fields.data_ptr()), POINTER(c_double))
        mat = JfftMaterial(MATERIAL[kind], fptr, float(nu_a[0]), float(em_a[0]), e_max, exponent)
        u = self._out((n_cells, nl, 2) + self.shape) if want_u else None
        chom = self._out((n_cells, 3, nl))
        its = self._out((n_cells, nl), np.int32)
        rel = self._out((n_cells, nl))
        res = JfftResult(_ptr(u), None, _ptr(chom), _ptr(its), _ptr(rel), None)
        st = self.lib.jfft_cells_solve(self.h, n_cells, ctypes.byref(mat), _ptr(nu_a), _ptr(em_a), nl, _ptr(eps),
                                       float(tol), PRECOND[precond], ctypes.byref(res))
        if st not in (JFFT_OK, JFFT_ERR_NOCONV, JFFT_ERR_BREAKDOWN):
            raise JfftError(st, self.lib.jfft_cells_last_error(self.h).decode())
        return {"u": u, "C_hom": chom, "iters": its, "rel_res": rel, "status": st}


class Server:
    """Request server with continuous batching (jfft_server_*): submit() queues a solve
    and returns its id at once; wait(id) returns its results and timings."""

    def __init__(self, max_active=4, hbm_budget=0, device=0):
        self.lib = load()
        opt = JfftServerOptions()
        self.lib.jfft_server_default_options(ctypes.byref(opt))
        opt.max_active = max_active
        opt.hbm_budget = hbm_budget
        opt.device = device
        h = c_void_p()
        st = self.lib.jfft_server_create(ctypes.byref(h), ctypes.byref(opt))
        if st != JFFT_OK:
            raise JfftError(st, "jfft_server_create failed")
        self.h = h
        self._meta = {}

    def close(self):
        if getattr(self, "h", None):
            self.lib.jfft_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, shape, field, nu, eps_bar, tol, precond="green_jacobi", precision="mixed", kind="young",
               e_min=0.0, e_max=1.0, exponent=1.0, want_u=False) -> int:
        shape = tuple(int(v) for v in shape)
        d = len(shape)
        fld = _f64(field).reshape(-1)
        eps = _f64(np.atleast_2d(eps_bar))
        g = JfftGrid(d, (c_int64 * 3)(*(list(shape) + [0] * (3 - d))))
        mat = JfftMaterial(MATERIAL[kind], fld.ctypes.data_as(POINTER(c_double)), nu, e_min, e_max, exponent)
        req = JfftRequest(g, mat, int(eps.shape[0]), eps.ctypes.data_as(c_void_p), float(tol), PRECOND[precond],
                          PRECISION[precision], 1 if want_u else 0)
        rid = c_int64()
        st = self.lib.jfft_server_submit(self.h, ctypes.byref(req), ctypes.byref(rid))
        if st != JFFT_OK:
            raise JfftError(st, self.lib.jfft_server_last_error(self.h).decode())
        self._meta[rid.value] = (shape, int(eps.shape[0]), bool(want_u))
        return rid.value

    def poll(self, rid) -> int:
        return int(self.lib.jfft_server_poll(self.h, int(rid)))

    def wait(self, rid):
        shape, nl, want_u = self._meta.pop(rid)
        d = len(shape)
        ds = d * (d + 1) // 2
        u = np.empty((nl, d) + shape) if want_u else None
        chom = np.empty((ds, nl))
        its = np.empty(nl, dtype=np.int32)
        rel = np.empty(nl)
        ref = np.empty(nl, dtype=np.int32)
        res = JfftResult(_ptr(u), None, _ptr(chom), _ptr(its), _ptr(rel), _ptr(ref))
        timing = np.zeros(4)
        st = self.lib.jfft_server_wait(self.h, int(rid), ctypes.byref(res), _ptr(timing))
        return {"u": u, "C_hom": chom, "iters": its, "rel_res": rel, "refine_steps": ref, "status": st,
                "queued_s": float(timing[0]), "run_s": float(timing[1]), "latency_s": float(timing[2]),
                "reused_solver": bool(timing[3])}

    def stats(self) -> dict:
        c = JfftServerCounters()
        self.lib.jfft_server_stats(self.h, ctypes.byref(c))
        return {f: int(getattr(c, f)) for f, _ in JfftServerCounters._fields_}


def workspace_estimate(shape, precision="fp64", max_loads=6, element="q1", material_bf16=False) -> int:
    """Device bytes jfft_create would allocate for this grid (jfft_workspace_estimate)."""
    lib = load()
    shape = tuple(int(v) for v in shape)
    g = JfftGrid(len(shape), (c_int64 * 3)(*(list(shape) + [0] * (3 - len(shape)))))
    opt = JfftOptions()
    lib.jfft_default_options(ctypes.byref(opt))
    opt.precision = PRECISION[precision]
    opt.max_loads = max_loads
    opt.element = ELEMENT[element]
    opt.material_bf16 = 1 if material_bf16 else 0
    out = c_size_t()
    st = lib.jfft_workspace_estimate(ctypes.byref(g), ctypes.byref(opt), ctypes.byref(out))
    if st != JFFT_OK:
        raise JfftError(st, "unsupported grid")
    return int(out.value)
