"""ctypes binding of the ddfd C ABI (include/ddfd.h).

Argument marshalling only: every step of the method runs in the CUDA library.
There is no fallback; if libddfd.so is missing or no GPU is usable, calls fail
with an exception.  The names mirror the C entry points; ``Problem`` wraps a
handle and converts numpy arrays (host calls) or torch CUDA tensors (the
``*_dev`` calls, by data pointer) to the C layout.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_int32, c_int64, c_uint32, c_void_p, c_char_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libddfd.so")

DDFD_OK, DDFD_E_ARG, DDFD_E_CFL, DDFD_E_STATE = 0, -1, -2, -3
DDFD_E_CUDA, DDFD_E_OOM, DDFD_E_NONFINITE, DDFD_E_TIMEOUT, DDFD_E_COEFF = -4, -5, -6, -7, -8
DDFD_FP64, DDFD_FP32 = 0, 1
DDFD_SRC_GAUSS, DDFD_SRC_SINE = 0, 1
DDFD_FEM_STENCIL, DDFD_FEM_EBE, DDFD_FEM_MESH = 0, 1, 2
DDFD_ABS_BOTTOM, DDFD_ABS_TOP, DDFD_ABS_X0, DDFD_ABS_X1, DDFD_ABS_Y0, DDFD_ABS_Y1 = 1, 2, 4, 8, 16, 32

STATUS_NAMES = {0: "DDFD_OK", -1: "DDFD_E_ARG", -2: "DDFD_E_CFL", -3: "DDFD_E_STATE",
                -4: "DDFD_E_CUDA", -5: "DDFD_E_OOM", -6: "DDFD_E_NONFINITE",
                -7: "DDFD_E_TIMEOUT", -8: "DDFD_E_COEFF"}

# Every entry point declared in include/ddfd.h.
ABI_SYMBOLS = (
    "ddfd_config_default", "ddfd_create", "ddfd_destroy", "ddfd_last_error",
    "ddfd_create_error", "ddfd_set_coeffs", "ddfd_set_coeffs_dev", "ddfd_forward",
    "ddfd_forward_dev", "ddfd_functional", "ddfd_functional_dev", "ddfd_adjoint",
    "ddfd_adjoint_dev", "ddfd_gradient", "ddfd_gradient_dev", "ddfd_get_info",
    "ddfd_set_capture", "ddfd_get_capture", "ddfd_get_timing", "ddfd_misfit_noalloc",
    "ddfd_autotune", "ddfd_create_batch", "ddfd_destroy_batch", "ddfd_batch_last_error",
    "ddfd_batch_member", "ddfd_batch_forward", "ddfd_batch_forward_dev", "ddfd_batch_adjoint",
    "ddfd_batch_adjoint_dev", "ddfd_batch_autotune", "ddfd_batch_get_info",
    "ddfd_cg_params_default", "ddfd_cg_run", "ddfd_test_gather_timeout", "ddfd_time_gather",
    "ddfd_test_step_items",
)


class ddfd_config(ctypes.Structure):
    _fields_ = [
        ("n", c_int32), ("fem_n", c_int32), ("n_steps", c_int32), ("cfl", c_double),
        ("precision", c_int32), ("fem_kind", c_int32), ("n_src", c_int32),
        ("src_dir", POINTER(c_double)), ("source_kind", c_int32), ("freq", c_double),
        ("t0", c_double), ("width", c_double), ("t1", c_double), ("n_det", c_int32),
        ("det_ij", POINTER(c_int32)), ("absorbing_faces", c_uint32), ("gamma_eps", c_double),
        ("gamma_sig", c_double), ("z_delta_frac", c_double), ("eps_max", c_double),
        ("sig_max", c_double), ("n_snapshots", c_int32), ("cfl_check", c_int32),
        ("mem_budget", c_int64), ("tile_kz", c_int32), ("forward_only", c_int32),
        ("mesh_n_new", c_int32), ("mesh_parents", POINTER(c_int32)), ("mesh_n_tets", c_int64),
        ("mesh_tets", POINTER(c_int32)), ("stream", c_void_p), ("grad_variant", c_int32),
        ("tile_kz_lean", c_int32),
    ]


class ddfd_info(ctypes.Structure):
    _fields_ = [
        ("n", c_int32), ("fem_n", c_int32), ("n_free", c_int32), ("n_det", c_int32),
        ("n_src", c_int32), ("n_steps", c_int32), ("a", c_int32), ("b", c_int32),
        ("switch_step", c_int32), ("h", c_double), ("tau", c_double),
        ("device_bytes", c_int64), ("kernel_launches", c_int64), ("forward_steps", c_int64),
        ("generation", c_int64),
    ]


class ddfd_timing(ctypes.Structure):
    _fields_ = [
        ("forward_loop_ms", c_double), ("adjoint_loop_ms", c_double),
        ("forward_step_kernels", c_int64), ("adjoint_step_kernels", c_int64),
    ]


class ddfd_batch_info(ctypes.Structure):
    _fields_ = [
        ("count", c_int32), ("tile_kz", c_int32),
        ("forward_loop_ms", c_double), ("adjoint_loop_ms", c_double),
        ("forward_step_kernels", c_int64), ("adjoint_step_kernels", c_int64),
        ("kernel_launches", c_int64), ("device_bytes", c_int64), ("tile_kz_lean", c_int32),
    ]


class ddfd_cg_params(ctypes.Structure):
    _fields_ = [
        ("max_iter", c_int32), ("gamma_eps0", c_double), ("gamma_sig0", c_double),
        ("alpha_eps0", c_double), ("alpha_sig0", c_double), ("p", c_double),
        ("eta1_eps", c_double), ("eta1_sig", c_double), ("eta2_eps", c_double),
        ("eta2_sig", c_double), ("eps_max", c_double), ("sig_max", c_double), ("restart", c_int32),
    ]


class ddfd_cg_iter(ctypes.Structure):
    _fields_ = [
        ("iter", c_int32), ("stop", c_int32), ("J", c_double), ("J_data", c_double),
        ("gnorm_eps", c_double), ("gnorm_sig", c_double), ("alpha_eps", c_double),
        ("alpha_sig", c_double), ("beta_eps", c_double), ("beta_sig", c_double),
        ("gamma_eps", c_double), ("gamma_sig", c_double), ("step_eps", c_double),
        ("step_sig", c_double), ("ms", c_double),
    ]


class DDFDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libddfd.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_2508_07780_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    P = c_void_p
    dp = POINTER(c_double)
    lib.ddfd_config_default.argtypes = [POINTER(ddfd_config)]
    lib.ddfd_config_default.restype = None
    lib.ddfd_create.argtypes = [POINTER(ddfd_config), POINTER(c_void_p)]
    lib.ddfd_destroy.argtypes = [P]
    lib.ddfd_destroy.restype = None
    lib.ddfd_last_error.argtypes = [P]
    lib.ddfd_last_error.restype = c_char_p
    lib.ddfd_create_error.argtypes = []
    lib.ddfd_create_error.restype = c_char_p
    for name in ("ddfd_set_coeffs", "ddfd_set_coeffs_dev"):
        getattr(lib, name).argtypes = [P, P, P, P, P]
    for name in ("ddfd_forward", "ddfd_forward_dev"):
        getattr(lib, name).argtypes = [P, P]
    for name in ("ddfd_functional", "ddfd_functional_dev"):
        getattr(lib, name).argtypes = [P, P, dp]
    for name in ("ddfd_adjoint", "ddfd_adjoint_dev"):
        getattr(lib, name).argtypes = [P, P]
    for name in ("ddfd_gradient", "ddfd_gradient_dev"):
        getattr(lib, name).argtypes = [P, P, P]
    lib.ddfd_get_info.argtypes = [P, POINTER(ddfd_info)]
    lib.ddfd_get_timing.argtypes = [P, POINTER(ddfd_timing)]
    lib.ddfd_misfit_noalloc.argtypes = [P, P, c_int32, c_int32, c_int32, c_double, c_double, P, P]
    lib.ddfd_set_capture.argtypes = [P, c_int32, P]
    lib.ddfd_get_capture.argtypes = [P, c_int32, c_int32, P]
    lib.ddfd_autotune.argtypes = [P, c_int32, POINTER(c_int32)]
    lib.ddfd_create_batch.argtypes = [POINTER(ddfd_config), c_int32, POINTER(c_void_p)]
    lib.ddfd_destroy_batch.argtypes = [P]
    lib.ddfd_destroy_batch.restype = None
    lib.ddfd_batch_last_error.argtypes = [P]
    lib.ddfd_batch_last_error.restype = c_char_p
    lib.ddfd_batch_member.argtypes = [P, c_int32, POINTER(c_void_p)]
    for name in ("ddfd_batch_forward", "ddfd_batch_forward_dev", "ddfd_batch_adjoint",
                 "ddfd_batch_adjoint_dev"):
        getattr(lib, name).argtypes = [P, P]
    lib.ddfd_batch_autotune.argtypes = [P, c_int32, POINTER(c_int32)]
    lib.ddfd_batch_get_info.argtypes = [P, POINTER(ddfd_batch_info)]
    lib.ddfd_test_gather_timeout.argtypes = [P, c_int32, ctypes.c_uint32]
    lib.ddfd_test_step_items.argtypes = [c_int32, c_int32, c_int32, POINTER(c_int32), c_int32, c_int32,
                                         POINTER(ctypes.c_uint32), c_int64, POINTER(c_int64), POINTER(c_int64)]
    lib.ddfd_time_gather.argtypes = [P, c_int32, P, P, P, P]
    lib.ddfd_cg_params_default.argtypes = [POINTER(ddfd_cg_params)]
    lib.ddfd_cg_params_default.restype = None
    lib.ddfd_cg_run.argtypes = [P, P, POINTER(ddfd_cg_params), P, P, POINTER(ddfd_cg_iter), POINTER(c_int32),
                                P, P]
    for name in ABI_SYMBOLS:
        if name not in ("ddfd_config_default", "ddfd_destroy", "ddfd_last_error",
                        "ddfd_create_error", "ddfd_destroy_batch", "ddfd_batch_last_error",
                        "ddfd_cg_params_default"):
            getattr(lib, name).restype = c_int
    _lib = lib
    return lib


def _ptr(a):
    """Host numpy array or torch tensor -> void pointer (None stays NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(c_void_p)
    return c_void_p(a.data_ptr())


def _host(a, dtype, count=None):
    arr = np.ascontiguousarray(a, dtype=dtype)
    if count is not None and arr.size != count:
        raise ValueError(f"expected {count} values, got {arr.size}")
    return arr


def _dev(t, count=None):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous()):
        raise TypeError("device arguments must be contiguous float64 CUDA tensors")
    if count is not None and t.numel() != count:
        raise ValueError(f"expected {count} values, got {t.numel()}")
    return t


def misfit_noalloc(trace, eobs, n_src, n_steps, n_det, tau, z_delta_frac, J, stream=None):
    """ddfd_misfit_noalloc on device tensors (float64 CUDA): writes the misfit
    to J[0] asynchronously on `stream` (a cudaStream_t handle or None).  For
    callers that cannot allocate device memory: no handle, no allocation."""
    lib = load_library()
    for t in (trace, eobs):
        if t is not None:
            _dev(t)
    _dev(J, 1)
    st = lib.ddfd_misfit_noalloc(_ptr(trace), _ptr(eobs), n_src, n_steps, n_det, tau, z_delta_frac,
                                 _ptr(J), c_void_p(stream) if stream else None)
    if st != DDFD_OK:
        raise DDFDError(st, lib.ddfd_create_error().decode())


def step_items(n, precision, boxes, kz, kz_lean):
    """ddfd_test_step_items (host only): the dispatch items of one step launch
    over len(boxes) problems of n^3 nodes, boxes = [(a, b, f0, nf), ...].
    Returns (items as a uint32 array, n_full)."""
    lib = load_library()
    prec = {"fp64": DDFD_FP64, "fp32": DDFD_FP32}[precision]
    bx = np.ascontiguousarray(np.asarray(boxes, dtype=np.int32).reshape(-1))
    ni, nf = c_int64(), c_int64()
    args = (int(n), prec, len(boxes), bx.ctypes.data_as(POINTER(c_int32)), int(kz), int(kz_lean))
    st = lib.ddfd_test_step_items(*args, None, 0, ctypes.byref(ni), ctypes.byref(nf))
    if st != DDFD_OK:
        raise DDFDError(st, "ddfd_test_step_items rejected its arguments")
    out = np.zeros(ni.value, dtype=np.uint32)
    st = lib.ddfd_test_step_items(*args, out.ctypes.data_as(POINTER(ctypes.c_uint32)), ni.value,
                                  ctypes.byref(ni), ctypes.byref(nf))
    if st != DDFD_OK:
        raise DDFDError(st, "ddfd_test_step_items rejected its arguments")
    return out, nf.value


def make_config(lib, kw, keep):
    """ddfd_config from keyword arguments (config field names; src_dir and
    det_ij as arrays, precision as "fp32"/"fp64" or the enum, stream as an
    integer handle).  Arrays the struct points to are appended to keep."""
    cfg = ddfd_config()
    lib.ddfd_config_default(ctypes.byref(cfg))
    for k, v in kw.items():
        if k == "src_dir":
            if v is not None:
                arr = _host(v, np.float64).reshape(-1, 3)
                keep.append(arr)
                cfg.src_dir = arr.ctypes.data_as(POINTER(c_double))
                cfg.n_src = arr.shape[0]
        elif k == "det_ij":
            arr = _host(v, np.int32).reshape(-1, 2)
            keep.append(arr)
            cfg.det_ij = arr.ctypes.data_as(POINTER(c_int32))
            cfg.n_det = arr.shape[0]
        elif k == "mesh":
            # (parents [E][2], tets [T][4]): an explicit refined FEM mesh
            par = _host(v[0], np.int32).reshape(-1, 2)
            tet = _host(v[1], np.int32).reshape(-1, 4)
            keep += [par, tet]
            cfg.fem_kind = DDFD_FEM_MESH
            cfg.mesh_n_new = par.shape[0]
            cfg.mesh_parents = par.ctypes.data_as(POINTER(c_int32))
            cfg.mesh_n_tets = tet.shape[0]
            cfg.mesh_tets = tet.ctypes.data_as(POINTER(c_int32))
        elif k == "stream":
            cfg.stream = c_void_p(v)
        elif k == "precision" and isinstance(v, str):
            cfg.precision = DDFD_FP32 if v == "fp32" else DDFD_FP64
        elif k == "grad_variant" and isinstance(v, str):
            cfg.grad_variant = {"exact": 0, "literal": 1}[v]
        else:
            setattr(cfg, k, v)
    return cfg


class Problem:
    """One ddfd handle.  Keyword arguments are ddfd_config fields; src_dir and
    det_ij are arrays ([n_src][3] floats, [n_det][2] ints)."""

    def __init__(self, **kw):
        lib = load_library()
        self._lib = lib
        self._keep = []
        cfg = make_config(lib, kw, self._keep)
        self.cfg = cfg
        h = c_void_p()
        st = lib.ddfd_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != DDFD_OK:
            raise DDFDError(st, lib.ddfd_create_error().decode())
        self._h = h
        self._owned = True
        self.info = self.get_info()

    @classmethod
    def _member(cls, lib, handle, batch):
        """A batch member: a handle the batch owns (close() does nothing)."""
        self = cls.__new__(cls)
        self._lib = lib
        self._keep = []
        self._h = handle
        self._owned = False
        self._batch = batch
        self.info = self.get_info()
        return self

    def autotune(self, steps=8):
        kz = c_int32()
        self._check(self._lib.ddfd_autotune(self._h, steps, ctypes.byref(kz)))
        return kz.value

    # -- helpers -------------------------------------------------------------
    def _check(self, st):
        if st != DDFD_OK:
            raise DDFDError(st, self._lib.ddfd_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            if self._owned:
                self._lib.ddfd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def n_free(self):
        return self.info.n_free

    @property
    def trace_shape(self):
        i = self.info
        return (i.n_src, i.n_steps + 1, i.n_det, 3)

    def get_info(self):
        inf = ddfd_info()
        self._check(self._lib.ddfd_get_info(self._h, ctypes.byref(inf)))
        return inf

    def get_timing(self):
        t = ddfd_timing()
        self._check(self._lib.ddfd_get_timing(self._h, ctypes.byref(t)))
        return t

    # -- host entry points ------------------------------------------------------
    def set_coeffs(self, eps, sig, eps0=None, sig0=None):
        nf = self.n_free
        a = [_host(x, np.float64, nf) if x is not None else None for x in (eps, sig, eps0, sig0)]
        self._check(self._lib.ddfd_set_coeffs(self._h, *[_ptr(x) for x in a]))

    def forward(self, want_trace=True):
        out = np.empty(self.trace_shape) if want_trace else None
        self._check(self._lib.ddfd_forward(self._h, _ptr(out)))
        return out

    def functional(self, eobs):
        e = _host(eobs, np.float64, int(np.prod(self.trace_shape)))
        J = c_double()
        self._check(self._lib.ddfd_functional(self._h, _ptr(e), ctypes.byref(J)))
        return J.value

    def adjoint(self, eobs):
        e = _host(eobs, np.float64, int(np.prod(self.trace_shape)))
        self._check(self._lib.ddfd_adjoint(self._h, _ptr(e)))

    def gradient(self):
        ge = np.empty(self.n_free)
        gs = np.empty(self.n_free)
        self._check(self._lib.ddfd_gradient(self._h, _ptr(ge), _ptr(gs)))
        return ge, gs

    # -- device entry points (torch float64 CUDA tensors) ------------------------
    def set_coeffs_dev(self, eps, sig, eps0=None, sig0=None):
        nf = self.n_free
        a = [_dev(x, nf) if x is not None else None for x in (eps, sig, eps0, sig0)]
        self._check(self._lib.ddfd_set_coeffs_dev(self._h, *[_ptr(x) for x in a]))

    def forward_dev(self, trace_out=None):
        if trace_out is not None:
            _dev(trace_out, int(np.prod(self.trace_shape)))
        self._check(self._lib.ddfd_forward_dev(self._h, _ptr(trace_out)))
        return trace_out

    def functional_dev(self, eobs):
        _dev(eobs, int(np.prod(self.trace_shape)))
        J = c_double()
        self._check(self._lib.ddfd_functional_dev(self._h, _ptr(eobs), ctypes.byref(J)))
        return J.value

    def adjoint_dev(self, eobs):
        _dev(eobs, int(np.prod(self.trace_shape)))
        self._check(self._lib.ddfd_adjoint_dev(self._h, _ptr(eobs)))

    def gradient_dev(self, g_eps, g_sig):
        _dev(g_eps, self.n_free)
        _dev(g_sig, self.n_free)
        self._check(self._lib.ddfd_gradient_dev(self._h, _ptr(g_eps), _ptr(g_sig)))

    # -- test hooks -------------------------------------------------------------
    def time_gather(self, reps=20):
        """ddfd_time_gather: (forward ms, adjoint ms, forward bytes, adjoint
        bytes) of one step's element-apply launches."""
        f, a = c_double(), c_double()
        fb, ab = ctypes.c_int64(), ctypes.c_int64()
        self._check(self._lib.ddfd_time_gather(self._h, int(reps), ctypes.byref(f), ctypes.byref(a),
                                               ctypes.byref(fb), ctypes.byref(ab)))
        return f.value, a.value, fb.value, ab.value

    def test_gather_timeout(self, fault, spin_limit=0):
        """ddfd_test_gather_timeout: fault=1 makes the element gather's first
        bounded wait run out (the next forward/adjoint fails with
        DDFD_E_TIMEOUT); fault=0 restores normal operation."""
        self._check(self._lib.ddfd_test_gather_timeout(self._h, int(fault), int(spin_limit)))

    def set_capture(self, steps):
        arr = _host(list(steps), np.int32)
        self._check(self._lib.ddfd_set_capture(self._h, len(arr), _ptr(arr) if len(arr) else None))
        self._cap = list(int(s) for s in arr)

    def get_capture(self, kind, idx):
        n = self.info.n
        out = np.empty(3 * n ** 3)
        self._check(self._lib.ddfd_get_capture(self._h, kind, idx, _ptr(out)))
        return out.reshape(3, n ** 3)


class Batch:
    """ddfd_batch: problems with the same grid, step count and precision,
    stepped together (one launch per time step for up to 16 members).
    ``configs`` is a list of keyword dicts as for ``Problem``; ``members``
    are Problem views of the batch's handles (set_coeffs, functional and
    gradient per member)."""

    def __init__(self, configs):
        lib = load_library()
        self._lib = lib
        self._keep = []
        arr = (ddfd_config * len(configs))()
        for i, kw in enumerate(configs):
            arr[i] = make_config(lib, kw, self._keep)
        h = c_void_p()
        st = lib.ddfd_create_batch(arr, len(configs), ctypes.byref(h))
        if st != DDFD_OK:
            raise DDFDError(st, lib.ddfd_create_error().decode())
        self._h = h
        self.members = []
        for i in range(len(configs)):
            m = c_void_p()
            self._check(lib.ddfd_batch_member(h, i, ctypes.byref(m)))
            self.members.append(Problem._member(lib, m, self))

    def _check(self, st):
        if st != DDFD_OK:
            raise DDFDError(st, self._lib.ddfd_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            for m in self.members:
                m._h = None
            self._lib.ddfd_destroy_batch(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __len__(self):
        return len(self.members)

    def get_info(self):
        inf = ddfd_batch_info()
        self._check(self._lib.ddfd_batch_get_info(self._h, ctypes.byref(inf)))
        return inf

    def autotune(self, steps=8):
        kz = c_int32()
        self._check(self._lib.ddfd_batch_autotune(self._h, steps, ctypes.byref(kz)))
        return kz.value

    def forward(self, want_trace=True):
        """Batched forward; returns the members' traces (host) or None."""
        outs = [np.empty(m.trace_shape) for m in self.members] if want_trace else None
        ptrs = (c_void_p * len(self.members))(*[o.ctypes.data for o in outs]) if outs else None
        self._check(self._lib.ddfd_batch_forward(self._h, ptrs))
        return outs

    def adjoint(self, eobs):
        es = [_host(e, np.float64, int(np.prod(m.trace_shape))) for e, m in zip(eobs, self.members)]
        ptrs = (c_void_p * len(es))(*[e.ctypes.data for e in es])
        self._check(self._lib.ddfd_batch_adjoint(self._h, ptrs))

    def forward_dev(self, trace_out=None):
        """trace_out: None or one float64 CUDA tensor (or None) per member."""
        ptrs = None
        if trace_out is not None:
            for t, m in zip(trace_out, self.members):
                if t is not None:
                    _dev(t, int(np.prod(m.trace_shape)))
            ptrs = (c_void_p * len(trace_out))(*[t.data_ptr() if t is not None else None
                                                 for t in trace_out])
        self._check(self._lib.ddfd_batch_forward_dev(self._h, ptrs))
        return trace_out

    def adjoint_dev(self, eobs):
        for e, m in zip(eobs, self.members):
            _dev(e, int(np.prod(m.trace_shape)))
        ptrs = (c_void_p * len(eobs))(*[e.data_ptr() for e in eobs])
        self._check(self._lib.ddfd_batch_adjoint_dev(self._h, ptrs))

    def cg_run(self, eobs, eps0, sig0, iterates=False, **params):
        """ddfd_cg_run: the CGA of Sec. 4 over the members (one model, several
        measurements).  eobs: one observed trace per member (host); eps0, sig0:
        initial guess on the free nodes; params: ddfd_cg_params fields.
        Returns (eps, sig, log) with log a list of dicts, one per iteration
        (with iterates=True each dict also holds that iteration's new eps, sig).
        A failed iteration raises DDFDError carrying .log (the iterations
        before it) and .eps, .sig (the iterate whose evaluation failed)."""
        prm = ddfd_cg_params()
        self._lib.ddfd_cg_params_default(ctypes.byref(prm))
        for k, v in params.items():
            setattr(prm, k, v)
        nf = self.members[0].n_free
        eps = _host(eps0, np.float64, nf).copy()
        sig = _host(sig0, np.float64, nf).copy()
        es = [_host(e, np.float64, int(np.prod(m.trace_shape))) for e, m in zip(eobs, self.members)]
        ptrs = (c_void_p * len(es))(*[e.ctypes.data for e in es])
        log = (ddfd_cg_iter * prm.max_iter)()
        iters = c_int32()
        ei = np.empty((prm.max_iter, nf)) if iterates else None
        si = np.empty((prm.max_iter, nf)) if iterates else None
        st = self._lib.ddfd_cg_run(self._h, ptrs, ctypes.byref(prm), _ptr(eps), _ptr(sig), log,
                                   ctypes.byref(iters), _ptr(ei), _ptr(si))
        out = [{f: getattr(log[i], f) for f, _ in ddfd_cg_iter._fields_} for i in range(iters.value)]
        if iterates:
            for i, r in enumerate(out):
                r["eps"], r["sig"] = ei[i], si[i]
        try:
            self._check(st)
        except DDFDError as e:
            e.log, e.eps, e.sig = out, eps, sig
            raise
        return eps, sig, out
