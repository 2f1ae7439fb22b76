"""ctypes declarations for libccm.so (mirrors include/ccm.h)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
Q_INF = 2147483647  # CCM_Q_INF: the int32 q that selects the max norm
_LIB = None

PREC_FP64, PREC_MIXED = 0, 1
ENGINE_AUTO, ENGINE_GRID, ENGINE_BLOCK = 0, 1, 2

STATUS = {
    0: "CCM_OK", 1: "CCM_ERR_INVALID_ARG", 2: "CCM_ERR_UNSUPPORTED", 3: "CCM_ERR_CUDA",
    4: "CCM_ERR_OOM", 5: "CCM_ERR_NOT_CONVERGED", 6: "CCM_ERR_TIMEOUT",
    7: "CCM_ERR_BUFFER_TOO_SMALL", 8: "CCM_ERR_BOUNDS",
}


class CCMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(C.Structure):
    _fields_ = [
        ("sigma0", C.c_double), ("sigma_max", C.c_double),
        ("max_outer", C.c_int32), ("max_newton", C.c_int32), ("max_cg", C.c_int32),
        ("precision", C.c_int32), ("engine", C.c_int32), ("profile", C.c_int32),
        ("relabel", C.c_int32), ("autotune", C.c_int32), ("coarse", C.c_int32),
        ("X0", C.c_void_p), ("U0", C.c_void_p),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("outer", C.c_int32), ("newton", C.c_int32), ("cg", C.c_int32),
        ("line_search", C.c_int32), ("n_clusters", C.c_int32),
        ("kkt", C.c_double), ("eta_d", C.c_double), ("eta_p", C.c_double), ("gap", C.c_double),
        ("f_p", C.c_double), ("f_d", C.c_double), ("sigma", C.c_double),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class Profile(C.Structure):
    _fields_ = [("matvec_launches", C.c_int64), ("matvec_ms_total", C.c_double),
                ("matvec_bytes_total", C.c_double), ("kernel_launches", C.c_int64),
                ("block_lanes", C.c_int32), ("block_quads", C.c_int32),
                ("coarse_steps", C.c_int32), ("coarse_max_aggregates", C.c_int32)]


class GraphInfo(C.Structure):
    _fields_ = [("candidates", C.c_int32), ("per_row", C.c_int32),
                ("rows_exhaustive", C.c_int64)]


class Problem(C.Structure):
    _fields_ = [("A", C.c_void_p), ("edges", C.c_void_p), ("w", C.c_void_p),
                ("n", C.c_int64), ("m", C.c_int64), ("X", C.c_void_p), ("labels", C.c_void_p)]


_P = C.c_void_p
_SIGS = {
    "ccm_default_options": (None, [C.POINTER(Options)]),
    "ccm_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int]),
    "ccm_destroy": (None, [_P]),
    "ccm_last_error": (C.c_char_p, []),
    "ccm_max_dim": (C.c_int32, []),
    "ccm_build_graph": (C.c_int, [_P, _P, C.c_int64, C.c_int32, C.c_int32, C.c_double, _P, _P,
                                  C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_double), _P]),
    "ccm_solve_path": (C.c_int, [_P, _P, C.c_int64, C.c_int32, _P, _P, C.c_int64,
                                 C.POINTER(C.c_double), C.c_int32, C.c_int32, C.c_double,
                                 C.POINTER(Options), _P, _P, _P, C.POINTER(Stats), _P]),
    "ccm_solve_path_admm": (C.c_int, [_P, _P, C.c_int64, C.c_int32, _P, _P, C.c_int64,
                                      C.POINTER(C.c_double), C.c_int32, C.c_int32, C.c_double,
                                      C.POINTER(Options), _P, _P, _P, C.POINTER(Stats), _P]),
    "ccm_solve_path_ama": (C.c_int, [_P, _P, C.c_int64, C.c_int32, _P, _P, C.c_int64,
                                     C.POINTER(C.c_double), C.c_int32, C.c_int32, C.c_double,
                                     C.POINTER(Options), _P, _P, _P, C.POINTER(Stats), _P]),
    "ccm_last_profile": (C.c_int, [_P, C.POINTER(Profile)]),
    "ccm_last_graph_info": (C.c_int, [_P, C.POINTER(GraphInfo)]),
    "ccm_launch_count": (C.c_int64, [_P]),
    "ccm_labels": (C.c_int, [_P, _P, C.c_int64, C.c_int32, _P, C.c_int64, _P,
                             C.POINTER(C.c_int32), _P]),
    "ccm_path_vjp": (C.c_int, [_P, _P, C.c_int64, C.c_int32, _P, _P, C.c_int64,
                               C.POINTER(C.c_double), C.c_int32, _P, _P, _P, _P, _P, _P]),
    "ccm_solve_path_batched": (C.c_int, [_P, C.c_int32, C.POINTER(Problem), C.c_int32,
                                         C.POINTER(C.c_double), C.c_int32, C.c_double,
                                         C.POINTER(Options), C.POINTER(Stats), _P]),
}


def lib_path() -> str:
    """The library to load: libccm.so next to this file, or the file named by the
    CCM_LIBRARY environment variable (for example the bounds-checked build
    libccm_debug.so)."""
    return os.environ.get("CCM_LIBRARY") or os.path.join(HERE, "libccm.so")


def debug_lib_path() -> str:
    """The bounds-checked build (compiled with CCM_DEBUG_BOUNDS)."""
    return os.path.join(HERE, "libccm_debug.so")


def load_library():
    """Load libccm.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build it with `python -m paper_2501_15964_b300.build`")
    try:  # share the CUDA runtime that PyTorch already loaded
        import torch  # noqa: F401
    except Exception:
        pass
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def exported_symbols():
    lib = load_library()
    return [n for n in _SIGS if hasattr(lib, n)]


def check(status: int):
    if status != 0:
        msg = load_library().ccm_last_error().decode()
        raise CCMError(status, msg)


class Context:
    """Owns a ccm_ctx (scratch memory) on one CUDA device."""

    def __init__(self, device: int = 0):
        lib = load_library()
        h = C.c_void_p()
        check(lib.ccm_create(C.byref(h), int(device)))
        self._h = h
        self.device = device

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load_library().ccm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
