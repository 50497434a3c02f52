"""ctypes view of libfdl.so (include/fdl.h).

Loading fails loudly when the library is missing: there is no fallback.
"""

from __future__ import annotations

import ctypes as ct
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfdl.so")

FDL_OK, FDL_EINVAL, FDL_ENOMEM, FDL_ECUDA, FDL_ETIMEOUT, FDL_ENOTSUP = range(6)
# bits of the device status word (fdl_sync_status)
ST_NONFINITE, ST_BREAKDOWN, ST_BAD_REQUEST = 1, 2, 4
REG = {"view2": 0, "layer2": 1, "l2": 2}
PREC = {"mixed": 0, "df": 1, "f64": 2, "f32": 3}
APERTURE = {"pinhole": 0, "disc": 1, "square": 2, "points": 3, "table": 4}


class FitOpts(ct.Structure):
    _fields_ = [("lam", ct.c_double), ("eps", ct.c_double), ("reg", ct.c_int), ("precision", ct.c_int),
                ("kappa_max", ct.c_double), ("df_error_budget", ct.c_double),
                ("f32_error_budget", ct.c_double)]


class Request(ct.Structure):
    """Mirror of ``fdl_request``."""

    _fields_ = [("layers", ct.c_void_p), ("d", ct.c_void_p), ("out", ct.c_void_p), ("pts", ct.c_void_p),
                ("N", ct.c_int), ("npts", ct.c_int), ("aperture", ct.c_int), ("u0x", ct.c_float),
                ("u0y", ct.c_float), ("s", ct.c_float), ("radius", ct.c_float), ("H", ct.c_int), ("W", ct.c_int),
                ("C", ct.c_int), ("pad_", ct.c_int * 2)]


class FdlError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {status_name(status)} (status {status})")
        self.status = status


_lib = None

# (name, restype, argtypes)
class System(ct.Structure):
    """fdl_system: device pointers (0 for NULL)."""
    _fields_ = [("u", ct.c_void_p), ("d", ct.c_void_p), ("P", ct.c_void_p), ("views", ct.c_void_p)]


_SIGS = [
    ("fdl_strerror", ct.c_char_p, [ct.c_int]),
    ("fdl_version", ct.c_int, []),
    ("fdl_rfft2_workspace_size", ct.c_size_t, [ct.c_int] * 3),
    ("fdl_rfft2", ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_size_t,
                             ct.c_void_p]),
    ("fdl_irfft2_workspace_size", ct.c_size_t, [ct.c_int] * 3),
    ("fdl_irfft2", ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_size_t,
                              ct.c_void_p]),
    ("fdl_fit_workspace_size", ct.c_size_t, [ct.c_int] * 5),
    ("fdl_fit", ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_int,
                           ct.POINTER(FitOpts), ct.c_void_p, ct.c_void_p, ct.c_size_t, ct.c_void_p]),
    ("fdl_fit_spectra_workspace_size", ct.c_size_t, [ct.c_int] * 5),
    ("fdl_fit_spectra", ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p,
                                   ct.c_int, ct.POINTER(FitOpts), ct.c_void_p, ct.c_void_p, ct.c_size_t,
                                   ct.c_void_p]),
    ("fdl_fit_spectra_noalloc", ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_void_p,
                                           ct.c_void_p, ct.c_int, ct.POINTER(FitOpts), ct.c_void_p, ct.c_void_p]),
    ("fdl_fit_tier_counts", ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int), ct.c_void_p]),
    ("fdl_sync_status", ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int), ct.c_void_p]),
    ("fdl_fit_render_host_workspace_size", ct.c_size_t, [ct.c_int] * 6),
    ("fdl_fit_render_host", ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p,
                                       ct.c_int, ct.POINTER(FitOpts), ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_void_p,
                                       ct.c_size_t, ct.c_void_p, ct.c_void_p, ct.c_size_t, ct.c_void_p]),
    ("fdl_render_workspace_size", ct.c_size_t, [ct.c_int] * 4),
    ("fdl_render", ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_void_p,
                              ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_size_t, ct.c_void_p]),
    ("fdl_refocus_workspace_size", ct.c_size_t, [ct.c_int] * 4),
    ("fdl_aperture_table_workspace_size", ct.c_size_t, [ct.c_int] * 2),
    ("fdl_fit_general_workspace_size", ct.c_size_t, [ct.c_int] * 5),
    ("fdl_fit_general", ct.c_int, [ct.c_void_p] + [ct.c_int] * 5 + [ct.POINTER(System), ct.POINTER(FitOpts),
                                                                   ct.c_void_p, ct.c_void_p, ct.c_size_t,
                                                                   ct.c_void_p]),
    ("fdl_render_shifts_workspace_size", ct.c_size_t, [ct.c_int] * 4),
    ("fdl_render_shifts", ct.c_int, [ct.c_void_p, ct.c_void_p] + [ct.c_int] * 5 + [ct.c_void_p, ct.c_void_p,
                                                                                    ct.c_size_t, ct.c_void_p]),
    ("fdl_calib_grad_shifts_workspace_size", ct.c_size_t, [ct.c_int] * 6),
    ("fdl_calib_grad_shifts", ct.c_int, [ct.c_void_p] + [ct.c_int] * 4 + [ct.c_void_p, ct.c_int, ct.POINTER(FitOpts),
                                                                          ct.c_void_p, ct.c_int, ct.c_void_p,
                                                                          ct.c_void_p, ct.c_void_p, ct.c_size_t,
                                                                          ct.c_void_p]),
    ("fdl_aperture_table", ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_size_t,
                                      ct.c_void_p]),
    ("fdl_refocus", ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_int,
                               ct.c_void_p, ct.c_size_t, ct.c_void_p]),
    ("fdl_calib_grad_workspace_size", ct.c_size_t, [ct.c_int] * 6),
    ("fdl_calib_grad", ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p,
                                  ct.c_int, ct.POINTER(FitOpts), ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p,
                                  ct.c_void_p, ct.c_void_p, ct.c_size_t, ct.c_void_p]),
]


def load(path: str | None = None):
    """Load libfdl.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libfdl.so is missing at {path}: build it with "
                           "`python -m paper_1901_06919_gb300.build` (there is no CPU fallback)")
    lib = ct.CDLL(path)
    for name, res, args in _SIGS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_name(status: int) -> str:
    names = {0: "FDL_OK", 1: "FDL_EINVAL", 2: "FDL_ENOMEM", 3: "FDL_ECUDA", 4: "FDL_ETIMEOUT", 5: "FDL_ENOTSUP"}
    return names.get(status, "unknown")


def check(status: int, where: str) -> None:
    if status != FDL_OK:
        raise FdlError(status, where)


def exported_symbols() -> list[str]:
    return [s[0] for s in _SIGS]
