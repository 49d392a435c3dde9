"""ctypes binding of liblx3c.so (argument marshalling only).

Every computation runs in the library's CUDA kernels; this module only loads
the shared library, declares the C signatures of include/lx3c.h and converts
arguments.  There is no CPU fallback: if the library cannot be loaded, every
call raises.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

c_i32p = ctypes.POINTER(ctypes.c_int32)
c_f64p = ctypes.POINTER(ctypes.c_double)
# int f(void* user, int64 row0, int64 nrow, int64 col0, int64 ncol, double* buf, int64 ld)
TILE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                           ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_int64)

EXPORTS = {
    # name: (restype, argtypes)
    "lx3c_last_error": (ctypes.c_char_p, []),
    "lx3c_version": (ctypes.c_char_p, []),
    "lx3c_basis_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "lx3c_basis_destroy": (None, [ctypes.c_void_p]),
    "lx3c_eri3c_plan": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_int, ctypes.c_void_p]),
    "lx3c_eri3c_execute": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "lx3c_plan_sizes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int64)]),
    "lx3c_plan_destroy": (None, [ctypes.c_void_p]),
    "lx3c_plan_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "lx3c_eri3c_host": (ctypes.c_int, [ctypes.c_int64] + [ctypes.c_void_p] * 5 + [ctypes.c_int64] +
                        [ctypes.c_void_p] * 5 + [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                                 ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "lx3c_boys": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "lx3c_fp64_rate": (ctypes.c_int, [ctypes.c_int64, c_f64p, c_f64p, ctypes.c_void_p]),
    "lx3c_class_flops": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, c_f64p]),
    "lx3c_solid_harmonics": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p]),
    "lx3c_eri3c_noalloc": (ctypes.c_int, [ctypes.c_int] * 7 + [ctypes.c_void_p] * 9 + [ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "lx3c_dfj_plan": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_void_p]),
    "lx3c_schwarz_pair": (ctypes.c_int, [ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 3 +
                          [ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 3 + [c_f64p]),
    "lx3c_schwarz_aux": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, c_f64p]),
    "lx3c_dfj_grad": (ctypes.c_int, [ctypes.c_void_p] * 5),
    "lx3c_dfj_energy": (ctypes.c_int, [ctypes.c_void_p] * 6),
    "lx3c_dfj_execute": (ctypes.c_int, [ctypes.c_void_p] * 6),
    "lx3c_dfj_execute_tiles": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, TILE_FN, TILE_FN, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "lx3c_dfj_execute_multi": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 5),
    "lx3c_dfj_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "lx3c_dfj_group": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 4),
    "lx3c_dfj_destroy": (None, [ctypes.c_void_p]),
    "lx3c_batch_plan": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_double, ctypes.c_char_p, ctypes.c_void_p]),
    "lx3c_batch_bind": (ctypes.c_int, [ctypes.c_void_p] * 6),
    "lx3c_batch_execute": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "lx3c_batch_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "lx3c_batch_destroy": (None, [ctypes.c_void_p]),
    "lx3c_metric_plan": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_void_p]),
    "lx3c_metric_execute": (ctypes.c_int, [ctypes.c_void_p] * 3),
    "lx3c_metric_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "lx3c_metric_destroy": (None, [ctypes.c_void_p]),
    "lx3c_cholesky": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                     ctypes.c_void_p, ctypes.c_void_p]),
    "lx3c_cholesky_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                           ctypes.c_int64, ctypes.c_void_p]),
    "lx3c_dfj_coulomb": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64] + [ctypes.c_void_p] * 5),
    "lx3c_cvrr2_expansion": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                            ctypes.POINTER(ctypes.c_int32)]),
    "lx3c_shape_hint": (ctypes.c_int, [ctypes.c_int] * 7),
    "lx3c_tile_hint": (ctypes.c_int, [ctypes.c_int] * 8),
    "lx3c_hrr_hint": (ctypes.c_int, [ctypes.c_int] * 5),
    "lx3c_hrr_tables_check": (ctypes.c_int, [ctypes.c_int] * 5 + [ctypes.c_void_p, c_f64p]),
    "lx3c_set_orientation_threshold": (ctypes.c_int, [ctypes.c_double]),
    "lx3c_set_compensation": (ctypes.c_int, [ctypes.c_int]),
    "lx3c_class_tables_check": (ctypes.c_int, [ctypes.c_int] * 4),
    "lx3c_shape_query": (ctypes.c_int, [ctypes.c_int] * 6 + [ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]),
}


class LibraryError(RuntimeError):
    pass


def lib_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load liblx3c.so (building it in-tree first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise LibraryError("liblx3c.so is not built (run paper_2210_03192_gb300.build.build())")
    L = ctypes.CDLL(_build.LIB)
    for name, (res, args) in EXPORTS.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(rc, what=""):
    if rc != 0:
        msg = load().lx3c_last_error()
        raise LibraryError("%s failed (status %d): %s" % (what, rc, msg.decode() if msg else ""))


def ptr(a):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()
