"""ctypes declarations of libgslens (include/gslens.h).  Loading fails loudly
if the library cannot be built or loaded: there is no fallback path."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

_lib = None

# argument type shorthands
_i32, _i64, _u32, _f64, _vp = ctypes.c_int, ctypes.c_int64, ctypes.c_uint, ctypes.c_double, ctypes.c_void_p

EXPORTS = {
    # name: (restype, argtypes)
    "lens_plan_create": (_i32, [ctypes.POINTER(_vp), _i32, _i32, _i32, _i64, _vp, _vp, _vp, _f64, _i32, _u32, _vp]),
    "lens_plan_create_ex": (_i32, [ctypes.POINTER(_vp), _i32, _i32, _i32, _i64, _vp, _vp, _vp, _f64, _i32, _u32,
                                   _vp, _vp]),
    "lens_plan_destroy": (_i32, [_vp]),
    "lens_plan_info": (_i32, [_vp, _vp]),
    "lens_plan_set_grouping": (_i32, [_vp, _i32]),
    "lens_plan_set_tensor_cores": (_i32, [_vp, _i32]),
    "lens_plan_status": (_i32, [_vp, _vp]),
    "lens_torus_coefficients": (_i32, [_vp, _vp, _vp, _vp]),
    "lens_selftest_bounded_wait": (_i32, [_vp]),
    "lens_synthesis": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "lens_adjoint": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "lens_synthesis_vjp": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "lens_adjoint_vjp": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "lens_deflection": (_i32, [_vp, _vp, _vp, _vp]),
    "lens_alm_eth": (_i32, [_i32, _i32, _i32, _i32, _i32, _vp, _vp, _vp]),
    "lens_phi_gradient": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "lens_batch_create": (_i32, [ctypes.POINTER(_vp), _i32]),
    "lens_batch_add": (_i32, [_vp, _vp, _i32, _vp, _vp, _i32]),
    "lens_batch_instantiate": (_i32, [_vp, _i32]),
    "lens_batch_launch": (_i32, [_vp, _vp]),
    "lens_batch_info": (_i32, [_vp, _vp, _vp, _vp]),
    "lens_batch_destroy": (_i32, [_vp]),
    "lens_autotune": (_i32, [_i32, _i32, _i32, _i64, _vp, _vp, _vp, _f64, _i32, _vp, _i32, _vp, _vp]),
    "lens_gl_grid": (_i32, [_i32, _i32, _vp, _vp, _vp, _vp]),
    "lens_scale_points": (_i32, [_i64, _i32, _i32, _vp, _vp, _vp, _vp]),
    "lens_magnification": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "lens_synthesis_host": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "lens_adjoint_host": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "lens_synthesis_host_async": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "lens_adjoint_host_async": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "lens_synthesis_static": (_i32, [_vp, _vp, _vp, _vp]),
    "lens_measure_fma_peak": (_i32, [_i32, _vp, _vp]),
    "lens_ring_synthesis": (_i32, [_vp, _vp, _vp, _vp]),
    "lens_ring_adjoint": (_i32, [_vp, _vp, _vp, _vp]),
    "lens_pointing": (_i32, [_i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "lens_profile_enable": (_i32, [_i32]),
    "lens_profile_read": (_i32, [_vp, _vp, _i32]),
    "lens_profile_reset": (_i32, []),
    "lens_nalm": (_i64, [_i32, _i32]),
    "lens_kernel_poly": (_i32, [_i32, _f64, _vp]),
    "lens_status_string": (ctypes.c_char_p, [_i32]),
    "lens_get_last_error": (_i32, []),
    "lens_last_error_message": (ctypes.c_char_p, []),
    "lens_version": (_i32, []),
}


class PlanParams(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("W", ctypes.c_int), ("beta", ctypes.c_double),
                ("ntheta", ctypes.c_int), ("legendre_rpt_fwd", ctypes.c_int), ("legendre_rpt_adj", ctypes.c_int),
                ("legendre_df32_mmin", ctypes.c_int), ("fft_cluster", ctypes.c_int), ("legendre_tables", ctypes.c_int),
                ("legendre_restart", ctypes.c_int), ("point_weights", ctypes.c_int),
                ("spread_tile_rows", ctypes.c_int)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("lmax", ctypes.c_int), ("mmax", ctypes.c_int), ("spin", ctypes.c_int), ("prec", ctypes.c_int),
                ("npoints", ctypes.c_int64), ("epsilon", ctypes.c_double), ("ntheta", ctypes.c_int),
                ("ntheta_fft", ctypes.c_int), ("n1", ctypes.c_int), ("n2", ctypes.c_int), ("W", ctypes.c_int),
                ("beta", ctypes.c_double), ("sigma", ctypes.c_double), ("rows_kept", ctypes.c_int),
                ("row_pitch", ctypes.c_int), ("workspace_bytes", ctypes.c_size_t),
                ("plan_bytes", ctypes.c_size_t), ("flags", ctypes.c_uint), ("alm_ncomp", ctypes.c_int),
                ("legendre_table_bytes", ctypes.c_size_t), ("legendre_restart", ctypes.c_int),
                ("restart_bytes", ctypes.c_size_t), ("legendre_df32_mmin", ctypes.c_int),
                ("legendre_triples", ctypes.c_int64), ("point_weight_bytes", ctypes.c_size_t)]


def lib_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libgslens.so (building it from csrc/ first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libgslens.so is missing; run `python -m paper_2304_10431_gb300.build`")
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class LensError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (status %d)" % (msg, status))
        self.status = status


def check(status: int):
    if status != 0:
        lib = load()
        msg = lib.lens_last_error_message().decode() or lib.lens_status_string(status).decode()
        raise LensError(status, msg)
