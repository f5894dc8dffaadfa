"""ctypes binding of the C ABI in include/cswgs.h: the same names, argument
marshalling only.  Every step of the method runs in libcswgs.so's CUDA
kernels; there is no Python or CPU fallback, and loading fails loudly when
the library cannot be built or found.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

CSWGS_OK, CSWGS_EINVAL, CSWGS_ENOMEM, CSWGS_ECUDA, CSWGS_ETIMEOUT, CSWGS_EBUSY, \
    CSWGS_ECANCELLED, CSWGS_ENOTFOUND = range(8)
CSWGS_FP64, CSWGS_FP32, CSWGS_FP32_FP16SINCOS = range(3)

c_double_p = ctypes.POINTER(ctypes.c_double)
c_float_p = ctypes.POINTER(ctypes.c_float)


class cswgs_plan_desc(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("max_P", ctypes.c_int), ("max_N", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("mem_cap_bytes", ctypes.c_size_t),
                ("precision", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("tune_cache", ctypes.c_char_p)]


CSWGS_APERTURE_SQUARE, CSWGS_APERTURE_ROUND = range(2)
CSWGS_SUBSET_FRESH, CSWGS_SUBSET_WINDOWS = range(2)
c_uint8_p = ctypes.POINTER(ctypes.c_uint8)


class cswgs_pupil(ctypes.Structure):
    _fields_ = [("aperture", ctypes.c_int), ("subset_mode", ctypes.c_int), ("beam_waist", ctypes.c_double)]


class cswgs_slm_frame(ctypes.Structure):
    _fields_ = [("frame", c_uint8_p), ("width", ctypes.c_int), ("height", ctypes.c_int),
                ("pitch", ctypes.c_int), ("offset_x", ctypes.c_int), ("offset_y", ctypes.c_int),
                ("lut", c_uint8_p), ("levels", ctypes.c_int)]


class cswgs_optics(ctypes.Structure):
    _fields_ = [("wavelength", ctypes.c_double), ("focal_length", ctypes.c_double),
                ("pixel_pitch", ctypes.c_double)]


class cswgs_solve_opts(ctypes.Structure):
    _fields_ = [("full_iterations", ctypes.c_int), ("first_iteration", ctypes.c_int),
                ("final_pass", ctypes.c_int), ("init_w", c_double_p), ("init_theta", c_double_p),
                ("final_w", c_double_p), ("final_theta", c_double_p),
                ("spot_intensity", c_double_p), ("pupil", cswgs_pupil),
                ("slm", ctypes.POINTER(cswgs_slm_frame))]


class cswgs_request(ctypes.Structure):
    # the data pointers are declared void* here (same size and place as the
    # header's const double* / float*): a batch of requests is filled with
    # plain addresses, without a ctypes cast per field
    _fields_ = [("spots_xyz", ctypes.c_void_p), ("amplitudes", ctypes.c_void_p), ("N", ctypes.c_int),
                ("P", ctypes.c_int), ("subset_fraction", ctypes.c_double),
                ("iterations", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("full_iterations", ctypes.c_int), ("phase_out", ctypes.c_void_p),
                ("out_on_host", ctypes.c_int), ("pupil", cswgs_pupil),
                ("slm", ctypes.POINTER(cswgs_slm_frame))]


class cswgs_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("e", ctypes.c_double), ("u", ctypes.c_double),
                ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double)]


class cswgs_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("cancelled", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("launches", ctypes.c_uint64), ("active", ctypes.c_int), ("queued", ctypes.c_int),
                ("bytes_in_use", ctypes.c_size_t), ("bytes_cap", ctypes.c_size_t),
                ("busy_ms", ctypes.c_double)]


# name -> (restype, argtypes)
_P = ctypes.c_void_p
SIGNATURES = {
    "cswgs_plan_desc_default": (None, [ctypes.POINTER(cswgs_plan_desc)]),
    "cswgs_plan_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(cswgs_plan_desc)]),
    "cswgs_plan_destroy": (ctypes.c_int, [_P]),
    "cswgs_solve": (ctypes.c_int, [_P, c_double_p, c_double_p, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_int, ctypes.c_uint64, c_float_p,
                                   ctypes.c_int, c_double_p, c_double_p]),
    "cswgs_solve_opts_default": (None, [ctypes.POINTER(cswgs_solve_opts)]),
    "cswgs_solve_ex": (ctypes.c_int, [_P, c_double_p, c_double_p, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_uint64,
                                      ctypes.POINTER(cswgs_solve_opts), c_float_p, ctypes.c_int,
                                      c_double_p, c_double_p]),
    "cswgs_subset": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int32)]),
    "cswgs_subset_ex": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_int,
                                       ctypes.POINTER(cswgs_pupil), ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_int64)]),
    "cswgs_batch_create": (ctypes.c_int, [_P, ctypes.POINTER(cswgs_request), ctypes.c_int,
                                          ctypes.POINTER(_P)]),
    "cswgs_batch_create_host": (ctypes.c_int, [_P, ctypes.POINTER(cswgs_request), ctypes.c_int,
                                               ctypes.POINTER(_P)]),
    "cswgs_batch_update": (ctypes.c_int, [_P, ctypes.POINTER(cswgs_request), ctypes.c_int]),
    "cswgs_batch_run": (ctypes.c_int, [_P]),
    "cswgs_batch_results": (ctypes.c_int, [_P, ctypes.POINTER(cswgs_result)]),
    "cswgs_batch_kernel_times": (ctypes.c_int, [_P, c_float_p, ctypes.c_int,
                                                ctypes.POINTER(ctypes.c_int)]),
    "cswgs_batch_pairs": (ctypes.c_int, [_P, c_double_p, c_double_p]),
    "cswgs_batch_tile_shape": (ctypes.c_int, [_P] + [ctypes.POINTER(ctypes.c_int)] * 5),
    "cswgs_batch_destroy": (ctypes.c_int, [_P]),
    "cswgs_solve_batch": (ctypes.c_int, [_P, ctypes.POINTER(cswgs_request), ctypes.c_int,
                                         ctypes.POINTER(cswgs_result)]),
    "cswgs_submit": (ctypes.c_int, [_P, ctypes.POINTER(cswgs_request), ctypes.POINTER(ctypes.c_uint64)]),
    "cswgs_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(cswgs_result)]),
    "cswgs_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(cswgs_result)]),
    "cswgs_cancel": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "cswgs_serve_stats_get": (ctypes.c_int, [_P, ctypes.POINTER(cswgs_serve_stats)]),
    "cswgs_autotune": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_double, c_double_p]),
    "cswgs_plan_test_waits": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_uint]),
    "cswgs_sincos_peak": (ctypes.c_int, [_P, c_double_p, c_double_p]),
    "cswgs_solve_noalloc": (ctypes.c_int, [c_double_p, c_double_p, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_int, ctypes.c_uint64, c_float_p, c_double_p, ctypes.c_void_p]),
    "cswgs_spots_from_physical": (ctypes.c_int, [ctypes.POINTER(cswgs_optics), c_double_p, ctypes.c_int, ctypes.c_int,
                                                 c_double_p]),
    "cswgs_abi_version": (ctypes.c_int, []),
    "cswgs_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "cswgs_last_error": (ctypes.c_char_p, []),
}

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Loads libcswgs.so (building it first when stale and nvcc is present)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_needed and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libcswgs.so is missing; run paper_2003_05293_gb300.build.build()")
        lib = ctypes.CDLL(_build.LIB)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class CswgsError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.cswgs_last_error().decode(errors="replace")
        self.status = status
        super().__init__("%s failed: %s (%s)" % (where, lib.cswgs_status_string(status).decode(), msg))


def check(status: int, where: str) -> int:
    if status != CSWGS_OK:
        raise CswgsError(status, where)
    return status


def __getattr__(name):
    # module-level access to the C functions under their C names
    if name in SIGNATURES:
        return getattr(load(), name)
    raise AttributeError(name)
