"""ctypes declarations of libdamas.so (include/damas.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int, c_double, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p

DAMAS_OK, DAMAS_EINVAL, DAMAS_ENOMEM, DAMAS_ECUDA, DAMAS_ETIMEDOUT, DAMAS_EBUSY, DAMAS_ENOTFOUND = 0, -1, -2, -3, -4, -5, -6
FORM_E, FORM_P = 0, 1
F32, BF16 = 1, 2
PRED_LINEAR, PRED_HAAR = 0, 1
EPS_ABS, EPS_REL_MAX, EPS_KEEP_FRAC = 0, 1, 2
INIT_ZERO, INIT_X, INIT_STATE = 0, 1, 2
OPT_BUILD_TIMEOUT_MS, OPT_TEST_HOLD_BUILD, OPT_HBM_BUDGET_BYTES = 1, 2, 3

ERROR_NAMES = {0: "DAMAS_OK", -1: "DAMAS_EINVAL", -2: "DAMAS_ENOMEM", -3: "DAMAS_ECUDA", -4: "DAMAS_ETIMEDOUT",
               -5: "DAMAS_EBUSY", -6: "DAMAS_ENOTFOUND"}


class damas_geom(ctypes.Structure):
    _fields_ = [("M", c_int), ("mic_xyz_dev", c_void_p), ("nx", c_int), ("ny", c_int), ("x0", c_double),
                ("y0", c_double), ("dx", c_double), ("dy", c_double), ("z", c_double), ("c", c_double),
                ("formulation", c_int), ("diag_removal", c_int)]


class damas_wavelet_cfg(ctypes.Structure):
    _fields_ = [("levels", c_int), ("predictor", c_int), ("eps_mode", c_int), ("eps", c_double)]


class damas_system(ctypes.Structure):
    _fields_ = [("A_dev", c_void_p), ("At_dev", c_void_p), ("a_dtype", c_int), ("lda", c_int), ("S", c_int),
                ("b_dev", c_void_p),
                ("x_dev", c_void_p), ("state_dev", c_void_p), ("init", c_int), ("iters", c_int), ("ctas", c_int)]


class damas_solve_cfg(ctypes.Structure):
    _fields_ = [("ctas_per_system", c_int), ("timeout_ms", c_int), ("status_dev", c_void_p),
                ("a_placement", c_int), ("withhold_block", c_int), ("stats_dev", c_void_p)]


class damas_mixed_system(ctypes.Structure):
    _fields_ = [("A_bulk_dev", c_void_p), ("At_bulk_dev", c_void_p), ("A_refine_dev", c_void_p),
                ("At_refine_dev", c_void_p), ("lda", c_int), ("S", c_int), ("b_dev", c_void_p), ("x_dev", c_void_p),
                ("iters_bulk", c_int), ("iters_refine", c_int), ("ctas", c_int)]


class damas_serve_cfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_inflight", c_int), ("sm_slots", c_int),
                ("rows_per_cta", c_int)]


class damas_request(ctypes.Structure):
    _fields_ = [("M", c_int), ("mic_xyz", c_void_p), ("nx", c_int), ("ny", c_int), ("x0", c_double),
                ("y0", c_double), ("dx", c_double), ("dy", c_double), ("z", c_double), ("c", c_double),
                ("formulation", c_int), ("n_bins", c_int), ("freqs", c_void_p), ("C", c_void_p),
                ("wavelet", damas_wavelet_cfg), ("iters", c_int)]


class damas_result(ctypes.Structure):
    _fields_ = [("status", c_int), ("n_bins", c_int), ("S", c_int), ("x", ctypes.POINTER(ctypes.c_float)),
                ("total_power", ctypes.POINTER(c_double)), ("S_sub", ctypes.POINTER(c_int)),
                ("t_submit", c_double), ("t_admit", c_double), ("t_done", c_double), ("t_solve", c_double),
                ("hbm_bytes", ctypes.c_size_t), ("sm_units", c_int)]


# every symbol include/damas.h declares, with its signature
SIGNATURES = {
    "damas_create": (c_int, [ctypes.POINTER(c_void_p), c_int]),
    "damas_destroy": (c_int, [c_void_p]),
    "damas_last_error": (ctypes.c_char_p, [c_void_p]),
    "damas_set_option": (c_int, [c_void_p, c_int, ctypes.c_longlong]),
    "damas_check": (c_int, [c_void_p, c_void_p]),
    "damas_lda": (c_int, [c_int]),
    "damas_state_floats": (c_int, [c_int]),
    "damas_build_psf": (c_int, [c_void_p, ctypes.POINTER(damas_geom), c_double, c_void_p, c_int, c_int, c_void_p,
                                c_int, c_void_p, c_void_p]),
    "damas_build_psf_f32_bf16": (c_int, [c_void_p, ctypes.POINTER(damas_geom), c_double, c_void_p, c_int, c_void_p,
                                         c_void_p, c_int, c_void_p, c_void_p]),
    "das_map": (c_int, [c_void_p, ctypes.POINTER(damas_geom), c_double, c_void_p, c_void_p, c_void_p]),
    "damas_build_psf_dr": (c_int, [c_void_p, ctypes.POINTER(damas_geom), c_double, c_void_p, c_int, c_void_p, c_int,
                                   c_void_p, c_void_p, c_void_p]),
    "damas_divide": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    "damas_csm": (c_int, [c_void_p, c_void_p, c_int, ctypes.c_longlong, c_int, c_int, c_void_p, c_int, c_void_p,
                          c_void_p]),
    "wavelet_compress_grid": (c_int, [c_void_p, c_void_p, c_int, c_int, ctypes.POINTER(damas_wavelet_cfg), c_void_p,
                                      c_void_p, c_void_p, c_void_p, c_void_p]),
    "wavelet_compress_grid_noalloc": (c_int, [c_void_p, c_void_p, c_int, c_int, ctypes.POINTER(damas_wavelet_cfg),
                                              c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "damas_pad_grid": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "damas_gather": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p]),
    "damas_scatter_power": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_int, c_void_p,
                                    c_void_p]),
    "damas_solve": (c_int, [c_void_p, ctypes.POINTER(damas_system), c_int, ctypes.POINTER(damas_solve_cfg), c_void_p]),
    "damas_solve_mixed": (c_int, [c_void_p, ctypes.POINTER(damas_mixed_system), c_int,
                                  ctypes.POINTER(damas_solve_cfg), c_void_p]),
    "damas_solve_plan": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, ctypes.POINTER(c_int),
                                 ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    "damas_handover_probe": (c_int, [c_void_p, c_int, c_int, c_int, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(c_int), c_void_p]),
    "damas_chain_probe": (c_int, [c_void_p, c_int, ctypes.POINTER(ctypes.c_double), c_void_p]),
    "damas_serve_start": (c_int, [c_void_p, ctypes.POINTER(damas_serve_cfg)]),
    "damas_serve_submit": (c_int, [c_void_p, ctypes.POINTER(damas_request), ctypes.POINTER(ctypes.c_uint64)]),
    "damas_serve_poll": (c_int, [c_void_p, ctypes.c_uint64, ctypes.POINTER(damas_result)]),
    "damas_serve_release": (c_int, [c_void_p, ctypes.c_uint64]),
    "damas_serve_stop": (c_int, [c_void_p]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libdamas.so.  There is no fallback: a missing library is an error."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libdamas.so is not built ({path}); run paper_1608_05179_gb300.build.build() "
                           "(or __graft_entry__.build()) first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib
