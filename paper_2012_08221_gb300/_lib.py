"""ctypes declarations of the C ABI in ``include/pdfgpu.h``.

Loading fails loudly when ``libpdfgpu.so`` has not been built: there is no
CPU fallback.  Build it with ``paper_2012_08221_gb300.build.build()`` (or
``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

c_grid = C.c_void_p
c_batch = C.c_void_p
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int32)
_U8 = C.POINTER(C.c_uint8)
_VP = C.c_void_p

PDF_MAX_PIDS = 64
PDF_S_DOMAIN = 1
PDF_S_RANGE = 2
INTERP = {"logbicubic": 0, "logbilinear": 1, "logbicubic_small_linear": 2}
EXTRAP = {"linear": 0, "freeze": 1, "error": 2, "continuation": 3}
ERRORS = {-1: "PDF_E_ARG", -2: "PDF_E_DESC", -3: "PDF_E_CUDA", -4: "PDF_E_UNBOUND",
          -5: "PDF_E_NOMEM", -6: "PDF_E_RANGE"}


class GridDesc(C.Structure):
    _fields_ = [("n_x", C.c_int32), ("x_knots", _D),
                ("n_sub", C.c_int32), ("n_q", _I), ("q_knots", _D),
                ("n_flav", C.c_int32), ("pids", _I),
                ("n_members", C.c_int32), ("values", _D), ("alphas", _D),
                ("interp", C.c_int32), ("extrap", C.c_int32)]


class BatchDesc(C.Structure):
    _fields_ = [("grid", c_grid), ("member", C.c_int32), ("n_pid", C.c_int32),
                ("pids", C.c_int32 * 16), ("x", _VP), ("q2", _VP), ("n", C.c_int64),
                ("out", _VP)]


# name -> (argtypes) ; every entry point returns int except pdf_last_error
SIGNATURES = {
    "pdf_load_grid": [C.POINTER(GridDesc), C.POINTER(c_grid)],
    "pdf_bind_values": [c_grid, _VP, _VP],
    "pdf_free_grid": [c_grid],
    "pdf_grid_info": [c_grid, _I, _I, _I, _I, _I],
    "xfxQ2": [c_grid, C.c_int32, _I, C.c_int32, _VP, _VP, C.c_int64, _VP, _VP],
    "xfxQ": [c_grid, C.c_int32, _I, C.c_int32, _VP, _VP, C.c_int64, _VP, _VP],
    "xfxQ2_pw": [c_grid, C.c_int32, _VP, _VP, _VP, C.c_int64, _VP, _VP],
    "xfxQ2_alphasQ2": [c_grid, C.c_int32, _I, C.c_int32, _VP, _VP, C.c_int64, _VP, _VP, _VP],
    "xfxQ2_tape": [c_grid, C.c_int32, _I, C.c_int32, _VP, _VP, C.c_int64, _VP, _VP, _VP],
    "xfxQ2_pw_tape": [c_grid, C.c_int32, _VP, _VP, _VP, C.c_int64, _VP, _VP, _VP, _VP],
    "alphasQ2": [c_grid, _VP, C.c_int64, _VP, _VP],
    "alphasQ": [c_grid, _VP, C.c_int64, _VP, _VP],
    "alphasQ2_grad": [c_grid, _VP, C.c_int64, _VP, _VP, _VP],
    "xfxQ2_host": [c_grid, C.c_int32, _I, C.c_int32, _VP, _VP, C.c_int64, _VP],
    "xfxQ2_backward": [c_grid, C.c_int32, _VP, C.c_int32, C.c_int32, _VP, _VP, C.c_int64,
                       _VP, _VP, _VP, _VP, _VP],
    "xfxQ2_backward_tape": [c_grid, C.c_int32, _VP, C.c_int32, C.c_int32, _VP, _VP, C.c_int64,
                            _VP, _VP, _VP, _VP, _VP, _VP, _VP],
    "pdf_batch_prepare": [C.POINTER(BatchDesc), C.c_int32, C.c_int32, _VP, C.POINTER(c_batch)],
    "pdf_batch_run": [c_batch, _VP],
    "pdf_batch_info": [c_batch, _I, _I, _I, _I, C.POINTER(C.c_float)],
    "pdf_batch_free": [c_batch],
    "pdf_batch_run_noalloc": [C.POINTER(BatchDesc), C.c_int32, _VP],
    "pdf_lumi": [c_grid, C.c_int32, _VP, _VP, _VP, _VP, _VP, C.c_double, C.c_int64,
                 _VP, _VP, _VP, _VP, _VP],
    "pdf_lumi_backward": [c_grid, C.c_int32, _VP, _VP, _VP, _VP, _VP, C.c_double, C.c_int64,
                          C.c_double, _VP, _VP, _VP],
    "pdf_get_status": [c_grid, _VP, C.POINTER(C.c_uint32)],
    "pdf_vegas_lumi_iteration": [c_grid, C.c_int32, C.c_double, C.c_double, C.c_int32, _VP, _VP,
                                 C.c_int64, C.c_double, _VP, _VP],
    "pdf_vegas_refine": [_D, C.c_int32, C.c_double, _D],
    "pdf_vegas_map": [C.c_int32, C.c_int32, _VP, _VP, C.c_int64, _VP, _VP, _VP, _VP],
    "pdf_vegas_accumulate": [C.c_int32, C.c_int32, _VP, _VP, C.c_int64, C.c_double, _VP, _VP],
    "pdf_lhapdf_open": [C.c_char_p, C.c_int32, C.c_int32, C.POINTER(C.c_void_p)],
    "pdf_lhapdf_desc": [C.c_void_p, C.POINTER(GridDesc)],
    "pdf_lhapdf_close": [C.c_void_p],
    "pdf_probe_fp64_peak": [_D],
    "pdf_probe_fp64_mma_peak": [C.c_int32, _D],
    "pdf_probe_fp64_mixed": [_D, _D, _D],
    "pdf_debug_log": [c_grid, _VP, C.c_int64, _VP, _VP],
    "pdf_debug_cells": [c_grid, _VP, _VP, C.c_int64, _VP, _VP, C.POINTER(C.c_int32), _VP],
}


def path() -> str:
    return _build.LIB


def lib():
    """The loaded library (raises if it was never built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path()
            if not os.path.exists(p):
                raise RuntimeError(
                    f"CUDA library not built ({p}); run paper_2012_08221_gb300.build.build()")
            L = C.CDLL(p)
            for name, args in SIGNATURES.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = C.c_int
            L.pdf_last_error.argtypes = []
            L.pdf_last_error.restype = C.c_char_p
            _lib = L
    return _lib


class PdfError(RuntimeError):
    def __init__(self, name, code):
        msg = lib().pdf_last_error().decode(errors="replace")
        super().__init__(f"{name} failed: {ERRORS.get(code, code)}: {msg}")
        self.code = code


def check(name, rc):
    if rc != 0:
        raise PdfError(name, rc)
    return rc
