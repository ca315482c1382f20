"""Host-side error paths of the C ABI (CPU only: validation happens before any
CUDA call, so malformed descriptions are rejected without a GPU)."""
import ctypes as C

import numpy as np
import pytest

from paper_2012_08221_gb300 import _lib, build, synth


@pytest.fixture(scope="module")
def L():
    build.build()
    return _lib.lib()


def _desc(x, nq, q, pids, nmem=1, interp=0, extrap=0):
    keep = [np.ascontiguousarray(x, np.float64), np.ascontiguousarray(nq, np.int32),
            np.ascontiguousarray(q, np.float64), np.ascontiguousarray(pids, np.int32)]
    d = _lib.GridDesc()
    d.n_x = keep[0].size
    d.x_knots = keep[0].ctypes.data_as(C.POINTER(C.c_double))
    d.n_sub = keep[1].size
    d.n_q = keep[1].ctypes.data_as(C.POINTER(C.c_int32))
    d.q_knots = keep[2].ctypes.data_as(C.POINTER(C.c_double))
    d.n_flav = keep[3].size
    d.pids = keep[3].ctypes.data_as(C.POINTER(C.c_int32))
    d.n_members = nmem
    d.values = None
    d.alphas = None
    d.interp = interp
    d.extrap = extrap
    return d, keep


def _load(L, *args, **kw):
    d, keep = _desc(*args, **kw)
    h = C.c_void_p()
    rc = L.pdf_load_grid(C.byref(d), C.byref(h))
    return rc, L.pdf_last_error().decode()


X = [1e-5, 1e-3, 0.1, 1.0]
Q = [1.0, 2.0, 2.0, 10.0, 100.0]
NQ = [2, 3]
P = [-1, 0, 1]


@pytest.mark.parametrize("args,code,needle", [
    (([1e-5], [2], [1.0, 2.0], P), -2, "at least 2 x knots"),
    (([1e-5, 1e-3, 1e-3, 1.0], NQ, Q, P), -2, "x knots not strictly ascending"),
    (([1e-5, 1e-3, 2.0], NQ, Q, P), -2, "outside (0, 1]"),
    (([0.0, 1e-3, 1.0], NQ, Q, P), -2, "outside (0, 1]"),
    ((X, [2, 3], [1.0, 2.0, 2.5, 10.0, 100.0], P), -2, "not duplicated"),
    ((X, [1, 4], Q, P), -2, "fewer than 2 knots"),
    ((X, [2, 3], [1.0, 2.0, 2.0, 2.0, 100.0], P), -2, "not strictly ascending inside"),
    ((X, NQ, [1.0, 2.0, 2.0, 10.0, float("nan")], P), -2, "not positive finite"),
    ((X, NQ, Q, [1, 1]), -2, "duplicate pid"),
    ((X, NQ, Q, [0, 21]), -2, "gluon listed twice"),
    ((X, NQ, Q, [99]), -2, "[-64, 64]"),
    ((X, NQ, Q, []), -2, "flavour count"),
])
def test_malformed_descriptions(L, args, code, needle):
    rc, msg = _load(L, *args)
    assert rc == code
    assert needle in msg


def test_unknown_modes(L):
    assert _load(L, X, NQ, Q, P, interp=3)[0] == -2
    assert _load(L, X, NQ, Q, P, extrap=-1)[0] == -2


def test_zero_members(L):
    rc, msg = _load(L, X, NQ, Q, P, nmem=0)
    assert rc == -2 and "member" in msg


def test_null_arguments(L):
    assert L.pdf_load_grid(None, None) == -1
    assert L.xfxQ2(None, 0, None, 0, None, None, 0, None, None) == -1
    assert "null grid" in L.pdf_last_error().decode()
    assert L.pdf_free_grid(None) == -1
    assert L.pdf_batch_run(None, None) == -1
    assert L.pdf_batch_free(None) == -1
    assert L.pdf_lumi(None, 0, None, None, None, None, None, 0.0, 0, None, None, None, None, None) == -1


def test_error_message_is_per_call(L):
    _load(L, [1e-5], [2], [1.0, 2.0], P)
    assert L.pdf_last_error() != b""
    L.pdf_grid_info(None, None, None, None, None, None)
    assert b"null grid" in L.pdf_last_error()


def test_python_errors_name_the_code(L):
    err = _lib.PdfError("pdf_load_grid", -2)
    assert "PDF_E_DESC" in str(err)


def test_synthetic_grids_pass_host_validation_shapes():
    """The generators produce descriptions the validator accepts (checked on
    the host rules the library applies)."""
    for g in (synth.grid_small(), synth.grid_nnpdf(), synth.grid_set_b()):
        assert np.all(np.diff(g.x_knots) > 0) and g.x_knots[0] > 0 and g.x_knots[-1] <= 1
        starts = np.concatenate([[0], np.cumsum(g.n_q)])
        for s in range(len(g.n_q)):
            seg = g.q_knots[starts[s]:starts[s + 1]]
            assert np.all(np.diff(seg * seg) > 0)
            if s + 1 < len(g.n_q):
                assert g.q_knots[starts[s + 1] - 1] == g.q_knots[starts[s + 1]]
        assert g.values.shape == (g.n_members, g.n_rows, g.n_x, g.n_flav)
