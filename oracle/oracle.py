"""Python front end of the FP64 CPU oracle (``pdf_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline arm.  The CUDA library never imports it; the two share
no code.  ``build()`` compiles the C file with gcc (-O2, no FMA contraction, no
fast-math, OpenMP) into ``oracle/_build/liborc.so``.

Every function here only marshals numpy arrays into the C routines; the
arithmetic is in ``pdf_oracle.c`` (see its header for the definition followed).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle if the shared object is missing or stale."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Grid(C.Structure):
    _fields_ = [
        ("n_x", C.c_int), ("x_knots", C.POINTER(C.c_double)),
        ("n_sub", C.c_int), ("n_q", C.POINTER(C.c_int)),
        ("q_knots", C.POINTER(C.c_double)),
        ("n_flav", C.c_int), ("pids", C.POINTER(C.c_int)),
        ("n_members", C.c_int), ("values", C.POINTER(C.c_double)),
        ("alphas", C.POINTER(C.c_double)),
        ("U", C.POINTER(C.c_double)), ("W", C.POINTER(C.c_double)),
        ("row0", C.POINTER(C.c_int)), ("rows", C.c_int),
        ("interp", C.c_int), ("extrap", C.c_int),
    ]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_G = C.POINTER(_Grid)


def load_library(path):
    """A handle on an oracle shared object with every prototype declared."""
    L = C.CDLL(path)
    _declare(L)
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            _declare(L)
            _lib = L
    return _lib


def _declare(L):
    """Argument and result types of every oracle entry point."""
    L.orc_init.argtypes = [_G]
    L.orc_init.restype = C.c_int
    L.orc_xfxq2.argtypes = [_G, C.c_int, C.c_int, C.c_double, C.c_double]
    L.orc_xfxq2.restype = C.c_double
    L.orc_xfxq2_uw.argtypes = [_G, C.c_int, C.c_int, C.c_double, C.c_double, _D, _D]
    L.orc_xfxq2_uw.restype = C.c_double
    L.orc_xfxq2_grad.argtypes = [_G, C.c_int, C.c_int, C.c_double, C.c_double, _D, _D]
    L.orc_xfxq2_grad.restype = C.c_double
    L.orc_alphas.argtypes = [_G, C.c_double]
    L.orc_alphas.restype = C.c_double
    L.orc_alphas_grad.argtypes = [_G, C.c_double, _D]
    L.orc_alphas_grad.restype = C.c_double
    L.orc_alphas_w.argtypes = [_G, C.c_double]
    L.orc_alphas_w.restype = C.c_double
    L.orc_cell_weight_uw.argtypes = [_G, C.c_int, C.c_int, C.c_double, C.c_double]
    L.orc_cell_weight_uw.restype = C.c_double
    L.orc_xfxq2_batch.argtypes = [_G, C.c_int, _I, C.c_int, _D, _D, C.c_int64, _D]
    L.orc_xfxq2_pw_batch.argtypes = [_G, C.c_int, _I, _D, _D, C.c_int64, _D]
    L.orc_alphas_batch.argtypes = [_G, _D, C.c_int64, _D]
    L.orc_grad_pw_batch.argtypes = [_G, C.c_int, _I, _D, _D, C.c_int64, _D, _D]
    L.orc_kappa_batch.argtypes = [_G, C.c_int, _I, C.c_int, C.c_int, _D, _D,
                                  C.c_int64, _D]
    L.orc_alphas_kappa_batch.argtypes = [_G, _D, C.c_int64, _D]
    L.orc_alphas_kappa_batch.restype = None
    L.orc_dgrid_pw.argtypes = [_G, _I, _D, _D, _D, C.c_int64, _D, C.c_int]
    L.orc_dgrid_batch.argtypes = [_G, _I, C.c_int, _D, _D, _D, C.c_int64, _D, C.c_int]
    U8 = C.POINTER(C.c_ubyte)
    L.orc_lumi_batch.argtypes = [_G, C.c_int, _D, _D, U8, _D, _D, C.c_double,
                                 C.c_int64, _D, _D]
    L.orc_lumi_batch.restype = C.c_double
    L.orc_lumi_dgrid.argtypes = [_G, C.c_int, _D, _D, U8, _D, _D, C.c_double,
                                 C.c_int64, _D, C.c_int]
    L.orc_vegas_sums.argtypes = [_G, C.c_int, C.c_double, C.c_double, C.c_int, _D, _D,
                                 C.c_int64, C.c_double, _D]
    L.orc_vegas_refine.argtypes = [_D, C.c_int, C.c_double, _D]
    L.orc_vegas_map.argtypes = [C.c_int, C.c_int, _D, _D, C.c_int64, _D, _D, C.POINTER(C.c_int)]
    L.orc_vegas_map.restype = None
    L.orc_vegas_accumulate.argtypes = [C.c_int, C.c_int, _D, C.POINTER(C.c_int), C.c_int64, C.c_double, _D]
    L.orc_vegas_accumulate.restype = None


def _d(a):
    return a.ctypes.data_as(_D)


def _i(a):
    return a.ctypes.data_as(_I)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def set_threads(n: int | None):
    """OpenMP thread count for the batch drivers (None: leave as is)."""
    if n is not None:
        os.environ["OMP_NUM_THREADS"] = str(int(n))
        try:
            gomp = C.CDLL("libgomp.so.1")
            gomp.omp_set_num_threads(C.c_int(int(n)))
        except OSError:
            pass


class OracleGrid:
    """A grid as the oracle sees it.  Arguments mirror the library's grid
    description: x knots, knots per Q subgrid, Q knots (GeV, thresholds
    duplicated), pids, values ``[members][rows][n_x][n_flav]`` and alpha_s
    knot values ``[rows]`` (or None)."""

    def __init__(self, x_knots, n_q, q_knots, pids, values, alphas=None, interp=0, extrap=0):
        self.x_knots = _f64(x_knots)
        self.n_q = _i32(n_q)
        self.q_knots = _f64(q_knots)
        self.pids = _i32(pids)
        v = _f64(values)
        if v.ndim == 3:
            v = v[None]
        self.values = v
        self.alphas = None if alphas is None else _f64(alphas)
        self.U = np.empty(self.x_knots.size)
        self.W = np.empty(self.q_knots.size)
        self.row0 = np.empty(self.n_q.size, dtype=np.int32)
        g = _Grid()
        g.n_x = self.x_knots.size
        g.x_knots = _d(self.x_knots)
        g.n_sub = self.n_q.size
        g.n_q = _i(self.n_q)
        g.q_knots = _d(self.q_knots)
        g.n_flav = self.pids.size
        g.pids = _i(self.pids)
        g.n_members = v.shape[0]
        g.values = _d(self.values)
        g.alphas = _d(self.alphas) if self.alphas is not None else None
        g.U = _d(self.U)
        g.W = _d(self.W)
        g.row0 = _i(self.row0)
        g.interp = int(interp)
        g.extrap = int(extrap)
        self.interp, self.extrap = int(interp), int(extrap)
        self._g = g
        rc = lib().orc_init(C.byref(g))
        if rc != 0:
            raise ValueError(f"oracle grid rejected ({rc})")
        assert self.values.shape[1:] == (g.rows, g.n_x, g.n_flav), "values shape"

    @classmethod
    def from_synth(cls, grid, interp=0, extrap=0):
        return cls(grid.x_knots, grid.n_q, grid.q_knots, grid.pids, grid.values, grid.alphas,
                   interp, extrap)

    @property
    def ptr(self):
        return C.byref(self._g)

    # -- scalar entry points
    def xfxq2(self, pid, x, q2, member=0):
        return lib().orc_xfxq2(self.ptr, member, int(pid), float(x), float(q2))

    def xfxq2_uw(self, pid, u, w, member=0):
        du, dw = C.c_double(), C.c_double()
        v = lib().orc_xfxq2_uw(self.ptr, member, int(pid), float(u), float(w),
                               C.byref(du), C.byref(dw))
        return v, du.value, dw.value

    def grad(self, pid, x, q2, member=0):
        dx, dq2 = C.c_double(), C.c_double()
        v = lib().orc_xfxq2_grad(self.ptr, member, int(pid), float(x), float(q2),
                                 C.byref(dx), C.byref(dq2))
        return v, dx.value, dq2.value

    def alphas_q2(self, q2):
        return lib().orc_alphas(self.ptr, float(q2))

    def alphas_grad(self, q2):
        """(alpha_s, d alpha_s / d Q^2) at one Q^2."""
        d = C.c_double()
        v = lib().orc_alphas_grad(self.ptr, float(q2), C.byref(d))
        return v, d.value

    def alphas_w(self, w):
        return lib().orc_alphas_w(self.ptr, float(w))

    def cell_weight(self, row, k, u, w):
        return lib().orc_cell_weight_uw(self.ptr, int(row), int(k), float(u), float(w))

    # -- batches
    def xfxq2_batch(self, pids, x, q2, member=0):
        pids, x, q2 = _i32(pids), _f64(x), _f64(q2)
        out = np.empty((x.size, pids.size))
        lib().orc_xfxq2_batch(self.ptr, member, _i(pids), pids.size, _d(x), _d(q2), x.size, _d(out))
        return out

    def xfxq2_pw(self, pid, x, q2, member=0):
        pid, x, q2 = _i32(pid), _f64(x), _f64(q2)
        out = np.empty(x.size)
        lib().orc_xfxq2_pw_batch(self.ptr, member, _i(pid), _d(x), _d(q2), x.size, _d(out))
        return out

    def alphas_batch(self, q2):
        q2 = _f64(q2)
        out = np.empty(q2.size)
        lib().orc_alphas_batch(self.ptr, _d(q2), q2.size, _d(out))
        return out

    def grad_pw(self, pid, x, q2, member=0):
        pid, x, q2 = _i32(pid), _f64(x), _f64(q2)
        dx, dq2 = np.empty(x.size), np.empty(x.size)
        lib().orc_grad_pw_batch(self.ptr, member, _i(pid), _d(x), _d(q2), x.size, _d(dx), _d(dq2))
        return dx, dq2

    def kappa(self, pids, x, q2, member=0, pointwise=False):
        pids, x, q2 = _i32(pids), _f64(x), _f64(q2)
        shape = (x.size,) if pointwise else (x.size, pids.size)
        out = np.empty(shape)
        lib().orc_kappa_batch(self.ptr, member, _i(pids), pids.size, int(pointwise),
                              _d(x), _d(q2), x.size, _d(out))
        return out

    def alphas_kappa(self, q2):
        """Sum of |weight * alpha_s knot value| over the knots (tolerance
        scale of alpha_s, as kappa is for x*f)."""
        q2 = _f64(q2)
        out = np.empty(q2.size)
        lib().orc_alphas_kappa_batch(self.ptr, _d(q2), q2.size, _d(out))
        return out

    def dgrid_pw(self, pid, x, q2, gw, absval=False):
        """dL/dvalues for L = sum_i gw_i xf_{pid_i} (the weights do not depend
        on the member).  absval: the sum of |term| instead (tolerance scale)."""
        pid, x, q2, gw = _i32(pid), _f64(x), _f64(q2), _f64(gw)
        grad = np.zeros(self.values.shape[1:])
        lib().orc_dgrid_pw(self.ptr, _i(pid), _d(x), _d(q2), _d(gw), x.size, _d(grad), int(absval))
        return grad

    def dgrid(self, pids, x, q2, gout, absval=False):
        pids, x, q2, gout = _i32(pids), _f64(x), _f64(q2), _f64(gout)
        grad = np.zeros(self.values.shape[1:])
        lib().orc_dgrid_batch(self.ptr, _i(pids), pids.size, _d(x), _d(q2), _d(gout),
                              x.size, _d(grad), int(absval))
        return grad

    def lumi(self, ev, member=0, n=None):
        n = ev.ln_tau.size if n is None else int(n)
        lt, y = _f64(ev.ln_tau[:n]), _f64(ev.y[:n])
        fl = np.ascontiguousarray(ev.flags[:n], dtype=np.uint8)
        lm, lx = _f64(ev.ln_mu2[:n]), _f64(ev.ln_x1[:n])
        lum, a_s = np.empty(n), np.empty(n)
        L = lib().orc_lumi_batch(self.ptr, member, _d(lt), _d(y),
                                 fl.ctypes.data_as(C.POINTER(C.c_ubyte)), _d(lm), _d(lx),
                                 float(ev.ln_s), n, _d(lum), _d(a_s))
        return L, lum, a_s

    def lumi_dgrid(self, ev, member=0, n=None, absval=False):
        n = ev.ln_tau.size if n is None else int(n)
        lt, y = _f64(ev.ln_tau[:n]), _f64(ev.y[:n])
        fl = np.ascontiguousarray(ev.flags[:n], dtype=np.uint8)
        lm, lx = _f64(ev.ln_mu2[:n]), _f64(ev.ln_x1[:n])
        grad = np.zeros(self.values.shape[1:])
        lib().orc_lumi_dgrid(self.ptr, member, _d(lt), _d(y),
                             fl.ctypes.data_as(C.POINTER(C.c_ubyte)), _d(lm), _d(lx),
                             float(ev.ln_s), n, _d(grad), int(absval))
        return grad


def vegas_refine(bin_w2, alpha, edges):
    """New edges (one dimension) from per-bin sums of w^2 (Lepage's rule)."""
    b = _f64(bin_w2)
    e = _f64(edges).copy()
    lib().orc_vegas_refine(_d(b), b.size, float(alpha), _d(e))
    return e


def vegas_map(edges, v):
    """The VEGAS map of uniforms v [n][dim] through edges [dim][n_bins+1]:
    (r [n][dim], Jacobian [n], bins [n][dim])."""
    e = _f64(np.atleast_2d(edges))
    dim, n_bins = e.shape[0], e.shape[1] - 1
    v = _f64(v).reshape(-1, dim)
    r = np.empty_like(v)
    jac = np.empty(v.shape[0])
    bins = np.empty(v.shape, dtype=np.int32)
    lib().orc_vegas_map(dim, n_bins, _d(e), _d(v), v.shape[0], _d(r), _d(jac),
                        bins.ctypes.data_as(C.POINTER(C.c_int)))
    return r, jac, bins


def vegas_accumulate(n_bins, w, bins, shift=0.0):
    """[sum w, sum (w - shift)^2, per-dimension per-bin sums of w^2] of
    weights w [n] with their bins [n][dim]."""
    w = _f64(w)
    bins = np.ascontiguousarray(bins, dtype=np.int32)
    dim = bins.shape[1]
    out = np.empty(2 + dim * n_bins)
    lib().orc_vegas_accumulate(dim, n_bins, _d(w), bins.ctypes.data_as(C.POINTER(C.c_int)), w.size,
                               float(shift), _d(out))
    return out


def vegas_sums(grid: "OracleGrid", member, ln_tau_min, ln_s, edges, v, shift=0.0):
    """Sums of one VEGAS iteration of the luminosity integral (see the C
    file): [sum w, sum (w - shift)^2, per-bin w^2 of dimension 0, of
    dimension 1]."""
    e = _f64(edges)
    n_bins = e.shape[1] - 1
    v = _f64(v)
    out = np.empty(2 + 2 * n_bins)
    lib().orc_vegas_sums(grid.ptr, member, float(ln_tau_min), float(ln_s), n_bins, _d(e), _d(v),
                         v.shape[0], float(shift), _d(out))
    return out
