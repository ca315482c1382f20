"""The PDF object: a grid loaded on the GPU and the queries of PDFFlow.

Mirrors the paper's Python interface (PDFFlow Sec. 2.1, Fig. 1): ``mkPDF``
builds a PDF object; ``xfxQ2`` / ``py_xfxQ`` evaluate x*f for a pid list over
arrays of x and Q^2 (or Q); ``alphasQ2`` / ``py_alphasQ`` give alpha_s;
``trace`` / ``alphas_trace`` warm the kernels up.  Every call only marshals
torch tensors (device memory, the current stream) into the C ABI of
``include/pdfgpu.h``; all arithmetic runs in the CUDA kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from ._lib import EXTRAP, INTERP, PDF_S_DOMAIN, PDF_S_RANGE, GridDesc, check, lib

__all__ = ["PDF", "mkPDF", "PDF_S_DOMAIN", "PDF_S_RANGE"]


def _stream(device=None):
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _f64_cuda(a, device):
    if isinstance(a, torch.Tensor):
        t = a.to(device=device, dtype=torch.float64)
    else:
        t = torch.as_tensor(np.asarray(a, dtype=np.float64), device=device)
    return t.contiguous()


def _pids_host(pids):
    arr = np.ascontiguousarray(np.atleast_1d(np.asarray(pids, dtype=np.int32)))
    return arr, arr.ctypes.data_as(C.POINTER(C.c_int32))


class PDF:
    """One PDF set (all its members) resident on a CUDA device.

    ``values`` is ``[members][rows][n_x][n_flav]`` (or ``[rows][n_x][n_flav]``)
    of x*f on the knots; Q knots are in GeV with duplicated thresholds.
    ``interp``: "logbicubic" (default), "logbilinear" or
    "logbicubic_small_linear"; ``extrap``: "linear" (default), "freeze" or
    "error" (see include/pdfgpu.h).
    """

    def __init__(self, x_knots, n_q, q_knots, pids, values=None, alphas=None, device="cuda:0",
                 interp="logbicubic", extrap="linear"):
        self.device = torch.device(device)
        torch.cuda.set_device(self.device)
        self._x = np.ascontiguousarray(x_knots, dtype=np.float64)
        self._nq = np.ascontiguousarray(n_q, dtype=np.int32)
        self._q = np.ascontiguousarray(q_knots, dtype=np.float64)
        self._pids = np.ascontiguousarray(pids, dtype=np.int32)
        v = None
        if values is not None:
            v = np.ascontiguousarray(values, dtype=np.float64)
            if v.ndim == 3:
                v = v[None]
        a = None if alphas is None else np.ascontiguousarray(alphas, dtype=np.float64)
        self.n_members = 1 if v is None else v.shape[0]
        desc = GridDesc()
        desc.n_x = self._x.size
        desc.x_knots = self._x.ctypes.data_as(C.POINTER(C.c_double))
        desc.n_sub = self._nq.size
        desc.n_q = self._nq.ctypes.data_as(C.POINTER(C.c_int32))
        desc.q_knots = self._q.ctypes.data_as(C.POINTER(C.c_double))
        desc.n_flav = self._pids.size
        desc.pids = self._pids.ctypes.data_as(C.POINTER(C.c_int32))
        desc.n_members = self.n_members
        desc.values = v.ctypes.data_as(C.POINTER(C.c_double)) if v is not None else None
        desc.alphas = a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None
        desc.interp = INTERP[interp] if isinstance(interp, str) else int(interp)
        desc.extrap = EXTRAP[extrap] if isinstance(extrap, str) else int(extrap)
        self.interp, self.extrap = desc.interp, desc.extrap
        h = C.c_void_p()
        check("pdf_load_grid", lib().pdf_load_grid(C.byref(desc), C.byref(h)))
        self.handle = h
        self.n_x = int(self._x.size)
        self.n_rows = int(self._q.size)
        self.n_flav = int(self._pids.size)
        self.pids = self._pids.copy()
        self.has_alphas = a is not None

    @classmethod
    def from_grid(cls, grid, device="cuda:0", with_values=True, interp="logbicubic", extrap="linear"):
        """From a ``synth.Grid`` (or any object with the same fields)."""
        return cls(grid.x_knots, grid.n_q, grid.q_knots, grid.pids,
                   grid.values if with_values else None, grid.alphas, device, interp, extrap)

    # ------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().pdf_free_grid(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -------------------------------------------------------------- values
    def value_shape(self):
        return (self.n_members, self.n_rows, self.n_x, self.n_flav)

    def bind_values(self, values: torch.Tensor):
        """Rebuild the interpolation coefficients from a device tensor of
        shape ``[members][rows][n_x][n_flav]`` (float64, contiguous)."""
        v = values.detach()
        if v.dim() == 3:
            v = v.unsqueeze(0)
        assert tuple(v.shape) == self.value_shape(), (tuple(v.shape), self.value_shape())
        v = v.to(device=self.device, dtype=torch.float64).contiguous()
        check("pdf_bind_values", lib().pdf_bind_values(self.handle, _ptr(v), _stream(self.device)))
        self._bound_ref = v      # keep alive until the stream has read it

    # ------------------------------------------------------------- queries
    def xfxQ2(self, pids, x, q2, member=0, out=None, tape=None):
        """x*f for every pid in ``pids`` at each (x_i, Q^2_i): ``[n][len(pids)]``.
        ``tape`` (``[n][4]`` float64 on the device, see ``new_tape``) also
        receives the adjoint tape of the points for ``xfxQ2_backward``."""
        return self._matrix("xfxQ2", pids, x, q2, member, out, tape)

    def xfxQ(self, pids, x, q, member=0, out=None):
        return self._matrix("xfxQ", pids, x, q, member, out)

    def xfxQ2_alphasQ2(self, pids, x, q2, member=0, out=None, alphas=None):
        """x*f for every pid in ``pids`` and alpha_s at the same points, in
        one launch that shares the Q^2 search: ``([n][len(pids)], [n])``."""
        arr, pp = _pids_host(pids)
        x = _f64_cuda(x, self.device)
        q2 = _f64_cuda(q2, self.device)
        n = x.numel()
        assert q2.numel() == n, "x and Q^2 arrays differ in length"
        if out is None:
            out = torch.empty((n, arr.size), dtype=torch.float64, device=self.device)
        if alphas is None:
            alphas = torch.empty(n, dtype=torch.float64, device=self.device)
        check("xfxQ2_alphasQ2", lib().xfxQ2_alphasQ2(self.handle, int(member), pp, arr.size, _ptr(x), _ptr(q2), n,
                                                     _ptr(out), _ptr(alphas), _stream(self.device)))
        return out, alphas

    py_xfxQ2 = xfxQ2
    py_xfxQ = xfxQ

    def _matrix(self, name, pids, x, q, member, out, tape=None):
        arr, pp = _pids_host(pids)
        x = _f64_cuda(x, self.device)
        q = _f64_cuda(q, self.device)
        n = x.numel()
        assert q.numel() == n, "x and Q arrays differ in length"
        if out is None:
            out = torch.empty((n, arr.size), dtype=torch.float64, device=self.device)
        if tape is not None:
            self._check_tape(tape, n)
            check("xfxQ2_tape", lib().xfxQ2_tape(self.handle, int(member), pp, arr.size, _ptr(x), _ptr(q), n,
                                                 _ptr(out), _ptr(tape), _stream(self.device)))
            return out
        f = getattr(lib(), name)
        check(name, f(self.handle, int(member), pp, arr.size, _ptr(x), _ptr(q), n, _ptr(out),
                      _stream(self.device)))
        return out

    def new_tape(self, n):
        """Device buffer for the adjoint tape of ``n`` points (32 bytes each)."""
        return torch.empty((n, 4), dtype=torch.float64, device=self.device)

    @staticmethod
    def dtape_doubles(n):
        """Size in doubles of a derivative tape of ``n`` points: 2 n doubles of
        patch derivatives, then n int32 bins (20 bytes per point)."""
        return 2 * n + (n + 1) // 2

    def new_dtape(self, n):
        """Device buffer for the derivative tape of ``n`` pointwise points (20
        bytes each): the patch derivatives and the accumulation bin the
        forward keeps for the adjoint.  ``dtape[:2 * n].view(n, 2)`` are the
        derivatives."""
        return torch.empty(self.dtape_doubles(n), dtype=torch.float64, device=self.device)

    def _check_tape(self, tape, n, per_point=4):
        assert tape.dtype == torch.float64 and tape.is_cuda and tape.is_contiguous(), "tape: contiguous float64"
        assert tape.numel() >= per_point * n, f"tape too small ({per_point} doubles per point)"

    def _check_dtape(self, dtape, n):
        assert dtape.dtype == torch.float64 and dtape.is_cuda and dtape.is_contiguous(), \
            "derivative tape: contiguous float64"
        assert dtape.numel() >= self.dtape_doubles(n), "derivative tape too small (20 bytes per point)"

    def xfxQ2_pw(self, pid, x, q2, member=0, out=None, tape=None, dtape=None):
        """One pid per point: ``out[i] = x*f_{pid_i}(x_i, Q^2_i)``; ``tape`` as
        for ``xfxQ2``; ``dtape`` (with ``tape``, from ``new_dtape``) also keeps
        each point's patch derivatives for ``xfxQ2_backward``."""
        x = _f64_cuda(x, self.device)
        q2 = _f64_cuda(q2, self.device)
        pid = torch.as_tensor(pid, device=self.device).to(torch.int32).contiguous()
        n = x.numel()
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=self.device)
        if tape is not None:
            self._check_tape(tape, n)
            if dtape is not None:
                self._check_dtape(dtape, n)
            check("xfxQ2_pw_tape", lib().xfxQ2_pw_tape(self.handle, int(member), _ptr(pid), _ptr(x), _ptr(q2),
                                                       n, _ptr(out), _ptr(tape), _ptr(dtape),
                                                       _stream(self.device)))
            return out
        assert dtape is None, "a derivative tape goes with a tape"
        check("xfxQ2_pw", lib().xfxQ2_pw(self.handle, int(member), _ptr(pid), _ptr(x), _ptr(q2), n,
                                         _ptr(out), _stream(self.device)))
        return out

    def alphasQ2(self, q2, out=None):
        return self._alphas("alphasQ2", q2, out)

    def alphasQ(self, q, out=None):
        return self._alphas("alphasQ", q, out)

    py_alphasQ2 = alphasQ2
    py_alphasQ = alphasQ

    def _alphas(self, name, q, out):
        q = _f64_cuda(q, self.device)
        n = q.numel()
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=self.device)
        check(name, getattr(lib(), name)(self.handle, _ptr(q), n, _ptr(out), _stream(self.device)))
        return out

    def alphasQ2_grad(self, q2, want_value=True):
        """(alpha_s or None, d alpha_s / d Q^2) at each Q^2."""
        q2 = _f64_cuda(q2, self.device)
        n = q2.numel()
        out = torch.empty(n, dtype=torch.float64, device=self.device) if want_value else None
        d = torch.empty(n, dtype=torch.float64, device=self.device)
        check("alphasQ2_grad", lib().alphasQ2_grad(self.handle, _ptr(q2), n, _ptr(out), _ptr(d),
                                                   _stream(self.device)))
        return out, d

    def xfxQ2_host(self, pids, x, q2, member=0, out=None):
        """End-to-end call on HOST arrays (CPU tensors, pinned for full copy
        speed); returns a CPU tensor ``[n][len(pids)]``."""
        arr, pp = _pids_host(pids)
        x = torch.as_tensor(x, dtype=torch.float64).contiguous()
        q2 = torch.as_tensor(q2, dtype=torch.float64).contiguous()
        assert not x.is_cuda and not q2.is_cuda
        n = x.numel()
        if out is None:
            out = torch.empty((n, arr.size), dtype=torch.float64, pin_memory=True)
        check("xfxQ2_host", lib().xfxQ2_host(self.handle, int(member), pp, arr.size, _ptr(x),
                                             _ptr(q2), n, _ptr(out)))
        return out

    # --------------------------------------------------------------- adjoint
    def xfxQ2_backward(self, pids, x, q2, grad_out, member=0, pointwise=False,
                       grad_x=True, grad_q2=True, grad_values=None, tape=None, dtape=None):
        """dL/dx, dL/dQ^2 and (accumulated into ``grad_values``, shape
        ``[rows][n_x][n_flav]``) dL/dvalues for
        L = sum grad_out * xf.  Returns (grad_x, grad_q2, grad_values).
        ``tape``: the adjoint tape a forward call wrote for the same points;
        ``dtape``: the derivative tape of that (pointwise) call, valid while
        its values are bound."""
        x = _f64_cuda(x, self.device)
        q2 = _f64_cuda(q2, self.device)
        n = x.numel()
        gout = grad_out.to(device=self.device, dtype=torch.float64).contiguous()
        gx = torch.empty(n, dtype=torch.float64, device=self.device) if grad_x else None
        gq = torch.empty(n, dtype=torch.float64, device=self.device) if grad_q2 else None
        if pointwise:
            pid = torch.as_tensor(pids, device=self.device).to(torch.int32).contiguous()
            pp, npid, keep = _ptr(pid), 0, pid
        else:
            arr, _ = _pids_host(pids)
            keep = arr
            pp, npid = C.c_void_p(arr.ctypes.data), arr.size
        assert dtape is None or tape is not None, "a derivative tape goes with a tape"
        if tape is not None:
            self._check_tape(tape, n)
            if dtape is not None:
                self._check_dtape(dtape, n)
            check("xfxQ2_backward_tape", lib().xfxQ2_backward_tape(
                self.handle, int(member), pp, npid, int(bool(pointwise)), _ptr(x), _ptr(q2), n,
                _ptr(tape), _ptr(dtape), _ptr(gout), _ptr(gx), _ptr(gq), _ptr(grad_values),
                _stream(self.device)))
        else:
            check("xfxQ2_backward", lib().xfxQ2_backward(
                self.handle, int(member), pp, npid, int(bool(pointwise)), _ptr(x), _ptr(q2), n,
                _ptr(gout), _ptr(gx), _ptr(gq), _ptr(grad_values), _stream(self.device)))
        del keep
        return gx, gq, grad_values

    # ------------------------------------------------------------- warm-up
    def trace(self):
        """Run every x*f kernel once on a tiny input (PDFFlow's `trace()`)."""
        x = torch.tensor([1e-3, 0.2], dtype=torch.float64, device=self.device)
        q2 = torch.tensor([10.0, 1e4], dtype=torch.float64, device=self.device)
        self.xfxQ2(self.pids, x, q2)
        self.xfxQ(self.pids, x, q2)
        self.xfxQ2_pw(self.pids[:1].repeat(2), x, q2)
        torch.cuda.synchronize(self.device)

    def alphas_trace(self):
        if self.has_alphas:
            self.alphasQ2(torch.tensor([10.0], dtype=torch.float64, device=self.device))
            torch.cuda.synchronize(self.device)

    # -------------------------------------------------------------- status
    def status(self) -> int:
        """Read and clear the status bits (synchronises the current stream)."""
        bits = C.c_uint32()
        check("pdf_get_status", lib().pdf_get_status(self.handle, _stream(self.device), C.byref(bits)))
        return bits.value

    def debug_log(self, v):
        v = _f64_cuda(v, self.device)
        out = torch.empty_like(v)
        check("pdf_debug_log", lib().pdf_debug_log(self.handle, _ptr(v), v.numel(), _ptr(out),
                                                   _stream(self.device)))
        return out

    def debug_cells(self, x, q2):
        """(x cells, Q^2 cells, (x guided, Q^2 guided)) of the kernels' knot
        searches at the points: a test hook."""
        x = _f64_cuda(x, self.device)
        q2 = _f64_cuda(q2, self.device)
        n = x.numel()
        xc = torch.empty(n, dtype=torch.int32, device=self.device)
        qc = torch.empty(n, dtype=torch.int32, device=self.device)
        guided = (C.c_int32 * 2)()
        check("pdf_debug_cells", lib().pdf_debug_cells(self.handle, _ptr(x), _ptr(q2), n, _ptr(xc), _ptr(qc),
                                                       guided, _stream(self.device)))
        return xc, qc, (bool(guided[0]), bool(guided[1]))


def mkPDF(grid, dirname=None, device="cuda:0", **kw) -> PDF:
    """Build a PDF object (PDFFlow Sec. 2.1 `mkPDF`): from an in-memory grid,
    or from member m of an LHAPDF lhagrid1 set named ``"<set>/<m>"`` inside
    the folder ``dirname`` (``"<set>"`` alone means member 0).  Keyword
    options (``interp``, ``extrap``) go to ``PDF.from_grid``."""
    if isinstance(grid, str):
        import os

        from .lhapdf import load
        name, _, member = grid.partition("/")
        return load(os.path.join(dirname or ".", name), first_member=int(member or 0), device=device, **kw)
    return PDF.from_grid(grid, device, **kw)


def fp64_peak() -> float:
    """Measured FP64 FMA throughput of the current GPU in FLOP/s."""
    v = C.c_double()
    check("pdf_probe_fp64_peak", lib().pdf_probe_fp64_peak(C.byref(v)))
    return v.value


MMA_SHAPES = ("m8n8k4", "m16n8k4", "m16n8k8", "m16n8k16")


def fp64_mma_peak(shape: str = "m8n8k4") -> float:
    """Measured throughput of the FP64 tensor instruction (``mma.sync`` with
    f64 operands) of one shape on the current GPU, in FLOP/s (2 M N K per
    warp-wide instruction)."""
    v = C.c_double()
    check("pdf_probe_fp64_mma_peak", lib().pdf_probe_fp64_mma_peak(MMA_SHAPES.index(shape), C.byref(v)))
    return v.value


def fp64_mixed() -> dict:
    """Rates (FLOP/s) of equal FP64 work issued as DFMA chains alone, as
    m8n8k4 ``mma.sync`` chains alone, and as both interleaved in each warp;
    a mixed rate well below the sum of the two says they share one pipe."""
    f, m, x = C.c_double(), C.c_double(), C.c_double()
    check("pdf_probe_fp64_mixed", lib().pdf_probe_fp64_mixed(C.byref(f), C.byref(m), C.byref(x)))
    return {"dfma": f.value, "dmma": m.value, "mixed": x.value}
