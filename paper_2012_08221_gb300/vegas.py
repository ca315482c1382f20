"""VEGAS integration on the GPU (PDFFlow Sec. 3.1: VegasFlow-style importance
sampling around the PDF calls).

``Vegas`` integrates any integrand over [0, 1]^dim that the caller writes
(in the paper's use, a matrix element times PDFs from ``xfxQ2``): per
iteration the library maps the uniforms through the grid
(`pdf_vegas_map`), the integrand runs as the caller's own device code, and
the library accumulates the sums (`pdf_vegas_accumulate`) and refines each
dimension (`pdf_vegas_refine`).  ``VegasLumi`` is the fused special case of
the parton luminosity, evaluated with the map in one kernel
(`pdf_vegas_lumi_iteration`).  Uniforms come from a torch generator on the
device or from arrays the caller passes; iterations are combined with
weights 1/sigma^2.  The variance of an iteration is taken about the previous
iteration's estimate (``shift``): the library sums (w - shift)^2, so that a
nearly flat adapted integrand does not lose its variance to the cancellation
of E[w^2] - E[w]^2.
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass, field

import numpy as np
import torch

from ._lib import check, lib
from .pdf import PDF, _ptr, _stream


@dataclass
class VegasResult:
    integral: float
    error: float
    chi2_dof: float
    iterations: list = field(default_factory=list)   # (estimate, error) per iteration
    edges: np.ndarray | None = None


class VegasLumi:
    def __init__(self, pdf: PDF, ln_tau_min: float, ln_s: float, n_bins: int = 50, alpha: float = 1.5,
                 member: int = 0):
        self.pdf, self.member = pdf, member
        self.ln_tau_min, self.ln_s = float(ln_tau_min), float(ln_s)
        self.n_bins, self.alpha = int(n_bins), float(alpha)
        self.edges = np.tile(np.linspace(0.0, 1.0, self.n_bins + 1), (2, 1))
        self.shift = 0.0               # previous estimate: the variance is taken about it
        self._sums = torch.empty(2 + 2 * self.n_bins, dtype=torch.float64, device=pdf.device)

    def iteration(self, v: torch.Tensor, refine: bool = True):
        """One iteration on the uniforms ``v`` ([n][2] float64 on the device).
        Returns (estimate, error, raw sums); the raw sums hold
        sum (w - shift)^2 with the shift in effect before the call."""
        dev = self.pdf.device
        v = v.to(device=dev, dtype=torch.float64).contiguous()
        n = v.shape[0]
        e = torch.as_tensor(self.edges, device=dev)
        check("pdf_vegas_lumi_iteration", lib().pdf_vegas_lumi_iteration(
            self.pdf.handle, self.member, self.ln_tau_min, self.ln_s, self.n_bins, _ptr(e), _ptr(v), n,
            float(self.shift), _ptr(self._sums), _stream(dev)))
        s = self._sums.cpu().numpy()
        mean, err = _mean_and_error(s, n, self.shift)
        if n:
            self.shift = mean
        if refine:
            for d in range(2):
                b = np.ascontiguousarray(s[2 + d * self.n_bins: 2 + (d + 1) * self.n_bins])
                ed = np.ascontiguousarray(self.edges[d])
                check("pdf_vegas_refine", lib().pdf_vegas_refine(
                    b.ctypes.data_as(C.POINTER(C.c_double)), self.n_bins, self.alpha,
                    ed.ctypes.data_as(C.POINTER(C.c_double))))
                self.edges[d] = ed
        return mean, err, s

    def integrate(self, n_iter: int = 5, n_per_iter: int = 1_000_000, seed: int = 0,
                  uniforms=None, warmup: int = 0) -> VegasResult:
        """``warmup`` iterations adapt the grid and are not averaged."""
        gen = torch.Generator(device=self.pdf.device)
        gen.manual_seed(seed)
        ests = []
        for it in range(warmup + n_iter):
            v = uniforms[it] if uniforms is not None else torch.rand(
                (n_per_iter, 2), generator=gen, dtype=torch.float64, device=self.pdf.device)
            est, err, _ = self.iteration(v)
            if it >= warmup:
                ests.append((est, err))
        return _combine(ests, self.edges.copy())


def _mean_and_error(s, n, shift):
    """Estimate and its standard error from [sum w, sum (w - shift)^2, ...]."""
    mean = s[0] / n
    d = mean - shift
    var = max(s[1] / n - d * d, 0.0) / max(n - 1, 1)
    return mean, math.sqrt(var)


def _combine(ests, edges):
    w = np.array([1.0 / max(e, 1e-300) ** 2 for _, e in ests])
    vals = np.array([m for m, _ in ests])
    integral = float(np.sum(w * vals) / np.sum(w))
    error = float(1.0 / math.sqrt(np.sum(w)))
    chi2 = float(np.sum(w * (vals - integral) ** 2) / max(len(ests) - 1, 1))
    return VegasResult(integral, error, chi2, ests, edges)


class Vegas:
    """VEGAS over [0, 1]^dim around a caller's integrand.

    ``integrand(r)`` receives the mapped points as a float64 device tensor
    [n][dim] and returns f(r) as a float64 device tensor [n]; it may call
    any of the library's PDF entry points."""

    def __init__(self, dim: int, n_bins: int = 50, alpha: float = 1.5, device="cuda:0"):
        self.dim, self.n_bins, self.alpha = int(dim), int(n_bins), float(alpha)
        self.device = torch.device(device)
        self.edges = np.tile(np.linspace(0.0, 1.0, self.n_bins + 1), (self.dim, 1))
        self.shift = 0.0               # previous estimate: the variance is taken about it
        self._sums = torch.empty(2 + self.dim * self.n_bins, dtype=torch.float64, device=self.device)

    def map(self, v: torch.Tensor):
        """(r [n][dim], Jacobian [n], bins [n][dim]) of uniforms v [n][dim]."""
        v = v.to(device=self.device, dtype=torch.float64).contiguous()
        n = v.shape[0]
        e = torch.as_tensor(self.edges, device=self.device)
        r = torch.empty_like(v)
        jac = torch.empty(n, dtype=torch.float64, device=self.device)
        bins = torch.empty((n, self.dim), dtype=torch.int32, device=self.device)
        check("pdf_vegas_map", lib().pdf_vegas_map(self.dim, self.n_bins, _ptr(e), _ptr(v), n, _ptr(r),
                                                   _ptr(jac), _ptr(bins), _stream(self.device)))
        return r, jac, bins

    def accumulate(self, w: torch.Tensor, bins: torch.Tensor, shift: float = 0.0) -> np.ndarray:
        """[sum w, sum (w - shift)^2, per-dimension per-bin sums of w^2]."""
        w = w.to(device=self.device, dtype=torch.float64).contiguous()
        check("pdf_vegas_accumulate", lib().pdf_vegas_accumulate(self.dim, self.n_bins, _ptr(w), _ptr(bins),
                                                                 w.numel(), float(shift), _ptr(self._sums),
                                                                 _stream(self.device)))
        return self._sums.cpu().numpy()

    def refine(self, s: np.ndarray):
        for d in range(self.dim):
            b = np.ascontiguousarray(s[2 + d * self.n_bins: 2 + (d + 1) * self.n_bins])
            ed = np.ascontiguousarray(self.edges[d])
            check("pdf_vegas_refine", lib().pdf_vegas_refine(
                b.ctypes.data_as(C.POINTER(C.c_double)), self.n_bins, self.alpha,
                ed.ctypes.data_as(C.POINTER(C.c_double))))
            self.edges[d] = ed

    def iteration(self, integrand, v: torch.Tensor, refine: bool = True):
        """One iteration on the uniforms v [n][dim]: (estimate, error, sums)."""
        r, jac, bins = self.map(v)
        w = integrand(r) * jac
        s = self.accumulate(w, bins, self.shift)
        n = r.shape[0]
        mean, err = _mean_and_error(s, n, self.shift)
        if n:
            self.shift = mean
        if refine:
            self.refine(s)
        return mean, err, s

    def integrate(self, integrand, n_iter: int = 5, n_per_iter: int = 1_000_000, seed: int = 0,
                  uniforms=None, warmup: int = 0) -> VegasResult:
        """``warmup`` iterations adapt the grid and are not averaged."""
        gen = torch.Generator(device=self.device)
        gen.manual_seed(seed)
        ests = []
        for it in range(warmup + n_iter):
            v = uniforms[it] if uniforms is not None else torch.rand(
                (n_per_iter, self.dim), generator=gen, dtype=torch.float64, device=self.device)
            est, err, _ = self.iteration(integrand, v)
            if it >= warmup:
                ests.append((est, err))
        return _combine(ests, self.edges.copy())
