"""Fused luminosity workload (PDFFlow Sec. 3.1-3.2) through the C ABI.

Events are given in log variables (ln tau, y, ln s) with the flags of the
injected low tail, as device tensors; see ``synth.events_lhc``.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from ._lib import check, lib
from .pdf import PDF, _ptr, _stream


@dataclass
class DeviceEvents:
    ln_tau: torch.Tensor
    y: torch.Tensor
    flags: torch.Tensor
    ln_mu2: torch.Tensor
    ln_x1: torch.Tensor
    ln_s: float

    @property
    def n(self) -> int:
        return int(self.ln_tau.numel())

    @classmethod
    def from_host(cls, ev, device="cuda", n=None):
        n = ev.ln_tau.size if n is None else int(n)

        def d(a, dt):
            return torch.as_tensor(np.ascontiguousarray(a[:n]), device=device).to(dt).contiguous()
        return cls(d(ev.ln_tau, torch.float64), d(ev.y, torch.float64), d(ev.flags, torch.uint8),
                   d(ev.ln_mu2, torch.float64), d(ev.ln_x1, torch.float64), float(ev.ln_s))


def luminosity(pdf: PDF, ev: DeviceEvents, member=0, want_lum=True, want_alphas=True, out=None,
               save_p=None):
    """Returns (L as a 0-d device tensor, lum[n] or None, alpha_s[n] or None).
    ``save_p``: optional float64 device tensor [n][2][n_flav] that receives the
    partner factors for ``luminosity_backward``."""
    dev = pdf.device
    n = ev.n
    lum = torch.empty(n, dtype=torch.float64, device=dev) if want_lum else None
    a_s = torch.empty(n, dtype=torch.float64, device=dev) if (want_alphas and pdf.has_alphas) else None
    L = out if out is not None else torch.empty((), dtype=torch.float64, device=dev)
    check("pdf_lumi", lib().pdf_lumi(pdf.handle, int(member), _ptr(ev.ln_tau), _ptr(ev.y),
                                     _ptr(ev.flags), _ptr(ev.ln_mu2), _ptr(ev.ln_x1), ev.ln_s, n,
                                     _ptr(lum), _ptr(a_s), _ptr(L), _ptr(save_p), _stream(dev)))
    return L, lum, a_s


def luminosity_backward(pdf: PDF, ev: DeviceEvents, dL: float, grad_values: torch.Tensor, member=0,
                        saved_p=None):
    """Accumulate dL/dvalues * dL into ``grad_values`` ([rows][n_x][n_flav]);
    ``saved_p`` from the forward call skips recomputing the partner factors."""
    check("pdf_lumi_backward", lib().pdf_lumi_backward(
        pdf.handle, int(member), _ptr(ev.ln_tau), _ptr(ev.y), _ptr(ev.flags), _ptr(ev.ln_mu2),
        _ptr(ev.ln_x1), ev.ln_s, ev.n, C.c_double(dL), _ptr(saved_p), _ptr(grad_values),
        _stream(pdf.device)))
    return grad_values
