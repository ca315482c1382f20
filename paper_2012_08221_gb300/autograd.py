"""torch.autograd bindings of the adjoint kernels.

``XfxQ2Fn`` evaluates x*f with the grid values as a differentiable tensor:
the forward rebuilds the interpolation coefficients from the tensor and runs
the forward kernel; the backward runs the hand-written adjoint kernel, which
returns dL/dx, dL/dQ^2 and the scatter of the 16 bicubic stencil weights
into dL/dvalues (the derivative a PDF fit needs).  The forward keeps a
32-byte adjoint tape per point (cells, local coordinates, flags), so that the
backward does not search the knots or take logarithms again; in the pointwise
form, when x or Q^2 needs a gradient, also the 20-byte derivative tape (the
patch derivatives, computed with the value, and the point's bin in the grid
gradient), so that the backward does not reload the coefficients, counts its
bins from 4 bytes per point and needs no rebinding.  ``LumiFn`` does the same
for the fused luminosity workload, L = (1/n) sum_e sum_a f_a(x1) f_-a(x2).

The coefficients live in ONE table per PDF handle, rebuilt by every forward and
backward call from the values tensor it is given: two differentiable
evaluations with different values on one handle, from two streams at once,
race on that table.  Use one handle per stream (or order the streams).
"""
from __future__ import annotations

import torch

from ._lib import EXTRAP
from .pdf import PDF


class XfxQ2Fn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, values, x, q2, pdf: PDF, pids, member: int, pointwise: bool, use_tape: bool = True):
        pdf.bind_values(values)
        # the adjoint tape (32 bytes per point) saves the backward pass the
        # knot searches and logarithms; the power-law continuation has no
        # adjoint, so it gets none
        tape = pdf.new_tape(x.numel()) if use_tape and pdf.extrap != EXTRAP["continuation"] else None
        dtape = None
        if pointwise:
            if tape is not None and (ctx.needs_input_grad[1] or ctx.needs_input_grad[2]):
                dtape = pdf.new_dtape(x.numel())
            out = pdf.xfxQ2_pw(pids, x, q2, member, tape=tape, dtape=dtape)
        else:
            out = pdf.xfxQ2(pids, x, q2, member, tape=tape)
        ctx.save_for_backward(values, x, q2)
        ctx.pdf, ctx.pids, ctx.member, ctx.pointwise = pdf, pids, member, pointwise
        ctx.tape, ctx.dtape = tape, dtape
        return out

    @staticmethod
    def backward(ctx, gout):
        values, x, q2 = ctx.saved_tensors
        pdf: PDF = ctx.pdf
        need_v, need_x, need_q = ctx.needs_input_grad[:3]
        if ctx.dtape is None:
            pdf.bind_values(values)       # the coefficients of these values
        gvals = None
        gslice = None
        if need_v:
            gvals = torch.zeros_like(values)
            gslice = gvals[ctx.member] if values.dim() == 4 else gvals
        gx, gq, _ = pdf.xfxQ2_backward(ctx.pids, x, q2, gout, ctx.member, ctx.pointwise,
                                       grad_x=need_x, grad_q2=need_q, grad_values=gslice, tape=ctx.tape,
                                       dtape=ctx.dtape)
        return gvals, gx, gq, None, None, None, None, None


def xfxQ2(pdf: PDF, values, pids, x, q2, member: int = 0, use_tape: bool = True):
    """Differentiable x*f for a shared pid list: ``[n][len(pids)]``."""
    return XfxQ2Fn.apply(values, x, q2, pdf, pids, member, False, use_tape)


def xfxQ2_pw(pdf: PDF, values, pid, x, q2, member: int = 0, use_tape: bool = True):
    """Differentiable x*f with one pid per point: ``[n]``."""
    return XfxQ2Fn.apply(values, x, q2, pdf, pid, member, True, use_tape)


class AlphasFn(torch.autograd.Function):
    """alpha_s(Q^2) differentiable in Q^2 (alpha_s knots are not a parameter)."""

    @staticmethod
    def forward(ctx, q2, pdf: PDF):
        ctx.save_for_backward(q2)
        ctx.pdf = pdf
        return pdf.alphasQ2(q2)

    @staticmethod
    def backward(ctx, gout):
        (q2,) = ctx.saved_tensors
        _, d = ctx.pdf.alphasQ2_grad(q2, want_value=False)
        return gout * d, None


def alphasQ2(pdf: PDF, q2):
    """Differentiable alpha_s(Q^2)."""
    return AlphasFn.apply(q2, pdf)


class LumiFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, values, pdf: PDF, events, member: int, save: bool):
        from .lumi import luminosity
        pdf.bind_values(values)
        saved = None
        if save:
            saved = torch.empty((events.n, 2, pdf.n_flav), dtype=torch.float64, device=pdf.device)
        L, lum, a_s = luminosity(pdf, events, member, want_lum=False, want_alphas=False, save_p=saved)
        ctx.save_for_backward(values)
        ctx.pdf, ctx.events, ctx.member, ctx.saved = pdf, events, member, saved
        return L

    @staticmethod
    def backward(ctx, gL):
        from .lumi import luminosity_backward
        (values,) = ctx.saved_tensors
        pdf = ctx.pdf
        pdf.bind_values(values)
        gvals = torch.zeros_like(values)
        gslice = gvals[ctx.member] if values.dim() == 4 else gvals
        luminosity_backward(pdf, ctx.events, float(gL.item()), gslice, ctx.member, saved_p=ctx.saved)
        ctx.saved = None
        return gvals, None, None, None, None


def lumi(pdf: PDF, values, events, member: int = 0, save: bool = True):
    """Differentiable luminosity L(values) of the event sample.  ``save``
    keeps the partner factors of the forward pass (16 F bytes per event) so
    that the backward pass does not recompute them."""
    return LumiFn.apply(values, pdf, events, member, save)
