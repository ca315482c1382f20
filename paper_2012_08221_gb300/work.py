"""Algorithmic work per unit of each kernel: the numerators of the roofline.

FP64 flops count a fused multiply-add as 2 and an add or multiply as 1; they
are the operations the method needs in the formulation the kernels use
(bicubic patch coefficients, table-driven log), not instruction counts
measured on the GPU.  Bytes are the compulsory HBM traffic: inputs read once
and outputs written once (the grid tables are cache-resident parameters).

Per point of the x*f kernel with F flavours:
  2 logs x 15 flops (1 FMA reduction, 4 FMA series, 1 multiply, 4 adds),
  2 axes x (subtract, multiply) for t, 15 FMA per flavour for the
  16-coefficient patch by Horner's rule:  34 + 30 F flops.
"""
from __future__ import annotations

LOG_FLOPS = 15
AXIS_FLOPS = 2          # t = (ln z - Z) * (1/dZ)
POWER_FLOPS = 2         # t^2, t^3 (adjoint kernels only)
PATCH_FLOPS = 30        # 15 FMA


def xfxq2_point_flops(n_flav: int) -> int:
    return 2 * LOG_FLOPS + 2 * AXIS_FLOPS + PATCH_FLOPS * n_flav


def xfxq2_point_flops_matrix_form(n_flav: int) -> int:
    """The same point counted in the separable-weight (matrix) form of the
    method: per axis 4 Hermite weights from the basis and the
    finite-difference coefficients (about 50 flops for both axes), then per
    flavour the contraction sum_j Wq_j sum_i Wx_i v_ij, 20 FMA; the two logs
    counted apart.  The kernels evaluate the same interpolant from
    precomputed patch coefficients in 15 FMA per flavour, so this count is
    larger than the work they do: a fraction on it can exceed 1."""
    return 40 * n_flav + 50


def xfxq2_point_bytes(n_flav: int) -> int:
    return 16 + 8 * n_flav            # x, Q^2 in; F outputs


def alphas_point_flops() -> int:
    return LOG_FLOPS + AXIS_FLOPS + 6  # 3 FMA for the cubic


ALPHAS_POINT_BYTES = 16


PATCH_D_FLOPS = 52      # the two patch derivatives alone: 26 FMA (patch_vd without the value)
PATCH_VD_EXTRA_FLOPS = 26  # the two derivatives beside the value: 13 FMA


def pw_fwd_point_flops(dtape: bool = False) -> int:
    """One pointwise forward point; with the derivative tape the patch's two
    derivatives are computed with its value (13 FMA more)."""
    return xfxq2_point_flops(1) + (PATCH_VD_EXTRA_FLOPS if dtape else 0)


PW_FWD_POINT_BYTES = 28                # x, Q^2, pid, out


PW_BWD_POINT_BYTES = 44                # grad_out, x, Q^2, pid in; dx, dQ^2 out


TAPE_POINT_BYTES = 32                  # written by the forward, read by the adjoint


def pw_bwd_sorted_point_flops(dtape: bool = False) -> int:
    """The pointwise adjoint as the kernels now run it (from the tape, grid
    gradient sorted by (cell, flavour)).  Record pass: the patch's tx- and
    tq-derivatives by Horner's rule (rows 1-3: 5 FMA each, row 0: 4, the Q
    step: 4, the tx-derivative over the rows: 3; 26 FMA), unless the
    forward kept them in the derivative tape, and the chain rule to x and
    Q^2 (3 multiplies and a reciprocal each).  Accumulation: g times the Q
    basis and the x basis (6 multiplies) and the 16 FMAs of g bq_n bx_m.
    The map back to the stencil values (8 FMA per lane per bin run) is per
    bin, not per point, and is not counted."""
    chain = 2 * 4
    record = chain if dtape else PATCH_D_FLOPS + chain
    accumulate = 6 + 2 * 16
    return record + accumulate


def pw_bwd_point_flops_separable() -> int:
    """The backward work of one pointwise point in the separable-weight count
    of the method (derivative weights of both axes, the contraction and its
    derivatives, and the 16-weight scatter into the grid: about 170)."""
    return 170


def pw_fwd_bwd_point_flops_separable() -> int:
    """The forward plus backward work of one pointwise point in the
    separable-weight count of the method (forward 90, backward about 170)."""
    return 90 + pw_bwd_point_flops_separable()


def lumi_event_flops(n_flav: int) -> int:
    """Kinematics (1 multiply, 3 adds), t for 3 axes, 2 F patches,
    F FMA for the flavour-paired sum, alpha_s cubic (3 FMA), 1 add to the
    running sum."""
    return 4 + 3 * AXIS_FLOPS + 2 * PATCH_FLOPS * n_flav + 2 * n_flav + 6 + 1


LUMI_EVENT_BYTES = 8 + 8 + 1 + 16      # ln tau, y, flags in; lum, alpha_s out


def lumi_bwd_event_flops(n_flav: int, saved: bool = False) -> int:
    """Adjoint of one event, as the kernels organise it: the kinematics and
    3 axes, the 2 F patch values (the partner factors; skipped when the
    forward pass saved them), then per parton the products of the powers of
    its two near-knot coordinates (4 multiplies for the powers, 9 for the
    products) and 16 F FMAs into its bin's accumulators.  The map back per
    bin run, and the stencil weights of the few partons outside the knot
    range, are not counted."""
    per_parton = 4 + 9 + 16 * n_flav * 2
    patches = 0 if saved else 2 * PATCH_FLOPS * n_flav
    return 4 + 3 * (AXIS_FLOPS + POWER_FLOPS) + patches + 2 * per_parton


LUMI_BWD_EVENT_BYTES = 8 + 8 + 1


def vegas_point_flops(n_flav: int) -> int:
    """One VEGAS point of the luminosity integral: the map of 2 dimensions
    (multiply, subtract, FMA, width difference, Jacobian multiply: 6 each),
    the kinematics (5), t for 3 axes, 2 F patches and F FMAs for the luminosity, the
    weight (3 multiplies) and its sums (add, FMA)."""
    return 2 * 6 + 5 + 3 * AXIS_FLOPS + 2 * PATCH_FLOPS * n_flav + 2 * n_flav + 3 + 3
