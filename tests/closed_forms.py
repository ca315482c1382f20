"""Grids whose interpolation has a closed form, and that closed form.

Every flavour a holds its own log-bilinear data f_a(u, w) = p_a + q_a u + r_a w
and alpha_s knots are linear in w.  The interpolant reproduces such data
exactly (to rounding) inside and outside the knot range, whatever the
interpolation details, so the luminosity of an event is a closed form of
its kinematics and of the flavour pairing."""
from __future__ import annotations

import numpy as np

from paper_2012_08221_gb300 import synth


def bilinear_flavour_grid(g: synth.Grid, seed: int = 80):
    rng = np.random.default_rng(seed)
    F = g.n_flav
    p, q, r = rng.uniform(-1, 1, F), rng.uniform(-0.2, 0.2, F), rng.uniform(-0.05, 0.05, F)
    U = np.log(g.x_knots)
    W = np.log(g.q_knots * g.q_knots)
    vals = p[None, None, :] + q[None, None, :] * U[None, :, None] + r[None, None, :] * W[:, None, None]
    v = np.broadcast_to(vals[None], g.values.shape).copy()
    a0, a1 = 0.2, -0.004
    grid = synth.Grid(g.x_knots, g.n_q, g.q_knots, g.pids, v, a0 + a1 * W, g.name + "-bilinear")
    return grid, (p, q, r, a0, a1)


def event_coordinates(ev: synth.Events):
    """(u1, u2, w) of each event: ln x1,2 = ln tau / 2 +- y and ln Q^2 =
    ln tau + ln s, with the injected tail (flag bit 0: ln Q^2 = ln mu^2, bit 1:
    ln x1 replaced)."""
    h = 0.5 * ev.ln_tau
    u1 = np.where(ev.flags & 2, ev.ln_x1, h + ev.y)
    u2 = h - ev.y
    w = np.where(ev.flags & 1, ev.ln_mu2, ev.ln_tau + ev.ln_s)
    return u1, u2, w


def luminosity(pids, params, ev: synth.Events):
    """Per event sum_a f_a(x1) f_-a(x2) (-0 = 0), the sum of |terms|, and
    alpha_s, for the grid of ``bilinear_flavour_grid``."""
    p, q, r, a0, a1 = params
    u1, u2, w = event_coordinates(ev)
    col = {int(pid): a for a, pid in enumerate(pids)}
    lum = np.zeros_like(w)
    mag = np.zeros_like(w)
    for a, pid in enumerate(pids):
        b = col.get(-int(pid))
        if b is None:
            continue
        t = (p[a] + q[a] * u1 + r[a] * w) * (p[b] + q[b] * u2 + r[b] * w)
        lum += t
        mag += np.abs(t)
    return lum, mag, a0 + a1 * w
