"""Pins of the oracle's interpolation kinds and extrapolation modes (CPU):
log-bilinear, log-bicubic with straight lines on small subgrids, values
frozen at the edge, NaN outside."""
import math

import numpy as np
import pytest

from oracle.bruteforce import ExactGrid
from oracle.oracle import OracleGrid
from paper_2012_08221_gb300 import synth
from tests.tinygrids import fill, tiny_two_sub


def orc(g, interp=0, extrap=0):
    return OracleGrid.from_synth(g, interp=interp, extrap=extrap)


def _exact(g, o, f, interp, extrap):
    starts = np.concatenate([[0], np.cumsum(g.n_q)])
    Wsub = [o.W[starts[s]:starts[s + 1]] for s in range(len(g.n_q))]
    Vsub = [g.values[0, starts[s]:starts[s + 1], :, f] for s in range(len(g.n_q))]
    return ExactGrid(o.U, Wsub, Vsub, interp, extrap)


@pytest.mark.parametrize("interp,extrap", [(1, 0), (2, 0), (0, 1), (1, 1), (2, 1)])
def test_modes_against_exact_brute_force(interp, extrap):
    g = tiny_two_sub(seed=21, dup_equal=False)       # subgrids of 3 knots
    o = orc(g, interp, extrap)
    rng = np.random.default_rng(22)
    U, W = o.U, o.W
    pts = list(zip(rng.uniform(U[0] - 2, 0.0, 80), rng.uniform(W[0] - 1.5, W[-1] + 1.5, 80)))
    pts += [(U[k], W[r]) for k in range(len(U)) for r in range(len(W))]
    for f in range(g.n_flav):
        ex = _exact(g, o, f, interp, extrap)
        for u, w in pts:
            v, du, dw = o.xfxq2_uw(g.pids[f], u, w)
            ev, edu, edw = ex.eval(u, w)
            assert abs(v - float(ev)) <= 4e-14, (u, w)
            assert abs(du - float(edu)) <= 1e-12 * (1 + abs(float(edu)))
            assert abs(dw - float(edw)) <= 1e-12 * (1 + abs(float(edw)))


def test_bilinear_reproduces_bilinear_data_and_averages_corners():
    g0 = synth.grid_nnpdf()
    g = fill(g0, lambda U, W: 0.3 - 0.2 * U + 0.07 * W + 0.01 * U * W)
    o = orc(g, interp=1)
    rng = np.random.default_rng(23)
    for u, w in zip(rng.uniform(-25, 0, 300), rng.uniform(-2, 25, 300)):
        assert abs(o.xfxq2_uw(0, u, w)[0] - (0.3 - 0.2 * u + 0.07 * w + 0.01 * u * w)) < 1e-12
    og = orc(g0, interp=1)
    U, W = og.U, og.W
    for k, r in [(3, 2), (100, 15), (190, 44)]:
        uc, wc = 0.5 * (U[k] + U[k + 1]), 0.5 * (W[r] + W[r + 1])
        want = 0.25 * sum(g0.values[0, rr, kk, 4] for rr in (r, r + 1) for kk in (k, k + 1))
        assert abs(og.xfxq2_uw(g0.pids[4], uc, wc)[0] - want) < 1e-13 * (1 + abs(want))


def test_small_subgrid_fallback_is_linear_only_where_knots_are_few():
    g = tiny_two_sub(seed=24)                        # both subgrids have 3 knots
    o2, o0, o1 = orc(g, 2), orc(g, 0), orc(g, 1)
    rng = np.random.default_rng(25)
    for u, w in zip(rng.uniform(o0.U[0], 0, 50), rng.uniform(o0.W[0], o0.W[-1], 50)):
        # x has 5 knots (cubic), Q subgrids 3 knots (straight) -> differs from both
        v2 = o2.xfxq2_uw(0, u, w)[0]
        assert v2 != o0.xfxq2_uw(0, u, w)[0] or v2 == o1.xfxq2_uw(0, u, w)[0]
    big = synth.grid_small()                         # 50 x 20 knots: no axis is small
    a, b = orc(big, 2), orc(big, 0)
    for u, w in zip(rng.uniform(-16, 0, 50), rng.uniform(1, 18, 50)):
        assert a.xfxq2_uw(1, u, w)[0] == b.xfxq2_uw(1, u, w)[0]


def test_freeze_and_error_outside():
    g = synth.grid_small()
    of, oe, ol = orc(g, 0, 1), orc(g, 0, 2), orc(g, 0, 0)
    U, W = ol.U, ol.W
    for u, w in [(U[0] - 3, 10.0), (-0.5, W[0] - 2), (U[0] - 1, W[-1] + 4), (-2.0, W[-1] + 1)]:
        cu, cw = min(max(u, U[0]), U[-1]), min(max(w, W[0]), W[-1])
        v, du, dw = of.xfxq2_uw(2, u, w)
        assert v == ol.xfxq2_uw(2, cu, cw)[0]
        if cu != u:
            assert du == 0.0
        if cw != w:
            assert dw == 0.0
        assert math.isnan(oe.xfxq2_uw(2, u, w)[0])
        assert math.isnan(oe.alphas_w(w)) == (cw != w)
    for u, w in [(-3.0, 10.0), (-10.0, 4.0)]:          # inside: all modes agree
        assert of.xfxq2_uw(2, u, w)[0] == oe.xfxq2_uw(2, u, w)[0] == ol.xfxq2_uw(2, u, w)[0]
    assert of.alphas_w(W[-1] + 5) == ol.alphas_w(W[-1])


# ------------------------------------------------ power-law continuation (3)

def _edge_grid():
    """x knots log-spaced in [1e-6, 0.5] (so that x above the grid exists),
    two Q subgrids [1.5, 5] and [5, 100] GeV (threshold knot duplicated)."""
    x = np.exp(np.linspace(math.log(1e-6), math.log(0.5), 30))
    q = np.concatenate([np.exp(np.linspace(math.log(1.5), math.log(5.0), 6)),
                        np.exp(np.linspace(math.log(5.0), math.log(100.0), 8))])
    nq = np.array([6, 8], dtype=np.int32)
    pids = np.array([-1, 0, 1], dtype=np.int32)
    v = np.zeros((1, q.size, x.size, 3))
    return synth.Grid(x, nq, q, pids, v, np.full(q.size, 0.2), "edges")


def _with_values(g, fn, alphas=None):
    U = np.log(g.x_knots)
    W = np.log(g.q_knots * g.q_knots)
    vals = fn(U[None, :], W[:, None])
    v = np.broadcast_to(vals[None, :, :, None], g.values.shape).copy()
    return synth.Grid(g.x_knots, g.n_q, g.q_knots, g.pids, v, g.alphas if alphas is None else alphas(W), g.name)


def test_continuation_reproduces_power_laws_outside():
    """Data c exp(a u + b w) are power laws in x and Q^2: the continuation
    reproduces them exactly (to rounding) outside the grid along knot rows
    and columns and in all four corners; alpha_s knots c_s exp(b_s w) too."""
    c, a, b = 2.0, -0.3, 0.05
    f = lambda u, w: c * np.exp(a * u + b * w)
    g = _with_values(_edge_grid(), f, alphas=lambda W: 0.3 * np.exp(-0.02 * W))
    o = orc(g, 0, 3)
    U, W = o.U, o.W
    pts = [(u, W[r]) for u in (U[0] - 3.0, U[0] - 0.2, U[-1] + 0.4) for r in (0, 3, 5, 6, 10, 13)]
    pts += [(U[k], w) for w in (W[0] - 2.5, W[0] - 0.1, W[-1] + 0.3, W[-1] + 4.0) for k in (0, 7, 29)]
    pts += [(u, w) for u in (U[0] - 2.0, U[-1] + 0.5) for w in (W[0] - 1.5, W[-1] + 2.0)]
    for u, w in pts:
        v = o.xfxq2_uw(0, u, w)[0]
        assert abs(v - f(u, w)) <= 1e-12 * f(u, w), (u, w)
    for w in (W[0] - 3.0, W[-1] + 3.0):
        assert abs(o.alphas_w(w) - 0.3 * math.exp(-0.02 * w)) <= 1e-13


def test_continuation_inside_equals_linear_and_falls_back_where_not_positive():
    """Inside the grid the options agree bit for bit.  Outside, with the two
    edge values y0, y1 (the linear option's values at the edge knots), the
    result is y0^(1-t) y1^t when both exceed 1e-3 and the linear option's
    value otherwise (synthetic values change sign near the Q edges)."""
    g = synth.grid_nnpdf()
    oc, ol = orc(g, 0, 3), orc(g, 0, 0)
    U, W = ol.U, ol.W
    rng = np.random.default_rng(31)
    for u, w in zip(rng.uniform(U[0], 0.0, 200), rng.uniform(W[0], W[-1], 200)):
        p = int(rng.choice(g.pids))
        assert oc.xfxq2_uw(p, u, w)[0] == ol.xfxq2_uw(p, u, w)[0]
    n_pow = n_lin = 0
    for _ in range(400):
        p = int(rng.choice(g.pids))
        if rng.uniform() < 0.5:           # u below the grid, w inside
            u, w = rng.uniform(U[0] - 4, U[0]), rng.uniform(W[0], W[-1])
            y0, y1 = ol.xfxq2_uw(p, U[0], w)[0], ol.xfxq2_uw(p, U[1], w)[0]
            t = (u - U[0]) / (U[1] - U[0])
        else:                             # w outside, u inside
            u = rng.uniform(U[0], 0.0)
            lo = rng.uniform() < 0.5
            w = rng.uniform(W[0] - 3, W[0]) if lo else rng.uniform(W[-1], W[-1] + 3)
            r = 0 if lo else len(W) - 2
            y0, y1 = ol.xfxq2_uw(p, u, W[r])[0], ol.xfxq2_uw(p, u, W[r + 1])[0]
            t = (w - W[r]) / (W[r + 1] - W[r])
        got = oc.xfxq2_uw(p, u, w)[0]
        if y0 > 1e-3 and y1 > 1e-3:
            want = y0 ** (1 - t) * y1 ** t
            assert abs(got - want) <= 1e-12 * want
            n_pow += 1
        else:
            assert got == ol.xfxq2_uw(p, u, w)[0]
            n_lin += 1
    assert n_pow > 50 and n_lin > 20


def test_continuation_derivatives_against_central_differences():
    g = synth.grid_nnpdf()
    o = orc(g, 0, 3)
    U, W = o.U, o.W
    rng = np.random.default_rng(32)
    h = 1e-6
    for _ in range(100):
        p = int(rng.choice(g.pids))
        u = rng.uniform(U[0] - 3, U[0] - 0.01) if rng.uniform() < 0.5 else rng.uniform(U[0] + 0.01, -0.01)
        w = rng.uniform(W[-1] + 0.01, W[-1] + 3) if rng.uniform() < 0.5 else rng.uniform(W[0] - 3, W[0] - 0.01)
        v, du, dw = o.xfxq2_uw(p, u, w)
        fu = (o.xfxq2_uw(p, u + h, w)[0] - o.xfxq2_uw(p, u - h, w)[0]) / (2 * h)
        fw = (o.xfxq2_uw(p, u, w + h)[0] - o.xfxq2_uw(p, u, w - h)[0]) / (2 * h)
        assert abs(du - fu) <= 1e-6 * (abs(du) + abs(v) + 1e-3)
        assert abs(dw - fw) <= 1e-6 * (abs(dw) + abs(v) + 1e-3)
