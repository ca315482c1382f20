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
