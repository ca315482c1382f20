"""Pins of the oracle's VEGAS pieces (CPU): the integrand through an identity
map against its closed form on a constant grid, the refinement's fixed point
and its equal-share rule, and variance reduction on a real-shaped grid."""
import math

import numpy as np

from oracle.oracle import OracleGrid, vegas_refine, vegas_sums
from paper_2012_08221_gb300 import synth
from tests.tinygrids import fill

LN_TAU_MIN = math.log(1e-6)
LN_S = 2 * math.log(13000.0)


def test_identity_map_on_constant_grid_is_the_closed_form():
    """With uniform edges w_i = F(v_i) = (ln tau_min)^2 (1 - v_i0) n_pairs c^2."""
    g = fill(synth.grid_nnpdf(), lambda U, W: 0.75 + 0 * U * W)
    o = OracleGrid.from_synth(g)
    v = np.random.default_rng(1).uniform(0, 1, (4000, 2))
    edges = np.tile(np.linspace(0, 1, 21), (2, 1))
    s = vegas_sums(o, 0, LN_TAU_MIN, LN_S, edges, v)
    per = LN_TAU_MIN ** 2 * g.n_flav * 0.75 ** 2
    want = per * np.sum(1.0 - v[:, 0])
    assert abs(s[0] - want) <= 1e-12 * abs(want)
    assert abs(s[1] - per ** 2 * np.sum((1.0 - v[:, 0]) ** 2)) <= 1e-12 * s[1]
    # per-bin sums of w^2 add up to sum w^2 in each dimension
    assert abs(s[2:22].sum() - s[1]) <= 1e-12 * s[1]
    assert abs(s[22:42].sum() - s[1]) <= 1e-12 * s[1]
    # and the exact integral (ln tau_min)^2 n_pairs c^2 / 2 within 4 sigma
    n = v.shape[0]
    mean = s[0] / n
    sig = math.sqrt((s[1] / n - mean ** 2) / (n - 1))
    assert abs(mean - per / 2) < 4 * sig


def test_refinement_fixed_point_and_equal_shares():
    e = np.linspace(0, 1, 11)
    assert np.allclose(vegas_refine(np.full(10, 3.0), 1.5, e), e, atol=1e-15)
    rng = np.random.default_rng(2)
    old = np.concatenate([[0.0], np.sort(rng.uniform(0, 1, 9)), [1.0]])
    w2 = np.exp(-np.arange(10) / 2.0) * 7.0
    new = vegas_refine(w2, 1.5, old)
    assert new[0] == 0.0 and new[-1] == 1.0 and np.all(np.diff(new) > 0)
    # damped weights of the smoothed sums (definition), cumulated over the old
    # bins with each bin's share spread uniformly over its width
    sm = np.empty(10)
    sm[0], sm[-1] = (w2[0] + w2[1]) / 2, (w2[-2] + w2[-1]) / 2
    sm[1:-1] = (w2[:-2] + w2[1:-1] + w2[2:]) / 3
    d = sm / sm.sum()
    r = ((1 - d) / np.log(1 / d)) ** 1.5
    cum = np.concatenate([[0.0], np.cumsum(r)])
    share = np.interp(new, old, cum)
    assert np.allclose(share, np.arange(11) * r.sum() / 10, rtol=0, atol=1e-12 * r.sum())
    # more resolution where w^2 is large: the first new bin is narrower
    assert new[1] - new[0] < old[1] - old[0] or new[1] < 0.1


def test_adaptation_reduces_the_variance():
    g = synth.grid_nnpdf()
    o = OracleGrid.from_synth(g)
    rng = np.random.default_rng(3)
    edges = np.tile(np.linspace(0, 1, 31), (2, 1))
    sig = []
    for it in range(4):
        v = rng.uniform(0, 1, (6000, 2))
        s = vegas_sums(o, 0, LN_TAU_MIN, LN_S, edges, v)
        n = v.shape[0]
        m = s[0] / n
        sig.append(math.sqrt(s[1] / n - m * m) / m)
        for dmn in range(2):
            edges[dmn] = vegas_refine(s[2 + 30 * dmn: 32 + 30 * dmn], 1.5, edges[dmn])
    assert sig[-1] < 0.7 * sig[0]


def test_non_uniform_map_midpoint_rule_is_exact():
    """On a constant grid the integrand depends on r1 only, linearly, so
    through any piecewise-linear map the weight w(v) = F(r(v)) J(v) is linear
    in v inside every bin: a midpoint lattice with a whole number of points
    per bin integrates it exactly.  With random non-uniform edges the mean
    weight must equal the integral (ln tau_min)^2 n_pairs c^2 / 2, which pins
    the bin index, the position inside the bin and the Jacobian."""
    g = fill(synth.grid_nnpdf(), lambda U, W: 0.75 + 0 * U * W)
    o = OracleGrid.from_synth(g)
    nb = 20
    rng = np.random.default_rng(4)
    edges = np.stack([np.concatenate([[0.0], np.sort(rng.uniform(0, 1, nb - 1)), [1.0]]) for _ in range(2)])
    N, M = 5 * nb, 3 * nb
    v0 = (np.arange(N) + 0.5) / N
    v1 = (np.arange(M) + 0.5) / M
    v = np.stack(np.meshgrid(v0, v1, indexing="ij"), axis=-1).reshape(-1, 2)
    s = vegas_sums(o, 0, LN_TAU_MIN, LN_S, edges, v)
    per = LN_TAU_MIN ** 2 * g.n_flav * 0.75 ** 2
    assert abs(s[0] / v.shape[0] - per / 2) <= 1e-12 * per
    assert abs(s[2:2 + nb].sum() - s[1]) <= 1e-12 * s[1]
    assert abs(s[2 + nb:].sum() - s[1]) <= 1e-12 * s[1]
