"""Pins of the oracle's VEGAS pieces (CPU): the integrand through an identity
map against its closed form on a constant grid, the refinement's fixed point
and its equal-share rule, and variance reduction on a real-shaped grid."""
import math

import numpy as np

from oracle.oracle import OracleGrid, vegas_accumulate, vegas_map, vegas_refine, vegas_sums
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


def test_general_map_midpoint_lattice_is_exact_for_multilinear_integrands():
    """Any dimension: through random non-uniform edges, f(r) = prod_d (a_d +
    b_d r_d) times the Jacobian is multilinear in v inside every bin cell, so
    a midpoint lattice with whole numbers of points per bin integrates it
    exactly: mean weight = prod_d (a_d + b_d / 2)."""
    rng = np.random.default_rng(5)
    dim, nb = 3, 8
    edges = np.stack([np.concatenate([[0.0], np.sort(rng.uniform(0, 1, nb - 1)), [1.0]]) for _ in range(dim)])
    m = (2 * nb, 3 * nb, nb)
    axes = [(np.arange(k) + 0.5) / k for k in m]
    v = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, dim)
    r, jac, bins = vegas_map(edges, v)
    a, b = np.array([0.5, 2.0, -1.0]), np.array([1.5, -0.7, 3.0])
    w = np.prod(a + b * r, axis=1) * jac
    s = vegas_accumulate(nb, w, bins)
    assert abs(s[0] / v.shape[0] - np.prod(a + b / 2)) <= 1e-12
    for d in range(dim):
        assert abs(s[2 + d * nb: 2 + (d + 1) * nb].sum() - s[1]) <= 1e-12 * s[1]
        # r stays in the bin the point was counted in
        lo, hi = edges[d][bins[:, d]], edges[d][bins[:, d] + 1]
        assert np.all((r[:, d] >= lo) & (r[:, d] <= hi))


def test_general_map_and_accumulate_reproduce_the_fused_luminosity_sums():
    """The fused luminosity iteration equals map -> the luminosity integrand
    computed outside (events built from r, the oracle's luminosity) ->
    accumulate: two independent routes through the oracle."""
    g = synth.grid_nnpdf()
    o = OracleGrid.from_synth(g)
    rng = np.random.default_rng(6)
    nb = 25
    edges = np.stack([np.concatenate([[0.0], np.sort(rng.uniform(0, 1, nb - 1)), [1.0]]) for _ in range(2)])
    v = rng.uniform(0, 1, (3000, 2))
    fused = vegas_sums(o, 0, LN_TAU_MIN, LN_S, edges, v)
    r, jac, bins = vegas_map(edges, v)
    ln_tau = (1.0 - r[:, 0]) * LN_TAU_MIN
    y = (2.0 * r[:, 1] - 1.0) * (-0.5 * ln_tau)
    n = v.shape[0]
    ev = synth.Events(ln_tau, y, np.zeros(n, np.uint8), np.zeros(n), np.zeros(n), LN_S)
    _, lum, _ = o.lumi(ev)
    w = (-LN_TAU_MIN) * (-ln_tau) * lum * jac
    split = vegas_accumulate(nb, w, bins)
    assert np.allclose(split, fused, rtol=1e-13, atol=0)


def test_second_moment_about_a_shift():
    """sum (w - c)^2 is the exactly rounded sum of the squared deviations,
    and for the fused luminosity it obeys the identity
    sum (w - c)^2 = sum w^2 - 2 c sum w + n c^2 (to rounding)."""
    rng = np.random.default_rng(5)
    w = rng.standard_normal(20_000) * 3.0 + 7.0
    bins = rng.integers(0, 16, (w.size, 2)).astype(np.int32)
    for c in (0.0, 7.0, -2.5):
        s = vegas_accumulate(16, w, bins, shift=c)
        want = math.fsum((w - c) ** 2)
        assert abs(s[1] - want) <= 1e-13 * want
        assert abs(s[0] - math.fsum(w)) <= 1e-13 * math.fsum(np.abs(w))
        # the per-bin sums stay sums of w^2 whatever the shift
        assert np.array_equal(s[2:], vegas_accumulate(16, w, bins)[2:])
    o = OracleGrid.from_synth(synth.grid_nnpdf())
    v = rng.uniform(0, 1, (3000, 2))
    edges = np.tile(np.linspace(0, 1, 11), (2, 1))
    s0 = vegas_sums(o, 0, LN_TAU_MIN, LN_S, edges, v)
    c = s0[0] / v.shape[0]
    sc = vegas_sums(o, 0, LN_TAU_MIN, LN_S, edges, v, shift=c)
    assert sc[0] == s0[0] and np.array_equal(sc[2:], s0[2:])
    assert abs(sc[1] - (s0[1] - 2 * c * s0[0] + v.shape[0] * c * c)) <= 1e-10 * s0[1]
    assert sc[1] < 0.9 * s0[1]


def test_variance_of_a_nearly_flat_integrand():
    """Weights 1 + 1e-7 g: about the mean, the variance comes out to full
    precision (against a two-pass sum of exact deviations); about 0 it is
    the difference of two sums of ~1 that agree to 1e-14, and is lost."""
    rng = np.random.default_rng(6)
    n = 200_000
    w = 1.0 + 1e-7 * np.sin(2 * np.pi * rng.uniform(0, 1, n))
    bins = np.zeros((n, 1), dtype=np.int32)
    mean = math.fsum(w) / n
    exact = math.fsum((w - mean) ** 2) / n
    s = vegas_accumulate(4, w, bins, shift=mean)
    assert abs((s[1] / n - (s[0] / n - mean) ** 2) - exact) <= 1e-9 * exact
    s = vegas_accumulate(4, w, bins, shift=1.0)          # a shift near, not at, the mean
    assert abs((s[1] / n - (s[0] / n - 1.0) ** 2) - exact) <= 1e-6 * exact
