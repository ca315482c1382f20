"""Pins of the FP64 oracle against what the mathematics fixes (CPU only).

Each test checks the oracle against something other than itself: knot values,
closed forms (log-bilinear and quadratic data), invariants (partition of unity,
subgrid isolation, continuity), exact-rational brute force on tiny grids,
central finite differences, and special cases.
"""
import math

import numpy as np
import pytest

from oracle.bruteforce import ExactGrid, exact_alphas
from oracle.oracle import OracleGrid
from paper_2012_08221_gb300 import synth
from tests.tinygrids import fill, tiny_single, tiny_two_sub


def orc(grid):
    return OracleGrid.from_synth(grid)


@pytest.fixture(scope="module")
def small():
    return synth.grid_small()


@pytest.fixture(scope="module")
def nnpdf():
    return synth.grid_nnpdf()


# ----------------------------------------------------------- knot values

@pytest.mark.parametrize("which", ["small", "nnpdf", "tiny2"])
def test_knot_values_reproduced_exactly(which, small, nnpdf):
    g = {"small": small, "nnpdf": nnpdf, "tiny2": tiny_two_sub()}[which]
    o = orc(g)
    starts = np.concatenate([[0], np.cumsum(g.n_q)[:-1]])
    for r in range(g.n_rows):
        # a duplicated threshold knot belongs to the upper subgrid's first row
        is_lower_copy = any(r == s + n - 1 for s, n in zip(starts[:-1], g.n_q[:-1]))
        row = r + 1 if is_lower_copy else r
        for k in range(0, g.n_x, max(1, g.n_x // 17)):
            for a, pid in enumerate(g.pids):
                got = o.xfxq2(pid, g.x_knots[k], g.q_knots[r] * g.q_knots[r])
                assert got == g.values[0, row, k, a], (r, k, pid)


# ------------------------------------------------------------ closed forms

def _grid_rel(g, got, want):
    scale = np.max(np.abs(g.values)) + 1.0
    return np.max(np.abs(got - want)) / scale


def test_log_bilinear_data_reproduced_everywhere(nnpdf):
    """a + b u + c w + d u w is reproduced in range, across thresholds and
    in all four extrapolation regions (finite-difference slopes are exact on
    linear data, and the continuation is linear)."""
    a, b, c, d = 0.7, -0.31, 0.045, 0.013
    g = fill(nnpdf, lambda U, W: a + b * U + c * W + d * U * W)
    o = orc(g)
    rng = np.random.default_rng(5)
    u = rng.uniform(math.log(1e-12), 0.0, 4000)
    w = rng.uniform(math.log(0.01), math.log(1e12), 4000)
    got = np.array([o.xfxq2_uw(1, ui, wi)[0] for ui, wi in zip(u, w)])
    want = a + b * u + c * w + d * u * w
    assert _grid_rel(g, got, want) < 1e-13


def test_log_bilinear_derivatives(nnpdf):
    b, c, d = -0.31, 0.045, 0.013
    g = fill(nnpdf, lambda U, W: 0.7 + b * U + c * W + d * U * W)
    o = orc(g)
    rng = np.random.default_rng(6)
    for ui, wi in zip(rng.uniform(-25, 0, 300), rng.uniform(-3, 26, 300)):
        _, du, dw = o.xfxq2_uw(0, ui, wi)
        assert abs(du - (b + d * wi)) < 1e-12
        assert abs(dw - (c + d * ui)) < 1e-12


def test_constant_data_partition_of_unity(small):
    g = fill(small, lambda U, W: 3.25 + 0 * U * W)
    o = orc(g)
    rng = np.random.default_rng(8)
    for ui, wi in zip(rng.uniform(-20, 0, 500), rng.uniform(-1, 20, 500)):
        assert abs(o.xfxq2_uw(-3, ui, wi)[0] - 3.25) < 1e-14


def test_quadratic_in_u_interior_exact_and_edge_closed_form(small):
    """On uniformly spaced knots the mean-of-secants derivative is exact for a
    quadratic, so interior intervals reproduce u^2; the first and last
    intervals use one-sided secants with known error
    h^2 t (1-t)^2 (first) and h^2 t^2 (1-t) (last)."""
    g = fill(small, lambda U, W: U * U + 0 * W)
    o = orc(g)
    U = np.log(g.x_knots)
    h = U[1] - U[0]
    assert np.allclose(np.diff(U), h, rtol=1e-12)
    w = math.log(50.0)
    for k in range(g.n_x - 1):
        for t in (0.13, 0.5, 0.91):
            u = U[k] + t * (U[k + 1] - U[k])
            got = o.xfxq2_uw(0, u, w)[0]
            want = u * u
            if k == 0:
                want += h * h * t * (1 - t) ** 2
            elif k == g.n_x - 2:
                want += h * h * t * t * (1 - t)
            assert abs(got - want) < 1e-12 * (1 + u * u), (k, t, got, want)


def test_quadratic_in_w_interior_exact_and_edge_closed_form(small):
    g = fill(small, lambda U, W: 0 * U + W * W)
    o = orc(g)
    W = np.log(g.q_knots ** 2)
    h = W[1] - W[0]
    u = math.log(3e-3)
    n = g.n_rows
    for k in range(n - 1):
        for t in (0.2, 0.77):
            w = W[k] + t * (W[k + 1] - W[k])
            want = w * w
            if k == 0:
                want += h * h * t * (1 - t) ** 2
            elif k == n - 2:
                want += h * h * t * t * (1 - t)
            assert abs(o.xfxq2_uw(0, u, w)[0] - want) < 1e-11 * (1 + w * w), (k, t)


# -------------------------------------------------------------- invariants

def test_subgrid_isolation(nnpdf):
    """Changing rows outside the subgrid that contains w never changes the
    result (no interpolation across a threshold)."""
    o = orc(nnpdf)
    rng = np.random.default_rng(9)
    starts = np.concatenate([[0], np.cumsum(nnpdf.n_q)])
    W = np.log(nnpdf.q_knots ** 2)
    for s in range(len(nnpdf.n_q)):
        lo, hi = starts[s], starts[s + 1]
        v2 = nnpdf.values.copy()
        mask = np.ones(nnpdf.n_rows, bool)
        mask[lo:hi] = False
        v2[:, mask] += rng.uniform(-5, 5, size=v2[:, mask].shape)
        o2 = OracleGrid(nnpdf.x_knots, nnpdf.n_q, nnpdf.q_knots, nnpdf.pids, v2, nnpdf.alphas)
        # strictly inside the subgrid (the lower edge of s > 0 belongs to s)
        ws = rng.uniform(W[lo], W[hi - 1], 50)
        us = rng.uniform(-20.0, -0.01, 50)
        for u, w in zip(us, ws):
            if w == W[hi - 1] and s < len(nnpdf.n_q) - 1:
                continue
            assert o.xfxq2_uw(2, u, w)[0] == o2.xfxq2_uw(2, u, w)[0]


def test_threshold_continuity_c0(nnpdf):
    o = orc(nnpdf)
    W = np.log(nnpdf.q_knots ** 2)
    starts = np.cumsum(nnpdf.n_q)[:-1]
    for r in starts:                     # first row of each upper subgrid
        wt = W[r]
        for u in (-18.0, -7.3, -0.4):
            below = o.xfxq2_uw(-2, u, wt * (1 - 1e-13) if wt > 0 else wt - 1e-13)[0]
            at = o.xfxq2_uw(-2, u, wt)[0]
            assert abs(below - at) <= 1e-9 * (abs(at) + 1e-3)


def test_c1_inside_subgrid(small):
    """Left and right derivatives agree at interior knots (Hermite with shared
    knot derivatives); second derivatives may jump."""
    o = orc(small)
    U = np.log(small.x_knots)
    W = np.log(small.q_knots ** 2)
    d = 1e-7
    for k in (5, 20, 40):
        w = 0.5 * (W[3] + W[4])
        l = o.xfxq2_uw(1, U[k] - d, w)[1]
        r = o.xfxq2_uw(1, U[k] + d, w)[1]
        assert abs(l - r) <= 1e-4 * (abs(l) + abs(r) + 1e-6)
    for k in (3, 10, 17):
        u = 0.5 * (U[20] + U[21])
        l = o.xfxq2_uw(1, u, W[k] - d)[2]
        r = o.xfxq2_uw(1, u, W[k] + d)[2]
        assert abs(l - r) <= 1e-4 * (abs(l) + abs(r) + 1e-6)


# ----------------------------------------------------------- brute force

def _exact_for(g, o, flav):
    starts = np.concatenate([[0], np.cumsum(g.n_q)])
    Wsub = [o.W[starts[s]:starts[s + 1]] for s in range(len(g.n_q))]
    Vsub = [g.values[0, starts[s]:starts[s + 1], :, flav] for s in range(len(g.n_q))]
    return ExactGrid(o.U, Wsub, Vsub), Wsub


@pytest.mark.parametrize("make", [tiny_single, tiny_two_sub,
                                  lambda: tiny_two_sub(seed=3, dup_equal=False)])
def test_brute_force_exact_rationals(make):
    g = make()
    o = orc(g)
    rng = np.random.default_rng(12)
    U, W = o.U, o.W
    pts = [(u, w) for u, w in zip(rng.uniform(U[0] - 2, U[-1] + 0.5, 60),
                                  rng.uniform(W[0] - 1.5, W[-1] + 1.5, 60))]
    pts += [(U[k], W[r]) for k in range(len(U)) for r in range(len(W))]
    pts += [(U[0] - 0.7, W[0] - 0.9), (U[-1], W[-1]), (0.5 * (U[1] + U[2]), W[-1] + 3.0)]
    pts = [(u, w) for u, w in pts if u <= 0.0]
    for f in range(g.n_flav):
        ex, _ = _exact_for(g, o, f)
        for u, w in pts:
            v, du, dw = o.xfxq2_uw(g.pids[f], u, w)
            ev, edu, edw = ex.eval(u, w)
            assert abs(v - float(ev)) <= 1e-14 * 4.0, (u, w, v, float(ev))
            assert abs(du - float(edu)) <= 1e-12 * (1 + abs(float(edu))), (u, w)
            assert abs(dw - float(edw)) <= 1e-12 * (1 + abs(float(edw))), (u, w)


@pytest.mark.parametrize("make", [tiny_single, tiny_two_sub])
def test_alphas_brute_force(make):
    g = make()
    o = orc(g)
    starts = np.concatenate([[0], np.cumsum(g.n_q)])
    Wsub = [o.W[starts[s]:starts[s + 1]] for s in range(len(g.n_q))]
    Asub = [g.alphas[starts[s]:starts[s + 1]] for s in range(len(g.n_q))]
    rng = np.random.default_rng(4)
    for w in list(rng.uniform(o.W[0] - 2, o.W[-1] + 2, 80)) + list(o.W):
        assert abs(o.alphas_w(w) - float(exact_alphas(Wsub, Asub, w))) < 1e-15


def test_window_holds_every_nonzero_weight():
    """The oracle's short indicator scan (used for gradients and kappa) misses
    no cell: compare with a scan of every cell of a tiny grid."""
    g = tiny_two_sub()
    o = orc(g)
    rng = np.random.default_rng(13)
    x = np.exp(rng.uniform(math.log(1e-6), 0, 40))
    q2 = np.exp(rng.uniform(math.log(0.3), math.log(5000.0), 40))
    gw = rng.standard_normal(40)
    pid = np.full(40, g.pids[1], np.int32)
    got = o.dgrid_pw(pid, x, q2, gw)
    want = np.zeros_like(got)
    for i in range(40):
        for r in range(g.n_rows):
            for k in range(g.n_x):
                want[r, k, 1] += gw[i] * o.cell_weight(r, k, math.log(x[i]), math.log(q2[i]))
    assert np.max(np.abs(got - want)) < 1e-14


# ----------------------------------------------------------------- alpha_s

def test_alphas_knots_and_linear_data(nnpdf):
    o = orc(nnpdf)
    W = np.log(nnpdf.q_knots ** 2)
    starts = np.cumsum(nnpdf.n_q)[:-1]
    for r in range(nnpdf.n_rows):
        if r + 1 in starts:
            continue                   # lower copy of a threshold
        assert o.alphas_q2(nnpdf.q_knots[r] ** 2) == nnpdf.alphas[r]
    lin = OracleGrid(nnpdf.x_knots, nnpdf.n_q, nnpdf.q_knots, nnpdf.pids, nnpdf.values,
                     0.3 - 0.01 * W)
    for w in np.linspace(W[0] - 3, W[-1] + 3, 301):
        assert abs(lin.alphas_w(w) - (0.3 - 0.01 * w)) < 1e-15


def test_alphas_close_to_one_loop_and_converges(small):
    """Against the one-loop closed form the interpolation error is set by the
    finite-difference slopes: O(h^2), largest on the one-sided edge
    intervals.  Halving the knot spacing must cut it about four times."""
    def max_err(n_knots):
        qk = synth.log_knots(1.65, 1e4, n_knots)
        a = synth.alphas_one_loop(qk, nf_fixed=5)
        o = OracleGrid(small.x_knots, [n_knots], qk, small.pids,
                       np.zeros((1, n_knots, small.n_x, small.n_flav)), a)
        q = np.exp(np.linspace(math.log(1.7), math.log(9e3), 400))
        got = np.array([o.alphas_q2(v * v) for v in q])
        return np.max(np.abs(got / synth.alphas_one_loop(q, nf_fixed=5) - 1))
    e20, e39 = max_err(20), max_err(39)
    assert e20 < 5e-3
    assert 3.0 < e20 / e39 < 6.0


# --------------------------------------------------------------- gradients

def test_gradients_against_central_differences(small):
    o = orc(small)
    rng = np.random.default_rng(14)
    U = np.log(small.x_knots)
    W = np.log(small.q_knots ** 2)
    n_ok = 0
    while n_ok < 200:
        x = math.exp(rng.uniform(math.log(1e-6), math.log(0.9)))
        q2 = math.exp(rng.uniform(math.log(4), math.log(2.5e7)))
        h = 1e-6
        u, w = math.log(x), math.log(q2)
        if np.min(np.abs(U - u)) < 4 * h or np.min(np.abs(W - w)) < 4 * h:
            continue
        pid = int(rng.choice(small.pids))
        v, dx, dq2 = o.grad(pid, x, q2)
        fx = (o.xfxq2(pid, x * (1 + h), q2) - o.xfxq2(pid, x * (1 - h), q2)) / (2 * h * x)
        fq = (o.xfxq2(pid, x, q2 * (1 + h)) - o.xfxq2(pid, x, q2 * (1 - h))) / (2 * h * q2)
        assert abs(dx - fx) <= 1e-5 * (abs(dx) + abs(v) / x)
        assert abs(dq2 - fq) <= 1e-5 * (abs(dq2) + abs(v) / q2)
        n_ok += 1


def test_grid_gradient_is_linear_response(small):
    """d xf / d v[cell] from the indicator grid equals the finite response of
    the result to a change of that one value (the result is linear in v)."""
    o = orc(small)
    rng = np.random.default_rng(15)
    for _ in range(30):
        x = math.exp(rng.uniform(math.log(1e-6), math.log(0.9)))
        q2 = math.exp(rng.uniform(math.log(4), math.log(2.5e7)))
        pid = int(rng.choice(small.pids))
        a = int(np.where(small.pids == pid)[0][0])
        gw = np.array([1.0])
        G = o.dgrid_pw(np.array([pid]), np.array([x]), np.array([q2]), gw)
        nz = np.argwhere(G[:, :, a] != 0)
        assert 4 <= len(nz) <= 16
        for r, k in nz[:6]:
            v2 = small.values.copy()
            v2[0, r, k, a] += 0.5
            o2 = OracleGrid(small.x_knots, small.n_q, small.q_knots, small.pids, v2, small.alphas)
            resp = (o2.xfxq2(pid, x, q2) - o.xfxq2(pid, x, q2)) / 0.5
            assert abs(resp - G[r, k, a]) < 1e-12 * (1 + abs(G[r, k, a])) + 1e-13


# ------------------------------------------------------ domain and flavour

def test_domain_and_flavour_rules(small):
    o = orc(small)
    nan = float("nan")
    for x, q2 in [(0.0, 10.0), (-1e-3, 10.0), (1.0 + 1e-15, 10.0), (0.1, 0.0),
                  (0.1, -4.0), (nan, 10.0), (0.1, nan), (0.1, float("inf"))]:
        assert math.isnan(o.xfxq2(1, x, q2))
        assert math.isnan(o.xfxq2(99, x, q2))          # domain error dominates
    assert not math.isnan(o.xfxq2(1, 1.0, 10.0))
    assert o.xfxq2(21, 0.01, 100.0) == o.xfxq2(0, 0.01, 100.0)
    assert o.xfxq2(6, 0.01, 100.0) == 0.0              # not in an 11-flavour grid
    assert o.xfxq2(99, 0.01, 100.0) == 0.0
    assert o.xfxq2(1, 1.0, 100.0) == 0.0                # x = 1 knot carries (1-x)^beta = 0


def test_gluon_listed_as_21_on_the_grid(nnpdf):
    """A grid may list its gluon as 21 (the LHAPDF flavour line does): the
    same values under pid 0 or 21 in a query, the same luminosity (the gluon
    pairs with itself) and the same gradients as with the gluon listed as 0."""
    g0 = nnpdf
    p21 = g0.pids.copy()
    p21[p21 == 0] = 21
    g21 = synth.Grid(g0.x_knots, g0.n_q, g0.q_knots, p21, g0.values, g0.alphas, "g21")
    o0, o21 = orc(g0), orc(g21)
    x, q2, _ = synth.queries_nnpdf(2000, seed=31)
    for q in (0, 21):
        assert np.array_equal(o21.xfxq2_batch([q, 2, -1], x, q2), o0.xfxq2_batch([0, 2, -1], x, q2))
    assert np.any(o21.xfxq2_batch([21], x, q2) != 0.0)
    ev = synth.events_lhc(500, seed=32)
    L0, lum0, _ = o0.lumi(ev)
    L21, lum21, _ = o21.lumi(ev)
    assert np.array_equal(lum0, lum21) and L0 == L21
    assert np.array_equal(o0.lumi_dgrid(ev), o21.lumi_dgrid(ev))
    pid = np.where(np.arange(x.size) % 2 == 0, 21, 2).astype(np.int32)
    w = np.ones(x.size)
    assert np.array_equal(o0.dgrid_pw(pid, x, q2, w), o21.dgrid_pw(pid, x, q2, w))


# --------------------------------------------------------------- luminosity

def test_luminosity_constant_grid_closed_form(nnpdf):
    g = fill(nnpdf, lambda U, W: 0.5 + 0 * U * W)
    o = orc(g)
    ev = synth.events_lhc(200, seed=77)
    L, lum, a_s = o.lumi(ev)
    assert np.allclose(lum, g.n_flav * 0.25, rtol=0, atol=1e-14)
    assert abs(L - g.n_flav * 0.25) < 1e-14
    assert np.all(np.isfinite(a_s))


def test_luminosity_flavour_pairing_and_kinematics_closed_form(nnpdf):
    """Flavour-dependent log-bilinear data (reproduced exactly inside and
    outside the grid) make every event's luminosity and alpha_s closed forms
    of ln x1 = ln tau/2 + y, ln x2 = ln tau/2 - y, ln Q^2 = ln tau + ln s (the
    injected tail included) and of the pairing a <-> -a (gluon with itself)."""
    from tests.closed_forms import bilinear_flavour_grid, luminosity
    g, params = bilinear_flavour_grid(nnpdf)
    o = orc(g)
    ev = synth.events_lhc(4000, seed=81, tail=0.3)
    L, lum, a_s = o.lumi(ev)
    want, mag, want_as = luminosity(g.pids, params, ev)
    assert np.all(np.abs(lum - want) <= 1e-13 * mag + 1e-15)
    assert abs(L - want.mean()) <= 1e-13 * mag.mean()
    assert np.all(np.abs(a_s - want_as) <= 1e-15)
    assert np.any(ev.flags & 1) and np.any(ev.flags & 2)


def test_luminosity_gradient_central_difference():
    """L is quadratic in the values: a central difference is exact (up to
    rounding) and must equal the oracle's analytic grid gradient."""
    g = tiny_two_sub(n_flav=3)
    o = orc(g)
    ev = synth.events_lhc(40, seed=78)
    ev.ln_tau[:] = np.random.default_rng(1).uniform(math.log(1e-5), 0, 40)
    ev.y[:] = 0.3 * ev.ln_tau * np.random.default_rng(2).uniform(-1, 1, 40)
    G = o.lumi_dgrid(ev)
    for (r, k, b) in [(0, 1, 0), (2, 3, 1), (4, 2, 2), (5, 4, 1), (1, 0, 2)]:
        d = 0.25
        vp = g.values.copy(); vp[0, r, k, b] += d
        vm = g.values.copy(); vm[0, r, k, b] -= d
        Lp = OracleGrid(g.x_knots, g.n_q, g.q_knots, g.pids, vp, g.alphas).lumi(ev)[0]
        Lm = OracleGrid(g.x_knots, g.n_q, g.q_knots, g.pids, vm, g.alphas).lumi(ev)[0]
        assert abs((Lp - Lm) / (2 * d) - G[r, k, b]) < 1e-12 * (1 + abs(G[r, k, b]))


# --------------------------------------------------------- golden fixture

def test_golden_tiny_exact_values():
    """tests/golden/tiny_exact.txt holds exact-rational values written by
    make_golden.py from the brute force; the oracle must agree to rounding."""
    from tests.golden_io import load
    g, x, q2, exp, exp_as = load()
    o = orc(g)
    got = o.xfxq2_batch(g.pids, x, q2)
    assert np.max(np.abs(got - exp)) < 1e-14
    assert np.max(np.abs(o.alphas_batch(q2) - exp_as)) < 1e-15


def test_alphas_derivative_against_central_differences(nnpdf):
    o = orc(nnpdf)
    W = np.log(nnpdf.q_knots ** 2)
    rng = np.random.default_rng(60)
    n_ok = 0
    while n_ok < 200:
        w = rng.uniform(W[0] - 2, W[-1] + 2)
        if np.min(np.abs(W - w)) < 1e-5:
            continue
        q2, h = math.exp(w), 1e-7
        v, d = o.alphas_grad(q2)
        fd = (o.alphas_q2(q2 * (1 + h)) - o.alphas_q2(q2 * (1 - h))) / (2 * h * q2)
        assert abs(d - fd) <= 1e-6 * (abs(d) + abs(v) / q2)
        n_ok += 1
