"""Pins of the oracle's tolerance scales (CPU only).

Every GPU parity test judges an output on the scale
max(|oracle|, kappa), where kappa is the sum of |weight * value| over the
values the interpolation combines (the reading of the tolerance for results
that vanish by cancellation), and every gradient test on the matching sum of
|term|.  These scales come from the oracle (`orc_kappa_batch`,
`orc_alphas_kappa_batch` and the `absval` modes of `orc_dgrid_pw`,
`orc_dgrid_batch` and `orc_lumi_dgrid`), so a mistake there would loosen the
whole GPU suite without failing it.  They are pinned here against what the
definition fixes:

* at a knot one weight is exactly 1 and the others exactly 0, so kappa is the
  magnitude of the result itself;
* everywhere (inside, at thresholds, outside on every side) the weights are
  those of the exact-rational brute force (`oracle/bruteforce.py`) evaluated
  on the indicator grid of each value (the interpolant is linear in the
  values, PDFFlow Sec. 2.1 with the LHAPDF algorithms of Sec. 4), so kappa
  and the |term| sums must equal the sums built from those exact weights.
"""
import math

import numpy as np
import pytest

from oracle.bruteforce import ExactGrid, exact_alphas
from oracle.oracle import OracleGrid
from paper_2012_08221_gb300 import synth
from tests.tinygrids import tiny_single, tiny_two_sub


def two_members(g, seed):
    """The grid with a second member of independent random values."""
    rng = np.random.default_rng(seed)
    v = np.concatenate([g.values, rng.uniform(-1.0, 2.0, g.values.shape)], axis=0)
    return synth.Grid(g.x_knots, g.n_q, g.q_knots, g.pids, v, g.alphas, g.name + "m2")


def _starts(g):
    return np.concatenate([[0], np.cumsum(g.n_q)]).astype(int)


def exact_weights(g, o, u, w):
    """W[r][k]: weight of grid value (row r, x knot k) at (u, w), from the
    brute force evaluated on the indicator grid of that value."""
    st = _starts(g)
    wsub = [o.W[st[s]:st[s + 1]] for s in range(len(g.n_q))]
    out = np.zeros((g.n_rows, g.n_x))
    for r in range(g.n_rows):
        s = int(np.searchsorted(st, r, side="right") - 1)
        for k in range(g.n_x):
            vals = [np.zeros((int(n), g.n_x)) for n in g.n_q]
            vals[s][r - st[s], k] = 1.0
            out[r, k] = float(ExactGrid(o.U, wsub, vals).eval(u, w)[0])
    return out


def exact_alphas_weights(g, o, w):
    st = _starts(g)
    wsub = [o.W[st[s]:st[s + 1]] for s in range(len(g.n_q))]
    out = np.zeros(g.n_rows)
    for r in range(g.n_rows):
        a = np.zeros(g.n_rows)
        a[r] = 1.0
        out[r] = float(exact_alphas(wsub, [a[st[s]:st[s + 1]] for s in range(len(g.n_q))], w))
    return out


def _points(g, o, n, seed):
    """(x, Q^2) inside, on thresholds and outside on every side and corner."""
    rng = np.random.default_rng(seed)
    U, W = o.U, o.W
    u = list(rng.uniform(U[0] - 1.5, U[-1], n))
    w = list(rng.uniform(W[0] - 1.5, W[-1] + 1.5, n))
    st = _starts(g)
    for s in range(1, len(g.n_q)):                 # internal thresholds
        u.append(float(rng.uniform(U[0], U[-1])))
        w.append(W[st[s]])
    u += [U[0] - 0.8, U[0] - 0.3, 0.5 * (U[1] + U[2]), U[-1]]
    w += [W[0] - 0.6, W[-1] + 0.9, W[-1] + 2.0, W[0]]
    x = np.exp(np.array(u))
    q2 = np.exp(np.array(w))
    # the oracle takes logs of x and Q^2; use the same libm log here
    return x, q2, [math.log(v) for v in x], [math.log(v) for v in q2]


GRIDS = [lambda: two_members(tiny_single(), 5),
         lambda: two_members(tiny_two_sub(seed=17, dup_equal=False), 6)]


def kappa_vs_exact_weights(make, n=14, seed=21):
    """Largest relative gap between the oracle's kappa (matrix and pointwise
    forms, both members) and the sum built from the exact weights."""
    g = make()
    o = OracleGrid.from_synth(g)
    x, q2, us, ws = _points(g, o, n, seed)
    pids = np.concatenate([g.pids, [5]]).astype(np.int32)     # pid 5 is absent
    worst = 0.0
    for member in range(g.n_members):
        kap = o.kappa(pids, x, q2, member=member)
        pid_pw = g.pids[np.arange(x.size) % g.n_flav].astype(np.int32)
        kap_pw = o.kappa(pid_pw, x, q2, member=member, pointwise=True)
        for i in range(x.size):
            Wt = exact_weights(g, o, us[i], ws[i])
            for p, pid in enumerate(pids):
                col = list(g.pids).index(pid) if pid in g.pids else -1
                want = 0.0 if col < 0 else float(np.sum(np.abs(Wt * g.values[member, :, :, col])))
                worst = max(worst, abs(kap[i, p] - want) / max(want, 1e-300) if want else abs(kap[i, p]))
            col = list(g.pids).index(pid_pw[i])
            want = float(np.sum(np.abs(Wt * g.values[member, :, :, col])))
            worst = max(worst, abs(kap_pw[i] - want) / want)
    return worst


@pytest.mark.parametrize("make", GRIDS)
def test_kappa_is_the_sum_of_exact_weight_magnitudes(make):
    assert kappa_vs_exact_weights(make) < 1e-13


@pytest.mark.parametrize("make", GRIDS)
def test_kappa_at_knots_is_the_magnitude_of_the_value(make):
    g = make()
    o = OracleGrid.from_synth(g)
    st = _starts(g)
    upper_copy = set(st[1:-1])      # a threshold Q belongs to the upper subgrid
    for member in range(g.n_members):
        for r in range(g.n_rows):
            if r + 1 in upper_copy:
                continue
            x = g.x_knots.copy()
            q2 = np.full(x.size, g.q_knots[r] ** 2)
            kap = o.kappa(g.pids, x, q2, member=member)
            ref = o.xfxq2_batch(g.pids, x, q2, member=member)
            assert np.array_equal(kap, np.abs(ref))
            assert np.array_equal(kap, np.abs(g.values[member, r]))


def dgrid_absval_vs_exact(n=12, seed=23):
    """Largest gap of the |term| sums (and of the signed sums) of the grid
    gradient, pointwise and matrix forms, against the exact weights."""
    g = tiny_two_sub(seed=19, dup_equal=False)
    o = OracleGrid.from_synth(g)
    x, q2, us, ws = _points(g, o, n, seed)
    rng = np.random.default_rng(seed)
    gw = rng.standard_normal(x.size)
    pid = g.pids[rng.integers(0, g.n_flav, x.size)].astype(np.int32)
    gout = rng.standard_normal((x.size, g.n_flav))
    Wts = [exact_weights(g, o, us[i], ws[i]) for i in range(x.size)]
    want_pw = np.zeros(g.values.shape[1:])
    want_pw_s = np.zeros_like(want_pw)
    want_b = np.zeros_like(want_pw)
    want_b_s = np.zeros_like(want_pw)
    for i, Wt in enumerate(Wts):
        col = list(g.pids).index(pid[i])
        want_pw[:, :, col] += np.abs(gw[i] * Wt)
        want_pw_s[:, :, col] += gw[i] * Wt
        for c in range(g.n_flav):
            want_b[:, :, c] += np.abs(gout[i, c] * Wt)
            want_b_s[:, :, c] += gout[i, c] * Wt
    got = [o.dgrid_pw(pid, x, q2, gw, absval=True), o.dgrid_pw(pid, x, q2, gw),
           o.dgrid(g.pids, x, q2, gout, absval=True), o.dgrid(g.pids, x, q2, gout)]
    want = [want_pw, want_pw_s, want_b, want_b_s]
    scale = [np.max(want_pw), np.max(want_pw), np.max(want_b), np.max(want_b)]
    return max(float(np.max(np.abs(a - b))) / s for a, b, s in zip(got, want, scale))


def test_grid_gradient_term_magnitudes_from_exact_weights():
    assert dgrid_absval_vs_exact() < 1e-13


def lumi_absval_vs_exact(n=10, seed=29):
    """Largest gap of the luminosity gradient's |term| sums (and signed sums)
    against exact weights and exact partner values.  Pairing: b with -b, the
    gluon with itself; the term of side 0 is W(x1) f_{-b}(x2) / n, of side 1
    f_{-b}(x1) W(x2) / n."""
    g = tiny_two_sub(seed=37, dup_equal=False)        # pids -1, 0, 1
    o = OracleGrid.from_synth(g)
    rng = np.random.default_rng(seed)
    ln_tau = rng.uniform(-9.0, -0.5, n)
    y = (2.0 * rng.uniform(0.0, 1.0, n) - 1.0) * (-0.5 * ln_tau)
    ln_s = 5.0                                       # ln Q^2 from -4 to 4.5
    ev = synth.Events(ln_tau, y, np.zeros(n, np.uint8), np.zeros(n), np.zeros(n), ln_s)
    st = _starts(g)
    wsub = [o.W[st[s]:st[s + 1]] for s in range(len(g.n_q))]
    exact = [ExactGrid(o.U, wsub, [g.values[0, st[s]:st[s + 1], :, c] for s in range(len(g.n_q))])
             for c in range(g.n_flav)]
    anti = [list(g.pids).index(-p) for p in g.pids]
    want = np.zeros(g.values.shape[1:])
    want_s = np.zeros_like(want)
    for e in range(n):
        h = 0.5 * ln_tau[e]
        u = (h + y[e], h - y[e])
        w = ln_tau[e] + ln_s
        f = [[float(ex.eval(u[side], w)[0]) for ex in exact] for side in (0, 1)]
        for side in (0, 1):
            Wt = exact_weights(g, o, u[side], w)
            for b in range(g.n_flav):
                t = Wt * f[1 - side][anti[b]] / n
                want[:, :, b] += np.abs(t)
                want_s[:, :, b] += t
    got = o.lumi_dgrid(ev, absval=True)
    got_s = o.lumi_dgrid(ev)
    return max(float(np.max(np.abs(got - want))), float(np.max(np.abs(got_s - want_s)))) / float(np.max(want))


def test_luminosity_gradient_term_magnitudes_from_exact_weights():
    assert lumi_absval_vs_exact() < 1e-13


def alphas_kappa_vs_exact(n=40, seed=31):
    worst = 0.0
    for make in (tiny_single, lambda: tiny_two_sub(seed=41, dup_equal=False)):
        g = make()
        o = OracleGrid.from_synth(g)
        rng = np.random.default_rng(seed)
        q2 = np.exp(rng.uniform(o.W[0] - 2.0, o.W[-1] + 2.0, n))
        q2 = np.concatenate([q2, g.q_knots ** 2])
        kap = o.alphas_kappa(q2)
        for i, v in enumerate(q2):
            Wt = exact_alphas_weights(g, o, math.log(v))
            want = float(np.sum(np.abs(Wt * g.alphas)))
            worst = max(worst, abs(kap[i] - want) / want)
    return worst


def test_alphas_kappa_is_the_sum_of_exact_weight_magnitudes():
    assert alphas_kappa_vs_exact() < 1e-13


def test_alphas_kappa_at_knots_and_domain():
    g = synth.grid_nnpdf()
    o = OracleGrid.from_synth(g)
    st = _starts(g)
    rows = [r for r in range(g.n_rows) if r + 1 not in set(st[1:-1])]
    q2 = g.q_knots[rows] ** 2
    assert np.array_equal(o.alphas_kappa(q2), g.alphas[rows])
    assert np.array_equal(o.alphas_kappa(q2), o.alphas_batch(q2))
    bad = np.array([0.0, -1.0, np.inf, np.nan])
    assert np.all(np.isnan(o.alphas_kappa(bad)))


def test_alphas_kappa_is_close_to_alphas_on_smooth_data():
    """Inside the grid, on positive, slowly varying one-loop values, kappa
    is alpha_s times at most the sum of |weights|: 1 at knots, and at most
    1.25 for the interior Hermite weights with finite-difference slopes on
    uniform knots (-1/16, 9/16, 9/16, -1/16 at the middle of an interval);
    a kappa that counted terms twice or took them from other knots would be
    far outside [1, 1.3)."""
    g = synth.grid_nnpdf()
    o = OracleGrid.from_synth(g)
    _, _, q2 = synth.queries_nnpdf(20_000, seed=3)
    r = o.alphas_kappa(q2) / o.alphas_batch(q2)
    assert np.all(r >= 1.0) and np.all(r < 1.3)
    assert np.max(r) > 1.2              # the middle of an interval is reached
