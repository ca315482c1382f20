"""120 randomly shaped grids against the oracle: 2 to 30 x knots with random
spacing (the last one at x = 1 or below it), 1 to 4 Q subgrids of 2 to 9
knots each (duplicated threshold rows equal or not), 1 to 14 flavours with
random distinct pids (the gluon as 0 or 21), 1 to 3 members, every
interpolation kind with the linear, freeze and error options.  Checked per
grid: x*f for a pid list with an absent pid, the pointwise form, alpha_s, and
the adjoint (dL/dx, dL/dQ^2, dL/dgrid, also through the tape and the derivative
tape)."""
import math

import numpy as np
import pytest

from oracle.oracle import OracleGrid
from paper_2012_08221_gb300 import synth
from tests import parity
from tests.tinygrids import random_grid

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_GRIDS = 120


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _points(g, rng, n):
    U, W = np.log(g.x_knots), np.log(g.q_knots ** 2)
    x = np.exp(rng.uniform(U[0] - 2.0, 0.0, n))
    q2 = np.exp(rng.uniform(W[0] - 2.0, W[-1] + 2.0, n))
    k = min(n // 4, g.x_knots.size * 4)
    x[:k] = rng.choice(g.x_knots, k)           # exact knots and thresholds
    q2[:k] = rng.choice(g.q_knots, k) ** 2
    return x, q2


@pytest.mark.parametrize("seed", range(N_GRIDS))
def test_random_grid_against_the_oracle(seed):
    from paper_2012_08221_gb300 import build
    from paper_2012_08221_gb300.pdf import PDF
    build.build()
    g, rng = random_grid(7000 + seed)
    interp, extrap = seed % 3, (seed // 3) % 3
    pdf = PDF.from_grid(g, interp=interp, extrap=extrap)
    o = OracleGrid.from_synth(g, interp=interp, extrap=extrap)
    x, q2 = _points(g, rng, 4001)
    X, Q = cuda(x), cuda(q2)
    member = int(rng.integers(0, g.values.shape[0]))
    pids = np.append(rng.permutation(g.pids), 5 if 5 not in g.pids else 6 if 6 not in g.pids else 22)
    pids = pids.astype(np.int32)
    got = pdf.xfxQ2(pids, X, Q, member).cpu().numpy()
    parity.check(got, o.xfxq2_batch(pids, x, q2, member=member), o.kappa(pids, x, q2, member=member),
                 what=f"fuzz {seed} xfxQ2")
    pid = rng.choice(pids, x.size).astype(np.int32)
    got = pdf.xfxQ2_pw(cuda(pid), X, Q, member).cpu().numpy()
    parity.check(got, o.xfxq2_pw(pid, x, q2, member=member), o.kappa(pid, x, q2, member=member, pointwise=True),
                 what=f"fuzz {seed} pointwise")
    ra = o.alphas_batch(q2)
    parity.check(pdf.alphasQ2(Q).cpu().numpy(), ra, o.alphas_kappa(q2), what=f"fuzz {seed} alpha_s")
    # the adjoint, pointwise, from scratch, from the tape and from the tape
    # with the forward's patch derivatives
    w = rng.standard_normal(x.size)
    T = pdf.new_tape(x.size)
    D = pdf.new_dtape(x.size)
    pdf.xfxQ2_pw(cuda(pid), X, Q, member, tape=T, dtape=D)
    rdx, rdq = o.grad_pw(pid, x, q2, member=member)
    U, W = np.log(g.x_knots), np.log(g.q_knots ** 2)
    vmax = np.max(np.abs(g.values))
    scale = {"x": np.abs(w) * vmax * 8 / np.min(np.diff(U)),
             "q": np.abs(w) * vmax * 8 / np.min(np.diff(W)[np.diff(W) > 0])}
    ref = o.dgrid_pw(pid, x, q2, w)
    kg = o.dgrid_pw(pid, x, q2, w, absval=True)
    for tape, dtape in ((None, None), (T, None), (T, D)):
        gv = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
        gx, gq, _ = pdf.xfxQ2_backward(cuda(pid), X, Q, cuda(w), member=member, pointwise=True,
                                       grad_values=gv, tape=tape, dtape=dtape)
        for got, want, z, sc in ((gx, w * rdx, x, scale["x"]), (gq, w * rdq, q2, scale["q"])):
            got = got.cpu().numpy()
            assert np.array_equal(np.isnan(got), np.isnan(want)), seed
            m = ~np.isnan(want)
            assert np.all(np.abs(got[m] - want[m]) <= 1e-9 * (np.abs(want[m]) + sc[m] / z[m])), seed
        if extrap != 2:
            # floor: stencil weights that vanish exactly (at the last knot of
            # an axis the oracle divides, the kernels multiply by the
            # interval's reciprocal, t = 1 - 1 ulp) leave rounding-size
            # contributions, at most a few ulp of the point weights
            floor = 1e-14 * np.abs(w).sum()
            assert np.all(np.abs(gv.cpu().numpy() - ref) <= 1e-9 * np.maximum(np.abs(ref), kg) + floor), seed


@pytest.mark.parametrize("seed", range(0, N_GRIDS, 3))
def test_random_grid_luminosity_against_the_oracle(seed):
    """The fused luminosity and its grid gradient on the same random grids
    (linear and freeze options): per-event values and dL/dvalues against the
    oracle; a gluon listed as 21 still pairs with itself."""
    from paper_2012_08221_gb300 import build
    from paper_2012_08221_gb300.lumi import DeviceEvents, luminosity, luminosity_backward
    from paper_2012_08221_gb300.pdf import PDF
    build.build()
    g, rng = random_grid(7000 + seed)
    interp, extrap = seed % 3, (seed // 3) % 2
    pdf = PDF.from_grid(g, interp=interp, extrap=extrap)
    o = OracleGrid.from_synth(g, interp=interp, extrap=extrap)
    ev = synth.events_lhc(3001, seed=8000 + seed)
    dev = DeviceEvents.from_host(ev)
    member = int(rng.integers(0, g.values.shape[0]))
    L, lum, _ = luminosity(pdf, dev, member=member)
    Lr, lumr, _ = o.lumi(ev, member=member)
    scale = g.pids.size * np.max(np.abs(g.values)) ** 2
    assert np.all(np.abs(lum.cpu().numpy() - lumr) <= 1e-11 * (np.abs(lumr) + scale)), seed
    gv = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
    luminosity_backward(pdf, dev, 1.0, gv, member=member)
    ref = o.lumi_dgrid(ev, member=member)
    kap = o.lumi_dgrid(ev, member=member, absval=True)
    assert np.all(np.abs(gv.cpu().numpy() - ref) <= 1e-9 * np.maximum(np.abs(ref), kap) + 1e-300), seed


@pytest.mark.parametrize("batch_seed", range(4))
def test_random_grids_in_one_batched_launch(batch_seed):
    """Requests over several random grids (and options) in one persistent
    launch, with and without the shared-memory staging of the knot tables:
    every request equals its standalone call bit for bit."""
    from paper_2012_08221_gb300 import build
    from paper_2012_08221_gb300.batch import Batch
    from paper_2012_08221_gb300.pdf import PDF
    build.build()
    rng = np.random.default_rng(9000 + batch_seed)
    grids = [random_grid(7100 + 10 * batch_seed + k)[0] for k in range(4)]
    pdfs = [PDF.from_grid(g, interp=k % 3, extrap=(k + batch_seed) % 3) for k, g in enumerate(grids)]
    reqs = []
    for r in range(40):
        k = int(rng.integers(0, len(grids)))
        g = grids[k]
        n = int(rng.integers(0, 5000))
        x, q2 = _points(g, rng, max(n, 1))
        pids = rng.choice(np.append(g.pids, 7), size=int(rng.integers(1, 4))).astype(np.int32)
        out = torch.empty((n, pids.size), dtype=torch.float64, device="cuda")
        reqs.append((pdfs[k], int(rng.integers(0, g.values.shape[0])), pids, cuda(x[:n]), cuda(q2[:n]), out))
    for tune in (False, True):
        for r in reqs:
            r[5].fill_(-7.0)
        Batch(reqs, autotune=tune).run()
        torch.cuda.synchronize()
        for pdf, member, pids, X, Q, out in reqs:
            ref = pdf.xfxQ2(pids, X, Q, member)
            assert torch.equal(torch.nan_to_num(out, nan=3.0), torch.nan_to_num(ref, nan=3.0)), (batch_seed, tune)


@pytest.mark.parametrize("seed", range(8))
def test_random_vegas_maps_against_the_oracle(seed):
    """The general VEGAS map and accumulation for random dimensions (1 to
    16), bin counts (2 to 1024) and uneven edges, with uniforms that include
    0 and values next to 1: bins bit for bit, points and Jacobians to
    rounding, sums to 1e-12 of their scale."""
    from paper_2012_08221_gb300 import build
    from paper_2012_08221_gb300.vegas import Vegas
    from oracle.oracle import vegas_accumulate, vegas_map
    build.build()
    rng = np.random.default_rng(9500 + seed)
    dim, n_bins = int(rng.integers(1, 17)), int(rng.choice([2, 3, 7, 50, 128, 1024]))
    widths = np.exp(rng.uniform(-2.0, 2.0, (dim, n_bins)))
    edges = np.concatenate([np.zeros((dim, 1)), np.cumsum(widths, 1) / widths.sum(1, keepdims=True)], 1)
    edges[:, -1] = 1.0
    v = rng.uniform(0, 1, (20_011, dim))
    v[:3] = np.array([0.0, np.nextafter(1.0, 0.0), 0.5])[:, None]
    vg = Vegas(dim, n_bins=n_bins)
    vg.edges = edges
    r, jac, bins = vg.map(cuda(v))
    rr, rj, rb = vegas_map(edges, v)
    assert np.array_equal(bins.cpu().numpy(), rb), seed
    assert np.allclose(r.cpu().numpy(), rr, rtol=0, atol=1e-15), seed
    assert np.allclose(jac.cpu().numpy(), rj, rtol=1e-13, atol=0), seed
    w = rng.standard_normal(v.shape[0]) * np.exp(rng.uniform(-3, 3, v.shape[0]))
    got = vg.accumulate(cuda(w), cuda(rb))
    ref = vegas_accumulate(n_bins, w, rb)
    scale = np.concatenate([[np.abs(w).sum()], ref[1:]])
    assert np.all(np.abs(got - ref) <= 1e-12 * scale + 1e-300), seed


def _edge_positions(knots_log, z):
    t = np.zeros_like(z)
    lo, hi = z < knots_log[0], z > knots_log[-1]
    t[lo] = (z[lo] - knots_log[0]) / (knots_log[1] - knots_log[0])
    t[hi] = (z[hi] - knots_log[-2]) / (knots_log[-1] - knots_log[-2])
    return t


@pytest.mark.parametrize("seed", range(0, N_GRIDS, 2))
def test_random_grid_power_law_continuation(seed):
    """The power-law continuation on the random grids (whose values change
    sign, so both the power law and its linear fallback occur): x*f and
    alpha_s against the oracle with the same option; inside the grid bit for
    bit the linear option's values.  Outside, the power law raises the edge
    values' rounding to the power |t| (up to 30 intervals out here, with edge
    values down to the 1e-3 threshold and results up to 1e19), so the check
    there is 1e-9 relative to the value or to kappa times the distance
    (1 + |t_x|)(1 + |t_Q|): a wrong branch, knot or exponent is off by far
    more."""
    from paper_2012_08221_gb300 import build
    from paper_2012_08221_gb300.pdf import PDF
    build.build()
    g, rng = random_grid(7000 + seed)
    interp = seed % 3
    pc = PDF.from_grid(g, interp=interp, extrap="continuation")
    pl = PDF.from_grid(g, interp=interp, extrap="linear")
    oc = OracleGrid.from_synth(g, interp=interp, extrap=3)
    ol = OracleGrid.from_synth(g, interp=interp, extrap=0)
    x, q2 = _points(g, rng, 4001)
    X, Q = cuda(x), cuda(q2)
    got = pc.xfxQ2(g.pids, X, Q).cpu().numpy()
    lin = pl.xfxQ2(g.pids, X, Q).cpu().numpy()
    tu = _edge_positions(np.log(g.x_knots), np.log(x))
    tw = _edge_positions(np.log(g.q_knots ** 2), np.log(q2))
    inside = (tu == 0) & (tw == 0)
    assert np.array_equal(got[inside], lin[inside]), seed
    grow = ((1 + np.abs(tu)) * (1 + np.abs(tw)))[:, None]
    ref = oc.xfxq2_batch(g.pids, x, q2)
    kap = ol.kappa(g.pids, x, q2)
    parity.check(got[inside], ref[inside], kap[inside], what=f"fuzz {seed} continuation inside")
    out = ~inside
    err = np.abs(got[out] - ref[out])
    assert np.all(err <= 1e-9 * (np.abs(ref[out]) + kap[out] * grow[out])), (seed, float(np.max(err)))
    ra = oc.alphas_batch(q2)
    parity.check(pc.alphasQ2(Q).cpu().numpy(), ra, ol.alphas_kappa(q2) * (1 + np.abs(tw)),
                 what=f"fuzz {seed} alpha_s")
