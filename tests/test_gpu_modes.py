"""GPU parity of the interpolation kinds and extrapolation modes against the
oracle with the same options: x*f, alpha_s, the adjoint, the batched launch
and the luminosity."""
import math

import numpy as np
import pytest

from oracle.oracle import OracleGrid
from paper_2012_08221_gb300 import synth
from tests import parity
from tests.tinygrids import tiny_two_sub

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MODES = [(i, e) for i in (0, 1, 2) for e in (0, 1, 2)]


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.fixture(scope="module")
def built():
    from paper_2012_08221_gb300 import build
    build.build()


def _points(g, n, seed):
    rng = np.random.default_rng(seed)
    x = np.exp(rng.uniform(math.log(g.x_knots[0]) - 3, 0.0, n))
    lq = np.log(g.q_knots ** 2)
    q2 = np.exp(rng.uniform(lq[0] - 2, lq[-1] + 2, n))
    return x, q2


@pytest.mark.parametrize("interp,extrap", MODES)
def test_forward_and_alphas(built, interp, extrap):
    from paper_2012_08221_gb300.pdf import PDF
    for g in (tiny_two_sub(seed=31, dup_equal=False), synth.grid_nnpdf()):
        pdf = PDF.from_grid(g, interp=interp, extrap=extrap)
        o = OracleGrid.from_synth(g, interp=interp, extrap=extrap)
        x, q2 = _points(g, 20_011, 32)
        pdf.status()
        got = pdf.xfxQ2(g.pids, cuda(x), cuda(q2)).cpu().numpy()
        st = pdf.status()
        assert bool(st & 2) == (extrap == 2)
        ref = o.xfxq2_batch(g.pids, x, q2)
        kap = o.kappa(g.pids, x, q2)
        parity.check(got, ref, kap, what=f"modes {interp},{extrap} {g.name}")
        ga = pdf.alphasQ2(cuda(q2)).cpu().numpy()
        ra = o.alphas_batch(q2)
        parity.check(ga, ra, o.alphas_kappa(q2), what="alphas")


@pytest.mark.parametrize("interp,extrap", MODES)
def test_adjoint(built, interp, extrap):
    from paper_2012_08221_gb300.pdf import PDF
    g = tiny_two_sub(seed=33)
    pdf = PDF.from_grid(g, interp=interp, extrap=extrap)
    o = OracleGrid.from_synth(g, interp=interp, extrap=extrap)
    x, q2 = _points(g, 3001, 34)
    pid = np.random.default_rng(35).choice(g.pids, x.size).astype(np.int32)
    w = np.random.default_rng(36).standard_normal(x.size)
    gv = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
    gx, gq, _ = pdf.xfxQ2_backward(cuda(pid), cuda(x), cuda(q2), cuda(w), pointwise=True, grad_values=gv)
    rdx, rdq = o.grad_pw(pid, x, q2)
    scale = np.abs(w) * (np.max(np.abs(g.values)) * 50)
    for got, ref, z in ((gx, w * rdx, x), (gq, w * rdq, q2)):
        got = got.cpu().numpy()
        assert np.array_equal(np.isnan(got), np.isnan(ref))
        m = ~np.isnan(ref)
        assert np.all(np.abs(got[m] - ref[m]) <= 1e-9 * (np.abs(ref[m]) + scale[m] / z[m]))
    if extrap != 2:
        ref = o.dgrid_pw(pid, x, q2, w)
        kg = o.dgrid_pw(pid, x, q2, w, absval=True)
        assert np.all(np.abs(gv.cpu().numpy() - ref) <= 1e-9 * np.maximum(np.abs(ref), kg) + 1e-300)


def test_batched_and_luminosity_follow_the_grid_modes(built):
    from paper_2012_08221_gb300.batch import Batch
    from paper_2012_08221_gb300.lumi import DeviceEvents, luminosity
    from paper_2012_08221_gb300.pdf import PDF
    g = synth.grid_nnpdf(seeds=(1005,))
    for interp, extrap in ((1, 1), (2, 0), (0, 2)):
        pdf = PDF.from_grid(g, interp=interp, extrap=extrap)
        o = OracleGrid.from_synth(g, interp=interp, extrap=extrap)
        x, q2 = _points(g, 5003, 37)
        out = torch.empty((x.size, 3), dtype=torch.float64, device="cuda")
        pids = np.array([-2, 0, 4], dtype=np.int32)
        Batch([(pdf, 0, pids, cuda(x), cuda(q2), out)], autotune=False).run()
        torch.cuda.synchronize()
        assert torch.equal(torch.nan_to_num(out, nan=7.0),
                           torch.nan_to_num(pdf.xfxQ2(pids, cuda(x), cuda(q2)), nan=7.0))
        ev = synth.events_lhc(4000, seed=38)
        L, lum, a_s = luminosity(pdf, DeviceEvents.from_host(ev))
        Lr, lumr, asr = o.lumi(ev)
        scale = np.abs(np.nan_to_num(lumr)) + 1e3
        got = lum.cpu().numpy()
        assert np.array_equal(np.isnan(got), np.isnan(lumr))
        m = ~np.isnan(lumr)
        assert np.all(np.abs(got[m] - lumr[m]) <= 1e-12 * scale[m])


# ------------------------------------------------ power-law continuation (3)

def _edge_positions(knots_log, z):
    """Position t of z in the edge interval of the knots when z is outside
    (t < 0 below, t > 1 above), 0 inside."""
    t = np.zeros_like(z)
    lo, hi = z < knots_log[0], z > knots_log[-1]
    t[lo] = (z[lo] - knots_log[0]) / (knots_log[1] - knots_log[0])
    t[hi] = (z[hi] - knots_log[-2]) / (knots_log[-1] - knots_log[-2])
    return t


@pytest.mark.parametrize("interp", [0, 1, 2])
def test_continuation_forward_and_alphas(built, interp):
    """x*f and alpha_s under the power-law continuation against the oracle
    with the same option.  The oracle's kappa is a linear-interpolation
    scale, so outside the grid it is widened by the continuation's growth
    (1 + |t_x|)(1 + |t_Q|) (rounding of the edge values carries through the
    power law with those weights); inside, the results equal the linear
    option's bit for bit."""
    from paper_2012_08221_gb300.pdf import PDF
    for g in (tiny_two_sub(seed=31, dup_equal=False), synth.grid_nnpdf()):
        pc = PDF.from_grid(g, interp=interp, extrap="continuation")
        pl = PDF.from_grid(g, interp=interp, extrap="linear")
        oc = OracleGrid.from_synth(g, interp=interp, extrap=3)
        ol = OracleGrid.from_synth(g, interp=interp, extrap=0)
        x, q2 = _points(g, 20_011, 41)
        X, Q = cuda(x), cuda(q2)
        got = pc.xfxQ2(g.pids, X, Q).cpu().numpy()
        lin = pl.xfxQ2(g.pids, X, Q).cpu().numpy()
        assert pc.status() == 0
        U, W = np.log(g.x_knots), np.log(g.q_knots ** 2)
        tu, tw = _edge_positions(U, np.log(x)), _edge_positions(W, np.log(q2))
        inside = (tu == 0) & (tw == 0)
        assert np.array_equal(got[inside], lin[inside])
        grow = ((1 + np.abs(tu)) * (1 + np.abs(tw)))[:, None]
        ref = oc.xfxq2_batch(g.pids, x, q2)
        kap = ol.kappa(g.pids, x, q2)
        parity.check(got, ref, kap * np.where(inside[:, None], 1.0, 10 * grow),
                     what=f"continuation interp {interp} {g.name}")
        ga = pc.alphasQ2(Q).cpu().numpy()
        ra = oc.alphas_batch(q2)
        # the power law carries the edge values' rounding with the linear
        # weights (1 - t, t), which kappa of the linear option already
        # holds, and adds |t| |ln(y1/y0)| ulps from the logarithm: (1 + |t|)
        parity.check(ga, ra, ol.alphas_kappa(q2) * (1 + np.abs(tw)), what="alphas continuation")
        v, d = pc.alphasQ2_grad(Q)
        rd = np.array([oc.alphas_grad(q)[1] for q in q2[:3000]])
        assert np.allclose(d.cpu().numpy()[:3000], rd, rtol=1e-9, atol=1e-12 * np.max(np.abs(rd)))


def test_continuation_refuses_the_adjoint_and_follows_into_batches_and_luminosity(built):
    from paper_2012_08221_gb300._lib import PdfError
    from paper_2012_08221_gb300.batch import Batch
    from paper_2012_08221_gb300.lumi import DeviceEvents, luminosity, luminosity_backward
    from paper_2012_08221_gb300.pdf import PDF
    g = synth.grid_nnpdf(seeds=(1005,))
    pdf = PDF.from_grid(g, extrap="continuation")
    o = OracleGrid.from_synth(g, extrap=3)
    x, q2 = _points(g, 5003, 42)
    pid = np.full(x.size, 2, np.int32)
    with pytest.raises(PdfError):
        pdf.xfxQ2_backward(cuda(pid), cuda(x), cuda(q2), cuda(np.ones(x.size)), pointwise=True)
    out = torch.empty((x.size, 3), dtype=torch.float64, device="cuda")
    pids = np.array([-2, 0, 4], dtype=np.int32)
    Batch([(pdf, 0, pids, cuda(x), cuda(q2), out)], autotune=False).run()
    torch.cuda.synchronize()
    assert torch.equal(out, pdf.xfxQ2(pids, cuda(x), cuda(q2)))
    ev = synth.events_lhc(4000, seed=43)
    dev = DeviceEvents.from_host(ev)
    L, lum, a_s = luminosity(pdf, dev)
    Lr, lumr, asr = o.lumi(ev)
    got = lum.cpu().numpy()
    # the injected tail sits up to ~40 x-intervals and ~30 Q-intervals below
    # the grid, where the power law multiplies the edge values' rounding
    assert np.all(np.abs(got - lumr) <= 1e-9 * (np.abs(lumr) + 1e3))
    assert np.allclose(a_s.cpu().numpy(), asr, rtol=1e-12, atol=0)
    gv = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
    with pytest.raises(PdfError):
        luminosity_backward(pdf, dev, 1.0, gv)
