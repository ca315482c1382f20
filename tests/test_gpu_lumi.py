"""GPU fused luminosity workload: per-event luminosity, alpha_s and
L = (1/n) sum lum against the oracle (including the injected low tail that
exercises the extrapolation), and the grid gradient of L."""
import math

import numpy as np
import pytest

from oracle.oracle import OracleGrid
from paper_2012_08221_gb300 import synth
from tests import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.fixture(scope="module")
def lhc():
    from paper_2012_08221_gb300 import build
    from paper_2012_08221_gb300.pdf import PDF
    build.build()
    g = synth.grid_nnpdf(seeds=(1005, 1006, 1007))   # three replicas, member 0 used
    return g, PDF.from_grid(g), OracleGrid.from_synth(g)


def _event_logs(ev, n):
    h = 0.5 * ev.ln_tau[:n]
    u1 = h + ev.y[:n]
    u2 = h - ev.y[:n]
    w = ev.ln_tau[:n] + ev.ln_s
    f = ev.flags[:n]
    w = np.where(f & 1, ev.ln_mu2[:n], w)
    u1 = np.where(f & 2, ev.ln_x1[:n], u1)
    return u1, u2, w


def _lum_kappa(g, o, ev, n, member=0):
    """Term scale of lum: sum_a kappa(x1)_a |f(x2)_-a| + |f(x1)_a| kappa(x2)_-a."""
    u1, u2, w = _event_logs(ev, n)
    x1, x2, q2 = np.exp(u1), np.exp(u2), np.exp(w)
    k1 = o.kappa(g.pids, x1, q2, member=member)
    k2 = o.kappa(g.pids, x2, q2, member=member)
    f1 = np.abs(o.xfxq2_batch(g.pids, x1, q2, member=member))
    f2 = np.abs(o.xfxq2_batch(g.pids, x2, q2, member=member))
    anti = np.array([list(g.pids).index(-p) for p in g.pids])
    return np.sum(k1 * f2[:, anti] + f1 * k2[:, anti] + k1 * k2[:, anti], axis=1)


def _as_kappa(o, ev, n):
    """Term scale of alpha_s at each event's scale (kappa of alpha_s at
    Q^2 = e^w; one rounding of the exponential moves only the scale)."""
    return o.alphas_kappa(np.exp(_event_logs(ev, n)[2]))


def test_luminosity_parity(lhc):
    from paper_2012_08221_gb300.lumi import DeviceEvents, luminosity
    g, pdf, o = lhc
    n = 30_011
    ev = synth.events_lhc(n, seed=91)
    dev = DeviceEvents.from_host(ev)
    L, lum, a_s = luminosity(pdf, dev)
    Lr, lumr, asr = o.lumi(ev)
    kap = _lum_kappa(g, o, ev, n)
    parity.check(lum.cpu().numpy(), lumr, kap, what="lum")
    parity.check(a_s.cpu().numpy(), asr, _as_kappa(o, ev, n), what="lumi alpha_s")
    assert abs(L.item() - Lr) <= 1e-12 * kap.sum() / n
    assert np.sum(ev.flags != 0) > 0.03 * n          # the tail is there


def test_luminosity_tail_only(lhc):
    from paper_2012_08221_gb300.lumi import DeviceEvents, luminosity
    g, pdf, o = lhc
    ev = synth.events_lhc(4000, seed=92, tail=1.0)   # every event in the low tail
    L, lum, a_s = luminosity(pdf, DeviceEvents.from_host(ev))
    Lr, lumr, asr = o.lumi(ev)
    parity.check(lum.cpu().numpy(), lumr, _lum_kappa(g, o, ev, 4000), what="tail lum")
    parity.check(a_s.cpu().numpy(), asr, _as_kappa(o, ev, 4000), what="tail alpha_s")


def test_luminosity_gradient_against_oracle(lhc):
    from paper_2012_08221_gb300.lumi import DeviceEvents, luminosity_backward
    g, pdf, o = lhc
    ev = synth.events_lhc(3001, seed=93)
    gv = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
    luminosity_backward(pdf, DeviceEvents.from_host(ev), 1.0, gv)
    ref = o.lumi_dgrid(ev)
    got = gv.cpu().numpy()
    tol = 1e-9 * np.maximum(np.abs(ref), o.lumi_dgrid(ev, absval=True)) + 1e-300
    assert np.all(np.abs(got - ref) <= tol), float(np.max(np.abs(got - ref) / tol))


def test_luminosity_gradient_near_the_knots(lhc):
    """Partons a little inside a cell next to a knot (t = 1e-3 ... 1e-4 above
    one, t = 1 - 1e-3 ... 1 - 1e-4 below the next) on both axes, each event
    in cells of its own (x1 and Q^2 set through the event overrides, x2 by
    the rapidity): the luminosity adjoint accumulates them in the patch's
    monomial basis in the near-knot coordinate of their half of the cell,
    so the stencil weights that vanish like t^2 or (1 - t)^2 at the near
    knot keep their relative accuracy.  The grid gradient matches the
    oracle's within 1e-9 of each value's own term scale, with no absolute
    floor."""
    from paper_2012_08221_gb300.lumi import DeviceEvents, luminosity_backward
    g, pdf, o = lhc
    U = np.log(g.x_knots)
    W = np.log(np.asarray(g.q_knots, dtype=np.float64) ** 2)
    r_sub = int(np.sum(g.n_q[:2]))                # first row of the third Q subgrid
    rows = []
    for k, d in enumerate([1e-3, 5e-4, 2e-4, 1e-4]):
        for lo in (False, True):
            kx1 = 20 + 17 * k + (0 if lo else 8)
            kx2 = kx1 + 40
            r = r_sub + 2 + 2 * k + (1 if lo else 0)
            t1, t2, tq = (d, 1.0 - d, 1.0 - d) if lo else (1.0 - d, d, d)
            rows.append((U[kx1] + t1 * (U[kx1 + 1] - U[kx1]), U[kx2] + t2 * (U[kx2 + 1] - U[kx2]),
                         W[r] + tq * (W[r + 1] - W[r])))
    u1, u2, w = (np.array(c) for c in zip(*rows))
    n = u1.size
    ln_tau = np.full(n, -1.0)
    ev = synth.Events(ln_tau, 0.5 * ln_tau - u2, np.full(n, 3, dtype=np.uint8), w, u1, 2.0 * math.log(13000.0))
    gv = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
    luminosity_backward(pdf, DeviceEvents.from_host(ev), 1.0, gv)
    ref = o.lumi_dgrid(ev)
    got = gv.cpu().numpy()
    tol = 1e-9 * np.maximum(np.abs(ref), o.lumi_dgrid(ev, absval=True))
    assert np.all(np.abs(got - ref) <= tol), float(np.max(np.abs(got - ref) / np.maximum(tol, 1e-300)))
    assert np.count_nonzero(ref) > 0


def test_luminosity_gradient_on_a_grid_with_more_bins_than_shared_memory():
    """A grid of 400 x knots and the NNPDF Q subgrids: 399 x 46 cells x 5
    bin kinds are more than the shared-memory counters of the histogram and
    the scatter hold, so both take their global-memory paths; the gradient
    against the oracle (events with the low tail)."""
    from paper_2012_08221_gb300.lumi import DeviceEvents, luminosity_backward
    from paper_2012_08221_gb300.pdf import PDF
    xk = synth.log_knots(1e-9, 1.0, 400)
    qk, nq = synth.subgrid_knots([1.0, 1.51, 4.92, 172.5, 1e5], [8, 12, 20, 10])
    g = synth._grid("lumi-400x50", xk, qk, nq, synth.PIDS_13, [1009])
    pdf, o = PDF.from_grid(g), OracleGrid.from_synth(g)
    ev = synth.events_lhc(20_001, seed=95)
    gv = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
    luminosity_backward(pdf, DeviceEvents.from_host(ev), 1.0, gv)
    ref = o.lumi_dgrid(ev)
    got = gv.cpu().numpy()
    tol = 1e-9 * np.maximum(np.abs(ref), o.lumi_dgrid(ev, absval=True)) + 1e-300
    assert np.all(np.abs(got - ref) <= tol), float(np.max(np.abs(got - ref) / tol))
    assert pdf.status() & 4 == 0


def test_saved_partner_factors_give_the_same_gradient(lhc):
    """The backward pass from the forward's saved partner factors equals the
    one that recomputes them (up to the summation order of the atomics)."""
    from paper_2012_08221_gb300.lumi import DeviceEvents, luminosity, luminosity_backward
    g, pdf, o = lhc
    evh = synth.events_lhc(50_003, seed=95)
    ev = DeviceEvents.from_host(evh)
    P = torch.empty((ev.n, 2, g.n_flav), dtype=torch.float64, device="cuda")
    L1, lum1, _ = luminosity(pdf, ev, save_p=P)
    L0, lum0, _ = luminosity(pdf, ev)
    assert torch.equal(lum0, lum1) and torch.equal(L0, L1)
    ga = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
    gb = torch.zeros_like(ga)
    luminosity_backward(pdf, ev, 2.0, ga)
    luminosity_backward(pdf, ev, 2.0, gb, saved_p=P)
    assert torch.allclose(ga, gb, rtol=1e-12, atol=1e-15 * float(ga.abs().max()))
    ref = 2.0 * o.lumi_dgrid(evh)
    kap = 2.0 * o.lumi_dgrid(evh, absval=True)
    assert np.all(np.abs(gb.cpu().numpy() - ref) <= 1e-9 * np.maximum(np.abs(ref), kap) + 1e-300)


def test_sixteen_flavours_with_an_unpaired_one(lhc):
    """The widest luminosity grid (16 flavours: -7..7 and a photon, 22, with
    no partner): forward and adjoint against the oracle."""
    from paper_2012_08221_gb300.lumi import DeviceEvents, luminosity, luminosity_backward
    from paper_2012_08221_gb300.pdf import PDF
    pids = np.concatenate([np.arange(-7, 8), [22]]).astype(np.int32)
    g = synth.grid_small(seed=1008, pids=pids)
    pdf, o = PDF.from_grid(g), OracleGrid.from_synth(g)
    ev = synth.events_lhc(3000, seed=96)
    dev = DeviceEvents.from_host(ev)
    L, lum, _ = luminosity(pdf, dev)
    Lr, lumr, _ = o.lumi(ev)
    assert np.allclose(lum.cpu().numpy(), lumr, rtol=1e-11, atol=1e-13 * np.max(np.abs(lumr)))
    gv = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
    luminosity_backward(pdf, dev, 1.0, gv)
    ref = o.lumi_dgrid(ev)
    kap = o.lumi_dgrid(ev, absval=True)
    assert np.all(np.abs(gv.cpu().numpy() - ref) <= 1e-9 * np.maximum(np.abs(ref), kap) + 1e-300)
    assert np.all(gv.cpu().numpy()[:, :, 15] == 0.0)        # the photon has no partner


def test_luminosity_autograd(lhc):
    from paper_2012_08221_gb300.autograd import lumi
    from paper_2012_08221_gb300.lumi import DeviceEvents
    g, pdf, o = lhc
    ev = synth.events_lhc(2000, seed=94)
    vals = torch.tensor(g.values, device="cuda", requires_grad=True)
    L = lumi(pdf, vals, DeviceEvents.from_host(ev))
    (3.0 * L).backward()
    ref = 3.0 * o.lumi_dgrid(ev)
    got = vals.grad[0].cpu().numpy()
    kap = 3.0 * o.lumi_dgrid(ev, absval=True)
    assert np.all(np.abs(got - ref) <= 1e-9 * np.maximum(np.abs(ref), kap) + 1e-300)
    assert torch.count_nonzero(vals.grad[1:]) == 0
    assert abs(L.item() - o.lumi(ev)[0]) <= 1e-12 * abs(L.item()) + 1e-15


def test_full_size_luminosity_sampled(lhc):
    """1e8 events in one launch: L equals the mean of the per-event values,
    2e5 sampled events match the oracle, and the grid gradient (12 chunks of
    events) obeys the exact flavour sum rule sum_cells dL/dv[.][b] =
    mean_e(f_-b(x2) + f_-b(x1)) with the right-hand side from the oracle (the
    interpolation's weights sum to 1), for the gluon and the u quark."""
    from paper_2012_08221_gb300.lumi import DeviceEvents, luminosity, luminosity_backward
    g, pdf, o = lhc
    n = 100_000_000
    ev = synth.events_lhc(n)
    dev = DeviceEvents.from_host(ev)
    L, lum, a_s = luminosity(pdf, dev)
    lum_h = lum.cpu().numpy()
    assert abs(L.item() - lum_h.sum() / n) <= 1e-12 * np.abs(lum_h).sum() / n
    idx = np.random.default_rng(5).choice(n, 200_000, replace=False)
    sub = synth.Events(ev.ln_tau[idx], ev.y[idx], ev.flags[idx], ev.ln_mu2[idx], ev.ln_x1[idx], ev.ln_s)
    Lr, lumr, asr = o.lumi(sub)
    parity.check(lum_h[idx], lumr, _lum_kappa(g, o, sub, idx.size), what="full lum")
    parity.check(a_s[cuda(idx)].cpu().numpy(), asr, _as_kappa(o, sub, idx.size), what="full alpha_s")
    del lum, a_s
    gv = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
    luminosity_backward(pdf, dev, 1.0, gv)
    G = gv.cpu().numpy()
    # sum rule, right-hand side from the oracle on the same partons, for the
    # gluon (its own partner) and the u quark (partner u-bar)
    u1, u2, w = _event_logs(ev, n)
    pids = list(g.pids)
    cols = [pids.index(0), pids.index(2)]
    partners = np.array([0, -2], dtype=np.int32)
    acc = np.zeros(2)
    acc_abs = np.zeros(2)
    step = 10_000_000
    for s in range(0, n, step):
        q2 = np.exp(w[s:s + step])
        f1 = o.xfxq2_batch(partners, np.exp(u1[s:s + step]), q2)
        f2 = o.xfxq2_batch(partners, np.exp(u2[s:s + step]), q2)
        acc += f1.sum(0) + f2.sum(0)
        acc_abs += np.abs(f1).sum(0) + np.abs(f2).sum(0)
    for k, b in enumerate(cols):
        want = acc[k] / n
        assert abs(G[:, :, b].sum() - want) <= 1e-9 * (abs(want) + acc_abs[k] / n)


def test_other_members_forward_and_gradient(lhc):
    """Replicas 1 and 2 of the three-member grid: luminosity and its grid
    gradient (into that member's slice) against the oracle for the same
    member; replica 2 differs from replica 0."""
    from paper_2012_08221_gb300.lumi import DeviceEvents, luminosity, luminosity_backward
    g, pdf, o = lhc
    ev = synth.events_lhc(3001, seed=94)
    dev = DeviceEvents.from_host(ev)
    for m in (1, 2):
        L, lum, a_s = luminosity(pdf, dev, member=m)
        Lr, lumr, asr = o.lumi(ev, member=m)
        parity.check(lum.cpu().numpy(), lumr, _lum_kappa(g, o, ev, 3001, member=m), what=f"lum member {m}")
        gv = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
        luminosity_backward(pdf, dev, 1.0, gv, member=m)
        ref = o.lumi_dgrid(ev, member=m)
        tol = 1e-9 * np.maximum(np.abs(ref), o.lumi_dgrid(ev, member=m, absval=True)) + 1e-300
        assert np.all(np.abs(gv.cpu().numpy() - ref) <= tol)
    assert not np.allclose(o.lumi(ev, member=2)[1], o.lumi(ev, member=0)[1])
