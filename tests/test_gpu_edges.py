"""Empty and one-point inputs through every entry point: n = 0 is a no-op
that leaves accumulated outputs untouched (and gives L = 0 and zero VEGAS
sums), a single point matches the oracle."""
import math

import numpy as np
import pytest

from oracle.oracle import OracleGrid
from paper_2012_08221_gb300 import synth
from tests import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nn():
    from paper_2012_08221_gb300 import build
    from paper_2012_08221_gb300.pdf import PDF
    build.build()
    g = synth.grid_nnpdf(seeds=(1005,))
    return g, PDF.from_grid(g), OracleGrid.from_synth(g)


def _e(dtype=torch.float64):
    return torch.empty(0, dtype=dtype, device="cuda")


def test_empty_inputs_everywhere(nn):
    from paper_2012_08221_gb300.batch import Batch
    from paper_2012_08221_gb300.lumi import DeviceEvents, luminosity, luminosity_backward
    from paper_2012_08221_gb300.vegas import Vegas
    g, pdf, o = nn
    e, ei = _e(), _e(torch.int32)
    gv = torch.full(g.values.shape[1:], 3.0, dtype=torch.float64, device="cuda")
    T = pdf.new_tape(0)
    assert pdf.xfxQ2(g.pids, e, e, tape=T).shape == (0, g.n_flav)
    assert pdf.xfxQ2_pw(ei, e, e, tape=T).shape == (0,)
    v, d = pdf.alphasQ2_grad(e)
    assert d.shape == (0,)
    for tape in (None, T):
        gx, gq, _ = pdf.xfxQ2_backward(ei, e, e, e, pointwise=True, grad_values=gv, tape=tape)
        assert gx.shape == (0,) and gq.shape == (0,)
        pdf.xfxQ2_backward(g.pids, e, e, torch.empty((0, g.n_flav), dtype=torch.float64, device="cuda"),
                           grad_values=gv, tape=tape)
    h = torch.empty(0, dtype=torch.float64)
    assert pdf.xfxQ2_host(g.pids, h, h).shape == (0, g.n_flav)
    ev = DeviceEvents(e, e, _e(torch.uint8), e, e, 2 * math.log(13000.0))
    L, lum, a_s = luminosity(pdf, ev)
    assert L.item() == 0.0 and lum.shape == (0,)
    luminosity_backward(pdf, ev, 1.0, gv)
    torch.cuda.synchronize()
    assert bool((gv == 3.0).all())                   # nothing accumulated
    vg = Vegas(2, n_bins=8)
    r, jac, bins = vg.map(torch.empty((0, 2), dtype=torch.float64, device="cuda"))
    assert r.shape == (0, 2) and jac.shape == (0,)
    assert np.all(vg.accumulate(jac, bins) == 0.0)
    # a batch with an empty request among others
    x, q2, _ = synth.queries_nnpdf(1003, seed=71)
    X, Q = torch.as_tensor(x, device="cuda"), torch.as_tensor(q2, device="cuda")
    out = torch.empty((x.size, 2), dtype=torch.float64, device="cuda")
    Batch([(pdf, 0, np.array([1, -1], np.int32), X[:0], Q[:0], out[:0]),
           (pdf, 0, np.array([1, -1], np.int32), X, Q, out)], autotune=False).run()
    torch.cuda.synchronize()
    assert torch.equal(out, pdf.xfxQ2(np.array([1, -1], np.int32), X, Q))


def test_one_point_everywhere(nn):
    from paper_2012_08221_gb300.lumi import DeviceEvents, luminosity
    g, pdf, o = nn
    x, q2 = np.array([3.3e-4]), np.array([97.0])
    X, Q = torch.as_tensor(x, device="cuda"), torch.as_tensor(q2, device="cuda")
    got = pdf.xfxQ2(g.pids, X, Q).cpu().numpy()
    parity.check(got, o.xfxq2_batch(g.pids, x, q2), o.kappa(g.pids, x, q2), what="one point")
    pid = np.array([2], np.int32)
    T = pdf.new_tape(1)
    got = pdf.xfxQ2_pw(torch.as_tensor(pid, device="cuda"), X, Q, tape=T).cpu().numpy()
    parity.check(got, o.xfxq2_pw(pid, x, q2), o.kappa(pid, x, q2, pointwise=True), what="one point pw")
    gx, gq, _ = pdf.xfxQ2_backward(torch.as_tensor(pid, device="cuda"), X, Q,
                                   torch.ones(1, dtype=torch.float64, device="cuda"), pointwise=True, tape=T)
    rdx, rdq = o.grad_pw(pid, x, q2)
    assert np.allclose(gx.cpu().numpy(), rdx, rtol=1e-9) and np.allclose(gq.cpu().numpy(), rdq, rtol=1e-9)
    ev = synth.events_lhc(1, seed=72)
    L, lum, a_s = luminosity(pdf, DeviceEvents.from_host(ev))
    Lr, lumr, asr = o.lumi(ev)
    assert abs(L.item() - Lr) <= 1e-12 * (abs(Lr) + 1e3) and L.item() == lum.item()


def test_out_of_device_memory_is_reported_and_leaves_nothing_behind(nn):
    """A grid whose coefficient table cannot fit on the device (2e4 members of
    15 MB: 300 GB) fails to load with PDF_E_NOMEM and a message naming the
    table; the failed allocation leaves no error state behind, so the next
    calls on the thread (a load, a launch) succeed."""
    import ctypes as C
    from paper_2012_08221_gb300._lib import GridDesc, lib
    from paper_2012_08221_gb300.pdf import PDF
    g, pdf, o = nn
    xk = np.ascontiguousarray(g.x_knots, dtype=np.float64)
    nq = np.ascontiguousarray(g.n_q, dtype=np.int32)
    qk = np.ascontiguousarray(g.q_knots, dtype=np.float64)
    pids = np.ascontiguousarray(g.pids, dtype=np.int32)
    d = GridDesc()
    d.n_x, d.x_knots = xk.size, xk.ctypes.data_as(C.POINTER(C.c_double))
    d.n_sub, d.n_q = nq.size, nq.ctypes.data_as(C.POINTER(C.c_int32))
    d.q_knots = qk.ctypes.data_as(C.POINTER(C.c_double))
    d.n_flav, d.pids = pids.size, pids.ctypes.data_as(C.POINTER(C.c_int32))
    d.n_members, d.values, d.alphas, d.interp, d.extrap = 20_000, None, None, 0, 0
    h = C.c_void_p()
    assert lib().pdf_load_grid(C.byref(d), C.byref(h)) == -5          # PDF_E_NOMEM
    assert b"coefficient table" in lib().pdf_last_error()
    x, q2, _ = synth.queries_nnpdf(5003, seed=73)
    p2 = PDF.from_grid(g)
    got = p2.xfxQ2(g.pids, torch.as_tensor(x, device="cuda"), torch.as_tensor(q2, device="cuda"))
    assert torch.equal(got, pdf.xfxQ2(g.pids, torch.as_tensor(x, device="cuda"), torch.as_tensor(q2, device="cuda")))


def _expected_cells(g, x, q2):
    """Largest cell whose lower knot is at or below the point (0 below the
    grid, the last cell above it), on the x knots and on the Q cells of all
    subgrids (a subgrid's last knot opens no cell: an internal threshold
    belongs to the upper subgrid)."""
    xk = np.asarray(g.x_knots)[:-1]
    q2k = np.asarray(g.q_knots, dtype=np.float64) ** 2
    lower, r0 = [], 0
    for n in g.n_q:
        lower.extend(q2k[r0:r0 + n - 1])
        r0 += n
    lower = np.array(lower)
    xc = np.clip(np.searchsorted(xk, x, side="right") - 1, 0, xk.size - 1)
    qc = np.clip(np.searchsorted(lower, q2, side="right") - 1, 0, lower.size - 1)
    return xc, qc


@pytest.mark.parametrize("clustered", [False, True])
def test_knot_search_guided_and_bisected(clustered):
    """The knot searches give the largest cell at or below each point, at
    every knot, one ulp either side of it, on internal thresholds and
    outside the grid: through the guide table on the NNPDF-shaped grid, and
    by bisection on a grid whose x knots cluster within a few hundred ulps
    (no guide width separates them) and whose Q^2 search keeps its guide."""
    import math
    from paper_2012_08221_gb300.pdf import PDF
    g = synth.grid_nnpdf()
    if clustered:
        x = np.concatenate([[1e-9 * (1 + k * 1e-13) for k in range(5)], np.geomspace(1e-6, 1.0, 12)])
        v = np.random.default_rng(70).uniform(0.1, 1.0, (1, g.values.shape[1], x.size, g.values.shape[3]))
        g = synth.Grid(x, g.n_q, g.q_knots, g.pids, v, g.alphas, "clustered")
    pdf = PDF.from_grid(g)
    rng = np.random.default_rng(71)
    xk = np.asarray(g.x_knots)
    q2k = np.asarray(g.q_knots, dtype=np.float64) ** 2
    xs = [np.exp(rng.uniform(math.log(xk[0]) - 2, 0.0, 200_000)), xk, np.nextafter(xk, 0), np.nextafter(xk, 2)]
    qs = [np.exp(rng.uniform(math.log(q2k[0]) - 2, math.log(q2k[-1]) + 2, 200_000)), q2k,
          np.nextafter(q2k, 0), np.nextafter(q2k, np.inf)]
    x, q2 = np.minimum(np.concatenate(xs), 1.0), np.concatenate(qs)
    n = max(x.size, q2.size)                     # every knot of both axes, paired cyclically
    x, q2 = np.resize(x, n), np.resize(q2, n)
    xc, qc, guided = pdf.debug_cells(x, q2)
    assert guided == ((not clustered), True)
    ex, eq = _expected_cells(g, x, q2)
    assert np.array_equal(xc.cpu().numpy(), ex)
    assert np.array_equal(qc.cpu().numpy(), eq)
