"""GPU adjoint: dL/dx, dL/dQ^2 and dL/dvalues against the oracle's analytic
derivative (1e-9 relative), central finite differences, torch.autograd.gradcheck,
and exact sum rules of the grid gradient at the full 1e7-point size."""
import math

import numpy as np
import pytest

from oracle.oracle import OracleGrid
from paper_2012_08221_gb300 import synth
from tests.tinygrids import tiny_two_sub

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GRAD_RTOL = 1e-9


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.fixture(scope="module")
def diffgrid():
    from paper_2012_08221_gb300 import build
    from paper_2012_08221_gb300.pdf import PDF
    build.build()
    g = synth.grid_small(seed=1003, pids=synth.PIDS_13)
    return g, PDF.from_grid(g), OracleGrid.from_synth(g)


def _check(got, ref, scale, what, floor=1e-300):
    err = np.abs(got - ref)
    bound = GRAD_RTOL * np.maximum(np.abs(ref), scale) + floor
    if not np.all(err <= bound):
        i = np.unravel_index(np.argmax(err / bound), err.shape)
        raise AssertionError(f"{what}: {int(np.sum(err > bound))} outside; worst at {i}: got {got[i]!r} "
                             f"ref {ref[i]!r} scale {np.broadcast_to(scale, err.shape)[i]!r} "
                             f"ratio {float(err[i] / bound[i]):.3g}")


def test_pointwise_gradients_against_oracle(diffgrid):
    g, pdf, o = diffgrid
    pid, x, q2, w = synth.queries_pointwise(20_011, seed=41)
    gv = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
    gx, gq, _ = pdf.xfxQ2_backward(cuda(pid), cuda(x), cuda(q2), cuda(w), pointwise=True,
                                   grad_values=gv)
    rdx, rdq = o.grad_pw(pid, x, q2)
    kap = o.kappa(pid, x, q2, pointwise=True)
    U = np.log(g.x_knots)
    W = np.log(g.q_knots ** 2)
    sx = 4 * kap / (np.min(np.diff(U)) * x)
    sq = 4 * kap / (np.min(np.diff(W)) * q2)
    _check(gx.cpu().numpy(), w * rdx, np.abs(w) * sx, "dL/dx")
    _check(gq.cpu().numpy(), w * rdq, np.abs(w) * sq, "dL/dQ2")
    ref = o.dgrid_pw(pid, x, q2, w)
    _check(gv.cpu().numpy(), ref, o.dgrid_pw(pid, x, q2, w, absval=True), "dL/dvalues")


def test_matrix_gradients_against_oracle(lib_small=None):
    from paper_2012_08221_gb300.pdf import PDF
    g = synth.grid_small()
    pdf, o = PDF.from_grid(g), OracleGrid.from_synth(g)
    x, q2 = synth.queries_small(5003, seed=42)
    x[:7] = [1e-9, 1e-9, 0.95, 1.0, 2e-3, 2e-3, 0.5]
    q2[:7] = [1.0, 1e9, 1e9, 30.0, 0.5, 2e8, 1e3]        # extrapolation corners
    pids = np.array([-3, 0, 2, 5, 6], dtype=np.int32)     # 6 absent
    gout = np.random.default_rng(2).standard_normal((x.size, pids.size))
    gv = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
    gx, gq, _ = pdf.xfxQ2_backward(pids, cuda(x), cuda(q2), cuda(gout), grad_values=gv)
    ref = o.dgrid(pids, x, q2, gout)
    _check(gv.cpu().numpy(), ref, o.dgrid(pids, x, q2, gout, absval=True), "matrix dL/dvalues")
    rdx = np.zeros(x.size)
    rdq = np.zeros(x.size)
    for p in range(pids.size):
        dx, dq = o.grad_pw(np.full(x.size, pids[p]), x, q2)
        rdx += gout[:, p] * dx
        rdq += gout[:, p] * dq
    # term scale: kappa of the values, plus the 1e-15 absolute floor of the
    # values (at a knot the oracle's weights vanish exactly, while the
    # coefficient form cancels terms of the neighbouring knots to rounding)
    kap = o.kappa(pids, x, q2).sum(axis=1) + 1e-6 * np.max(np.abs(g.values)) * pids.size
    U = np.log(g.x_knots)
    W = np.log(g.q_knots ** 2)
    gs = np.abs(gout).max(axis=1)
    _check(gx.cpu().numpy(), rdx, gs * 4 * kap / (np.min(np.diff(U)) * x), "matrix dL/dx")
    _check(gq.cpu().numpy(), rdq, gs * 4 * kap / (np.min(np.diff(W)) * q2), "matrix dL/dQ2")


def test_gradient_larger_than_shared_memory():
    """The NNPDF-shaped grid's gradient (1 MB per member) does not fit in
    shared memory: the adjoint adds straight into global memory."""
    from paper_2012_08221_gb300.pdf import PDF
    g = synth.grid_nnpdf()
    pdf, o = PDF.from_grid(g), OracleGrid.from_synth(g)
    x, q2, _ = synth.queries_nnpdf(3001, seed=44)
    pids = np.array([-2, 0, 5], dtype=np.int32)
    gout = np.random.default_rng(45).standard_normal((x.size, pids.size))
    gv = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
    assert gv.numel() * 8 > 200 * 1024
    pdf.xfxQ2_backward(pids, cuda(x), cuda(q2), cuda(gout), grad_values=gv)
    ref = o.dgrid(pids, x, q2, gout)
    _check(gv.cpu().numpy(), ref, o.dgrid(pids, x, q2, gout, absval=True), "global-memory dL/dvalues")


def test_central_finite_differences(diffgrid):
    """h = 1e-6 relative, on points more than 2h (in log) from every knot."""
    g, pdf, o = diffgrid
    rng = np.random.default_rng(43)
    U, W = np.log(g.x_knots), np.log(g.q_knots ** 2)
    x = np.exp(rng.uniform(math.log(1e-6), math.log(0.9), 3000))
    q2 = np.exp(rng.uniform(math.log(4), math.log(2.5e7), 3000))
    h = 1e-6
    far = (np.min(np.abs(np.log(x)[:, None] - U[None]), axis=1) > 4 * h) & \
          (np.min(np.abs(np.log(q2)[:, None] - W[None]), axis=1) > 4 * h)
    x, q2 = x[far][:1000], q2[far][:1000]
    pid = rng.choice(g.pids, x.size).astype(np.int32)
    ones = np.ones(x.size)
    gx, gq, _ = pdf.xfxQ2_backward(cuda(pid), cuda(x), cuda(q2), cuda(ones), pointwise=True)
    f = lambda xx, qq: pdf.xfxQ2_pw(cuda(pid), cuda(xx), cuda(qq)).cpu().numpy()
    fdx = (f(x * (1 + h), q2) - f(x * (1 - h), q2)) / (2 * h * x)
    fdq = (f(x, q2 * (1 + h)) - f(x, q2 * (1 - h))) / (2 * h * q2)
    v = f(x, q2)
    assert np.all(np.abs(gx.cpu().numpy() - fdx) <= 1e-5 * (np.abs(fdx) + np.abs(v) / x))
    assert np.all(np.abs(gq.cpu().numpy() - fdq) <= 1e-5 * (np.abs(fdq) + np.abs(v) / q2))


def test_autograd_gradcheck_tiny_grid():
    """gradcheck in FP64 on a tiny two-subgrid grid.  The differentiable
    inputs are the grid values, ln x and ln Q^2 (x = exp(u) inside), which
    keeps the finite-difference steps well scaled; points stay away from
    knots, where the interpolant is only C1."""
    from paper_2012_08221_gb300.autograd import xfxQ2
    from paper_2012_08221_gb300.pdf import PDF
    g = tiny_two_sub(seed=5)
    pdf = PDF.from_grid(g)
    vals = torch.tensor(g.values, dtype=torch.float64, device="cuda", requires_grad=True)
    rng = np.random.default_rng(44)
    U, W = np.log(g.x_knots), np.log(g.q_knots ** 2)
    us, ws = [], []
    while len(us) < 7:
        u = rng.uniform(math.log(3e-5), math.log(0.5))
        w = rng.uniform(math.log(1.2), math.log(1500.0))
        if np.min(np.abs(U - u)) > 1e-3 and np.min(np.abs(W - w)) > 1e-3:
            us.append(u)
            ws.append(w)
    u = torch.tensor(us, dtype=torch.float64, device="cuda", requires_grad=True)
    w = torch.tensor(ws, dtype=torch.float64, device="cuda", requires_grad=True)
    pids = np.array([-1, 0, 1], dtype=np.int32)
    f = lambda v, a, b: xfxQ2(pdf, v, pids, torch.exp(a), torch.exp(b))
    assert torch.autograd.gradcheck(f, (vals, u, w), eps=1e-6, atol=1e-8, rtol=1e-6)


def test_autograd_matches_oracle_gradient(diffgrid):
    from paper_2012_08221_gb300.autograd import xfxQ2_pw
    g, pdf, o = diffgrid
    pid, x, q2, w = synth.queries_pointwise(5000, seed=45)
    vals = torch.tensor(g.values, device="cuda", requires_grad=True)
    X = cuda(x).requires_grad_(True)
    Q = cuda(q2).requires_grad_(True)
    L = (xfxQ2_pw(pdf, vals, cuda(pid), X, Q) * cuda(w)).sum()
    L.backward()
    ref = o.dgrid_pw(pid, x, q2, w)
    got = vals.grad[0].cpu().numpy()
    _check(got, ref, o.dgrid_pw(pid, x, q2, w, absval=True), "autograd grid")
    rdx, rdq = o.grad_pw(pid, x, q2)
    # per-element term scale of the two derivatives, as in the direct adjoint
    # test above: kappa over the smallest knot spacing, through the chain rule
    kap = o.kappa(pid, x, q2, pointwise=True)
    sx = 4 * kap / (np.min(np.diff(np.log(g.x_knots))) * x)
    sq = 4 * kap / (np.min(np.diff(np.log(g.q_knots ** 2))) * q2)
    _check(X.grad.cpu().numpy(), w * rdx, np.abs(w) * sx, "autograd dL/dx")
    _check(Q.grad.cpu().numpy(), w * rdq, np.abs(w) * sq, "autograd dL/dQ2")


def _pw_points_with_edges(g, n, seed):
    """Pointwise queries over the grid and around it (every side and corner
    outside, knots, an absent pid)."""
    rng = np.random.default_rng(seed)
    U, W = np.log(g.x_knots), np.log(g.q_knots ** 2)
    x = np.exp(rng.uniform(U[0] - 2.0, 0.0, n))
    q2 = np.exp(rng.uniform(W[0] - 1.5, W[-1] + 1.5, n))
    x[:6] = [g.x_knots[0], g.x_knots[3], 1.0, 1e-12, 1e-12, g.x_knots[-2]]
    q2[:6] = [g.q_knots[2] ** 2, 1e12, g.q_knots[-1] ** 2, 1e-3, g.q_knots[4] ** 2, 1e-3]
    pid = rng.choice(np.concatenate([g.pids, [9]]), n).astype(np.int32)     # pid 9 is absent
    w = rng.standard_normal(n)
    return pid, x, q2, w


def test_pointwise_grid_gradient_large_grid_and_edges():
    """Pointwise grid gradient on the NNPDF-shaped grid: 195 x 46 cells x 13
    flavours are more bins than a block's shared-memory counters hold, so the
    sort takes its global-memory path; points outside the grid, at knots and
    with an absent pid included."""
    from paper_2012_08221_gb300.pdf import PDF
    g = synth.grid_nnpdf()
    pdf, o = PDF.from_grid(g), OracleGrid.from_synth(g)
    pid, x, q2, w = _pw_points_with_edges(g, 30_011, 47)
    gv = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
    gx, gq, _ = pdf.xfxQ2_backward(cuda(pid), cuda(x), cuda(q2), cuda(w), pointwise=True, grad_values=gv)
    # absolute floor of 1e-14 sum |w|: points exactly at the last knot of an
    # axis (x = 1, the top Q) get t = 1 - 1 ulp in the kernels, so weights
    # that vanish exactly in the oracle come out at rounding size
    _check(gv.cpu().numpy(), o.dgrid_pw(pid, x, q2, w), o.dgrid_pw(pid, x, q2, w, absval=True),
           "NNPDF pointwise dL/dvalues", floor=1e-14 * np.abs(w).sum())
    rdx, rdq = o.grad_pw(pid, x, q2)
    kap = o.kappa(pid, x, q2, pointwise=True)
    U, W = np.log(g.x_knots), np.log(g.q_knots ** 2)
    dW = np.diff(W)
    _check(gx.cpu().numpy(), w * rdx, np.abs(w) * 4 * kap / (np.min(np.diff(U)) * x), "NNPDF dL/dx")
    _check(gq.cpu().numpy(), w * rdq, np.abs(w) * 4 * kap / (np.min(dW[dW > 0]) * q2), "NNPDF dL/dQ2")
    # the same from the forward's tapes: its bins (466k of them) are counted in
    # global memory too, and dL/dx, dL/dQ^2 keep their bits
    X, Q = cuda(x), cuda(q2)
    T, D = pdf.new_tape(x.size), pdf.new_dtape(x.size)
    pdf.xfxQ2_pw(cuda(pid), X, Q, tape=T, dtape=D)
    gv2 = torch.zeros_like(gv)
    gx2, gq2, _ = pdf.xfxQ2_backward(cuda(pid), X, Q, cuda(w), pointwise=True, grad_values=gv2, tape=T, dtape=D)
    same = lambda a, b: torch.equal(torch.nan_to_num(a, nan=7.0), torch.nan_to_num(b, nan=7.0))
    assert same(gx2, gx) and same(gq2, gq)
    _check(gv2.cpu().numpy(), o.dgrid_pw(pid, x, q2, w), o.dgrid_pw(pid, x, q2, w, absval=True),
           "NNPDF pointwise dL/dvalues from the tapes", floor=1e-14 * np.abs(w).sum())
    assert pdf.status() & 4 == 0                     # no bin out of range (checked builds)


def test_pointwise_grid_gradient_with_more_bins_than_the_block_scan_takes():
    """400 x knots and the NNPDF Q subgrids, 13 flavours: 954k bins, more than
    the scan's one block per 8192 bins goes to (64 blocks), so one block
    scans them all in passes; from the tapes and without."""
    from paper_2012_08221_gb300.pdf import PDF
    xk = synth.log_knots(1e-9, 1.0, 400)
    qk, nq = synth.subgrid_knots([1.0, 1.51, 4.92, 172.5, 1e5], [8, 12, 20, 10])
    g = synth._grid("pw-400x50", xk, qk, nq, synth.PIDS_13, [1010])
    pdf, o = PDF.from_grid(g), OracleGrid.from_synth(g)
    pid, x, q2, w = _pw_points_with_edges(g, 20_011, 48)
    X, Q = cuda(x), cuda(q2)
    ref = o.dgrid_pw(pid, x, q2, w)
    mag = o.dgrid_pw(pid, x, q2, w, absval=True)
    T, D = pdf.new_tape(x.size), pdf.new_dtape(x.size)
    pdf.xfxQ2_pw(cuda(pid), X, Q, tape=T, dtape=D)
    for tape, dtape in ((None, None), (T, D)):
        gv = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
        pdf.xfxQ2_backward(cuda(pid), X, Q, cuda(w), pointwise=True, grad_values=gv, tape=tape, dtape=dtape)
        _check(gv.cpu().numpy(), ref, mag, "400x50 pointwise dL/dvalues", floor=1e-14 * np.abs(w).sum())


def test_pointwise_grid_gradient_in_several_sort_rounds(diffgrid, monkeypatch):
    """The sorted adjoint works in rounds of at most $PDFGPU_SORT_CHUNK points:
    with rounds of 1000 points (several rounds, a ragged last one), with and
    without the forward tape, the gradients equal the oracle's and dL/dx,
    dL/dQ^2 equal those of one round bit for bit."""
    g, pdf, o = diffgrid
    pid, x, q2, w = _pw_points_with_edges(g, 20_011, 48)
    P, X, Q, Wt = cuda(pid), cuda(x), cuda(q2), cuda(w)
    tape = pdf.new_tape(x.size)
    pdf.xfxQ2_pw(P, X, Q, tape=tape)
    ref = o.dgrid_pw(pid, x, q2, w)
    mag = o.dgrid_pw(pid, x, q2, w, absval=True)
    one = pdf.xfxQ2_backward(P, X, Q, Wt, pointwise=True,
                             grad_values=torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda"))
    monkeypatch.setenv("PDFGPU_SORT_CHUNK", "1000")
    for t in (tape, None):
        gv = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
        gx, gq, _ = pdf.xfxQ2_backward(P, X, Q, Wt, pointwise=True, grad_values=gv, tape=t)
        _check(gv.cpu().numpy(), ref, mag, "rounds of 1000 points", floor=1e-14 * np.abs(w).sum())
        assert torch.equal(gx, one[0]) and torch.equal(gq, one[1])


def test_full_size_sum_rules(diffgrid):
    """Full 1e7 pointwise workload through autograd.  Exact sum rules of the
    grid gradient (the interpolation reproduces constants and functions
    linear in ln x): sum_cells dL/dv[.][a] = sum_{i: a_i = a} w_i and
    sum_cells U_k dL/dv[.][k][a] = sum_{i: a_i = a} w_i ln x_i; the whole grid
    gradient against the oracle; sampled dL/dx and dL/dQ^2 against the
    oracle."""
    from paper_2012_08221_gb300.autograd import xfxQ2_pw
    g, pdf, o = diffgrid
    pid, x, q2, w = synth.queries_pointwise()
    vals = torch.tensor(g.values, device="cuda", requires_grad=True)
    X = cuda(x).requires_grad_(True)
    Q = cuda(q2).requires_grad_(True)
    W_ = cuda(w)
    L = (xfxQ2_pw(pdf, vals, cuda(pid), X, Q) * W_).sum()
    L.backward()
    G = vals.grad[0].cpu().numpy()
    U = np.log(g.x_knots)
    for a, p in enumerate(g.pids):
        m = pid == p
        s0 = G[:, :, a].sum()
        want0 = w[m].sum()
        assert abs(s0 - want0) <= 1e-9 * np.abs(w[m]).sum()
        s1 = (G[:, :, a] * U[None, :]).sum()
        want1 = (w[m] * np.log(x[m])).sum()
        assert abs(s1 - want1) <= 1e-9 * np.abs(w[m] * np.log(x[m])).sum()
    # the whole grid gradient against the oracle (run chunked on the host cores)
    from tests.oracle_pool import dgrid_pw_parallel
    spec = ("grid_small", {"seed": 1003, "pids": synth.PIDS_13})
    ref = dgrid_pw_parallel(*spec, pid, x, q2, w)
    mag = dgrid_pw_parallel(*spec, pid, x, q2, w, absval=True)
    _check(G, ref, mag, "full-size grid gradient")
    idx = np.random.default_rng(6).choice(x.size, 2000, replace=False)
    rdx, rdq = o.grad_pw(pid[idx], x[idx], q2[idx])
    gx = X.grad[cuda(idx)].cpu().numpy()
    gq = Q.grad[cuda(idx)].cpu().numpy()
    kap = o.kappa(pid[idx], x[idx], q2[idx], pointwise=True)
    Ud, Wd = np.min(np.diff(U)), np.min(np.diff(np.log(g.q_knots ** 2)))
    _check(gx, w[idx] * rdx, np.abs(w[idx]) * 4 * kap / (Ud * x[idx]), "full dL/dx")
    _check(gq, w[idx] * rdq, np.abs(w[idx]) * 4 * kap / (Wd * q2[idx]), "full dL/dQ2")


def test_matrix_form_full_size_through_autograd(diffgrid):
    """The matrix form as the benchmark times it: 1e6 points x all 13
    flavours, L = sum_ia w_ia xf_a(x_i, Q^2_i) through torch.autograd (the
    forward keeps the tape; the adjoint sorts by cell and half pair with one
    accumulator per column).  The whole grid gradient against the oracle;
    sampled dL/dx and dL/dQ^2 against the oracle's analytic derivative; the
    flavour sum rule sum_cells dL/dv[.][a] = sum_i w_ia."""
    from paper_2012_08221_gb300.autograd import xfxQ2
    g, pdf, o = diffgrid
    nm = 1_000_000
    _, x, q2, _ = synth.queries_pointwise()
    x, q2 = x[:nm].copy(), q2[:nm].copy()
    gout = np.random.default_rng(7).standard_normal((nm, g.n_flav))
    pids = np.asarray(g.pids, dtype=np.int32)
    vals = torch.tensor(g.values, device="cuda", requires_grad=True)
    X = cuda(x).requires_grad_(True)
    Q = cuda(q2).requires_grad_(True)
    (xfxQ2(pdf, vals, pids, X, Q) * cuda(gout)).sum().backward()
    G = vals.grad[0].cpu().numpy()
    for a in range(g.n_flav):
        assert abs(G[:, :, a].sum() - gout[:, a].sum()) <= 1e-9 * np.abs(gout[:, a]).sum()
    from tests.oracle_pool import dgrid_parallel
    spec = ("grid_small", {"seed": 1003, "pids": synth.PIDS_13})
    ref = dgrid_parallel(*spec, pids, x, q2, gout)
    mag = dgrid_parallel(*spec, pids, x, q2, gout, absval=True)
    _check(G, ref, mag, "full-size matrix-form grid gradient")
    idx = np.random.default_rng(8).choice(nm, 2000, replace=False)
    rdx, rdq = np.zeros(idx.size), np.zeros(idx.size)
    for a, p in enumerate(pids):
        dx, dq = o.grad_pw(np.full(idx.size, p, dtype=np.int32), x[idx], q2[idx])
        rdx += gout[idx, a] * dx
        rdq += gout[idx, a] * dq
    kap = o.kappa(pids, x[idx], q2[idx]).sum(axis=1)
    gs = np.abs(gout[idx]).max(axis=1)
    U, W = np.log(g.x_knots), np.log(g.q_knots ** 2)
    gx = X.grad[cuda(idx)].cpu().numpy()
    gq = Q.grad[cuda(idx)].cpu().numpy()
    _check(gx, rdx, gs * 4 * kap / (np.min(np.diff(U)) * x[idx]), "full matrix dL/dx")
    _check(gq, rdq, gs * 4 * kap / (np.min(np.diff(W)) * q2[idx]), "full matrix dL/dQ2")


def test_alphas_derivative_and_autograd():
    from paper_2012_08221_gb300.autograd import alphasQ2
    from paper_2012_08221_gb300.pdf import PDF
    g = synth.grid_nnpdf()
    pdf, o = PDF.from_grid(g), OracleGrid.from_synth(g)
    q2 = np.exp(np.random.default_rng(50).uniform(math.log(0.1), math.log(1e11), 5000))
    v, d = pdf.alphasQ2_grad(cuda(q2))
    ref = np.array([o.alphas_grad(q) for q in q2])
    assert np.allclose(v.cpu().numpy(), ref[:, 0], rtol=1e-12, atol=0)
    assert np.allclose(d.cpu().numpy(), ref[:, 1], rtol=1e-9, atol=1e-12 * np.max(np.abs(ref[:, 1])))
    Q = cuda(q2[:6]).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda z: alphasQ2(pdf, z), (Q,), eps=1e-6 * float(Q.min()),
                                    atol=1e-9, rtol=1e-5)


def _points_with_edges(g, n, seed):
    """Points inside, below and above both knot ranges, plus domain errors."""
    rng = np.random.default_rng(seed)
    U, W = np.log(g.x_knots), np.log(g.q_knots ** 2)
    x = np.exp(rng.uniform(U[0] - 2, 0.0, n))
    q2 = np.exp(rng.uniform(W[0] - 2, W[-1] + 2, n))
    x[:4] = [0.0, 1.5, np.nan, 1.0]
    q2[4:7] = [-1.0, np.inf, np.nan]
    return x, q2


@pytest.mark.parametrize("extrap", ["linear", "freeze", "error"])
def test_tape_gives_the_same_forward_and_adjoint(extrap):
    """The forward calls that write the adjoint tape give the same outputs,
    and the adjoint from the tape the same dL/dx and dL/dQ^2 bit for bit (the
    grid gradient up to the order of the atomic sums), pointwise and for a
    shared pid list, on a two-subgrid grid, the small grid (shared-memory
    gradient) and the NNPDF-shaped grid (global-memory gradient), with
    points outside the grid and domain errors."""
    from paper_2012_08221_gb300.pdf import PDF
    same = lambda a, b: torch.equal(torch.nan_to_num(a, nan=7.0), torch.nan_to_num(b, nan=7.0))
    for g in (tiny_two_sub(seed=51), synth.grid_small(seed=1003, pids=synth.PIDS_13), synth.grid_nnpdf()):
        pdf = PDF.from_grid(g, extrap=extrap)
        x, q2 = _points_with_edges(g, 30_011, 52)
        X, Q = cuda(x), cuda(q2)
        rng = np.random.default_rng(53)
        pid = cuda(rng.choice(np.append(g.pids, 7), x.size).astype(np.int32))   # 7: absent
        pids = np.array([g.pids[0], 21, g.pids[-1], 7], dtype=np.int32)
        T = pdf.new_tape(x.size)
        D = pdf.new_dtape(x.size)
        for pointwise in (True, False):
            if pointwise:
                ref = pdf.xfxQ2_pw(pid, X, Q)
                got = pdf.xfxQ2_pw(pid, X, Q, tape=T)
                assert same(pdf.xfxQ2_pw(pid, X, Q, tape=T, dtape=D), ref)
                gout = cuda(rng.standard_normal(x.size))
                ids = pid
            else:
                ref = pdf.xfxQ2(pids, X, Q)
                got = pdf.xfxQ2(pids, X, Q, tape=T)
                gout = cuda(rng.standard_normal((x.size, pids.size)))
                ids = pids
            assert same(got, ref)
            gv0 = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
            gv1 = torch.zeros_like(gv0)
            gx0, gq0, _ = pdf.xfxQ2_backward(ids, X, Q, gout, pointwise=pointwise, grad_values=gv0)
            gx1, gq1, _ = pdf.xfxQ2_backward(ids, X, Q, gout, pointwise=pointwise, grad_values=gv1, tape=T)
            assert same(gx1, gx0) and same(gq1, gq0)
            assert torch.allclose(gv1, gv0, rtol=1e-12, atol=1e-15 * float(gv0.abs().max()))
            assert bool(torch.isnan(gx1[[0, 1, 2, 4, 5, 6]]).all()) and not bool(torch.isnan(gx1[3]))   # x = 1 is valid
            if pointwise:
                # the derivative tape: the same bits, with and without the grid
                # gradient (sorted record pass / plain adjoint)
                gv2 = torch.zeros_like(gv0)
                gx2, gq2, _ = pdf.xfxQ2_backward(ids, X, Q, gout, pointwise=True, grad_values=gv2, tape=T,
                                                 dtape=D)
                assert same(gx2, gx0) and same(gq2, gq0)
                assert torch.allclose(gv2, gv0, rtol=1e-12, atol=1e-15 * float(gv0.abs().max()))
                gx3, gq3, _ = pdf.xfxQ2_backward(ids, X, Q, gout, pointwise=True, tape=T, dtape=D)
                assert same(gx3, gx0) and same(gq3, gq0)
                absent = (pid == 7).nonzero().flatten()
                n = x.size
                assert bool((D[:2 * n].view(n, 2)[absent] == 0).all())
                bins = D[2 * n:].view(torch.int32)[:n]
                assert bool((bins[absent] == -1).all()) and bool((bins[[0, 1, 2, 4, 5, 6]] == -1).all())
        torch.cuda.synchronize()


def test_tape_survives_new_values_and_other_members():
    """A tape depends on the points and the knots only: after binding other
    values, and for another member, the adjoint from the old tape equals the
    adjoint that recomputes the coordinates."""
    from paper_2012_08221_gb300.pdf import PDF
    g = synth.grid_nnpdf(seeds=(1005, 1006))
    pdf = PDF.from_grid(g)
    x, q2, _ = synth.queries_nnpdf(20_003, seed=54)
    X, Q = cuda(x), cuda(q2)
    pids = np.array([-1, 0, 2], dtype=np.int32)
    T = pdf.new_tape(x.size)
    pdf.xfxQ2(pids, X, Q, tape=T)
    pdf.bind_values(cuda(g.values * 1.5 - 0.25))
    gout = cuda(np.random.default_rng(55).standard_normal((x.size, 3)))
    for m in (0, 1):
        gv0 = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
        gv1 = torch.zeros_like(gv0)
        gx0, gq0, _ = pdf.xfxQ2_backward(pids, X, Q, gout, member=m, grad_values=gv0)
        gx1, gq1, _ = pdf.xfxQ2_backward(pids, X, Q, gout, member=m, grad_values=gv1, tape=T)
        assert torch.equal(gx0, gx1) and torch.equal(gq0, gq1)
        assert torch.allclose(gv1, gv0, rtol=1e-12, atol=1e-15 * float(gv0.abs().max()))


def test_derivative_tape_keeps_the_forward_values():
    """The derivative tape holds the patch derivatives of the values bound
    at the forward call: after other values are bound, the adjoint from it
    still gives dL/dx and dL/dQ^2 of the forward's values (the same bits as
    the adjoint with those values bound again), and its grid gradient, which
    does not depend on the values, is unchanged.  Through autograd two
    evaluations with different values on one handle, backward in the
    opposite order, each get their own values' gradients."""
    from paper_2012_08221_gb300.autograd import xfxQ2_pw as ad_xfxQ2_pw
    from paper_2012_08221_gb300.pdf import PDF
    g = synth.grid_small(seed=1003, pids=synth.PIDS_13)
    pdf = PDF.from_grid(g)
    pid, x, q2, w = synth.queries_pointwise(20_011, seed=57)
    P, X, Q, W_ = cuda(pid), cuda(x), cuda(q2), cuda(w)
    T, D = pdf.new_tape(x.size), pdf.new_dtape(x.size)
    V1, V2 = cuda(g.values), cuda(g.values * 1.5 - 0.25)
    pdf.bind_values(V1)
    pdf.xfxQ2_pw(P, X, Q, tape=T, dtape=D)
    pdf.bind_values(V2)
    gv = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
    gx, gq, _ = pdf.xfxQ2_backward(P, X, Q, W_, pointwise=True, grad_values=gv, tape=T, dtape=D)
    pdf.bind_values(V1)
    gv0 = torch.zeros_like(gv)
    gx0, gq0, _ = pdf.xfxQ2_backward(P, X, Q, W_, pointwise=True, grad_values=gv0, tape=T)
    assert torch.equal(gx, gx0) and torch.equal(gq, gq0)
    assert torch.allclose(gv, gv0, rtol=1e-12, atol=1e-15 * float(gv0.abs().max()))
    # autograd: forward V1, forward V2, backward V2, backward V1
    A1, A2 = V1.clone().requires_grad_(True), V2.clone().requires_grad_(True)
    X1, X2 = X.clone().requires_grad_(True), X.clone().requires_grad_(True)
    L1 = (ad_xfxQ2_pw(pdf, A1, P, X1, Q) * W_).sum()
    L2 = (ad_xfxQ2_pw(pdf, A2, P, X2, Q) * W_).sum()
    L2.backward()
    L1.backward()
    assert torch.equal(X1.grad, gx0)
    pdf.bind_values(V2)
    gx2, _, _ = pdf.xfxQ2_backward(P, X, Q, W_, pointwise=True, tape=T)
    assert torch.equal(X2.grad, gx2)


def test_tape_arguments_are_checked():
    from paper_2012_08221_gb300._lib import PdfError
    from paper_2012_08221_gb300.pdf import PDF
    g = synth.grid_small(seed=1003, pids=synth.PIDS_13)
    pdf = PDF.from_grid(g)
    x, q2 = synth.queries_small(1001, seed=56)
    X, Q = cuda(x), cuda(q2)
    pid = cuda(np.full(x.size, 2, np.int32))
    buf = torch.empty(4 * x.size + 4, dtype=torch.float64, device="cuda")
    odd = buf[1:1 + 4 * x.size]                       # 8-byte aligned only
    with pytest.raises(PdfError):
        pdf.xfxQ2_pw(pid, X, Q, tape=odd)
    with pytest.raises(PdfError):
        pdf.xfxQ2_backward(pid, X, Q, cuda(np.ones(x.size)), pointwise=True, tape=odd)
    pc = PDF.from_grid(g, extrap="continuation")
    with pytest.raises(PdfError):
        pc.xfxQ2(g.pids, X, Q, tape=pc.new_tape(x.size))
    with pytest.raises(AssertionError):
        pdf.xfxQ2_pw(pid, X, Q, tape=pdf.new_tape(x.size - 1))
    # the derivative tape: 16-byte aligned, with a tape, pointwise form only
    from paper_2012_08221_gb300._lib import lib
    from paper_2012_08221_gb300.pdf import _ptr, _stream
    T = pdf.new_tape(x.size)
    D = pdf.new_dtape(x.size)
    dbuf = torch.empty(pdf.dtape_doubles(x.size) + 2, dtype=torch.float64, device="cuda")
    out = torch.empty(x.size, dtype=torch.float64, device="cuda")
    gout = cuda(np.ones(x.size))
    st = _stream(pdf.device)
    assert lib().xfxQ2_pw_tape(pdf.handle, 0, _ptr(pid), _ptr(X), _ptr(Q), x.size, _ptr(out), _ptr(T),
                               _ptr(dbuf[1:]), st) != 0
    assert lib().xfxQ2_pw_tape(pdf.handle, 0, _ptr(pid), _ptr(X), _ptr(Q), x.size, _ptr(out), None,
                               _ptr(D), st) != 0
    pdf.xfxQ2_pw(pid, X, Q, tape=T, dtape=D)
    pids = np.array([2], dtype=np.int32)
    assert lib().xfxQ2_backward_tape(pdf.handle, 0, pids.ctypes.data, 1, 0, _ptr(X), _ptr(Q), x.size,
                                     _ptr(T), _ptr(D), _ptr(gout), None, None, None, st) != 0
    assert lib().xfxQ2_backward_tape(pdf.handle, 0, _ptr(pid), 0, 1, _ptr(X), _ptr(Q), x.size,
                                     _ptr(T), _ptr(dbuf[1:]), _ptr(gout), None, None, None, st) != 0
    torch.cuda.synchronize()
    # autograd on a continuation grid still runs its forward (no tape)
    from paper_2012_08221_gb300.autograd import xfxQ2 as ad_xfxQ2
    vals = torch.tensor(g.values, device="cuda", requires_grad=True)
    assert torch.equal(ad_xfxQ2(pc, vals, g.pids, X, Q), pc.xfxQ2(g.pids, X, Q))


@pytest.mark.parametrize("n_pid", [1, 3, 16, 17])
def test_matrix_grid_gradient_sorted_and_beyond_16_columns(n_pid):
    """The matrix form's grid gradient: up to 16 columns the points are
    sorted by cell and every column accumulates in the same bin; beyond 16
    the weights are scattered with atomics.  Columns include an absent pid
    and the gluon twice (0 and 21, both adding to one column); points on
    every side of the grid and at knots; with and without the tape."""
    from paper_2012_08221_gb300.pdf import PDF
    g = synth.grid_small(seed=1003, pids=synth.PIDS_13)
    pdf, o = PDF.from_grid(g), OracleGrid.from_synth(g)
    base = [0, 21, 9, -3, 2, 5] + list(synth.PIDS_13)
    pids = np.array((base * 2)[:n_pid], dtype=np.int32)
    _, x, q2, _ = _pw_points_with_edges(g, 8_003, 49)
    gout = np.random.default_rng(50).standard_normal((x.size, pids.size))
    X, Q = cuda(x), cuda(q2)
    T = pdf.new_tape(x.size)
    pdf.xfxQ2(pids, X, Q, tape=T)
    ref = o.dgrid(pids, x, q2, gout)
    mag = o.dgrid(pids, x, q2, gout, absval=True)
    rdx = np.zeros(x.size)
    rdq = np.zeros(x.size)
    for p in range(pids.size):
        dx, dq = o.grad_pw(np.full(x.size, pids[p]), x, q2)
        rdx += gout[:, p] * dx
        rdq += gout[:, p] * dq
    kap = o.kappa(pids, x, q2).sum(axis=1) + 1e-6 * np.max(np.abs(g.values)) * pids.size
    U, W = np.log(g.x_knots), np.log(g.q_knots ** 2)
    gs = np.abs(gout).max(axis=1)
    for tape in (None, T):
        gv = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
        gx, gq, _ = pdf.xfxQ2_backward(pids, X, Q, cuda(gout), grad_values=gv, tape=tape)
        _check(gv.cpu().numpy(), ref, mag, f"matrix dL/dvalues, {n_pid} columns",
               floor=1e-14 * np.abs(gout).sum())
        _check(gx.cpu().numpy(), rdx, gs * 4 * kap / (np.min(np.diff(U)) * x), "matrix dL/dx")
        _check(gq.cpu().numpy(), rdq, gs * 4 * kap / (np.min(np.diff(W)) * q2), "matrix dL/dQ2")


def test_grid_gradient_near_the_knots_is_accurate():
    """Points a little below a knot (t = 1 - 1e-3 ... 1 - 1e-4) and a little
    above one (t = 1e-3 ... 1e-4) on both axes, each alone in its cell: the
    stencil weights that vanish at the near knot are of order (1 - t)^2 or
    t^2 there (powers of t alone would lose 15 ulp / (1 - t)^2 of them, over
    1e-9 below t = 1 - 1e-3).  Both the pointwise and the matrix form must
    match the oracle's gradient within 1e-9 of each value's own term scale,
    with no absolute floor.  (Closer to a knot the rounding of t itself,
    about 1e-15 between the two sides' logarithms, moves such a weight by
    more than 1e-9 of itself.)"""
    from paper_2012_08221_gb300.pdf import PDF
    g = synth.grid_small(seed=1003, pids=synth.PIDS_13)
    pdf, o = PDF.from_grid(g), OracleGrid.from_synth(g)
    U, W = np.log(g.x_knots), np.log(g.q_knots ** 2)
    us, ws = [], []
    for k, d in enumerate([1e-3, 5e-4, 2e-4, 1e-4]):
        for lo in (False, True):
            kx, kq = 3 + 7 * k + (0 if lo else 3), 2 + 3 * k
            tx = d if lo else 1.0 - d
            tq = 1.0 - d if lo else d
            us.append(U[kx] + tx * (U[kx + 1] - U[kx]))
            ws.append(W[kq] + tq * (W[kq + 1] - W[kq]))
    x, q2 = np.exp(np.array(us)), np.exp(np.array(ws))
    rng = np.random.default_rng(60)
    pid = g.pids[rng.integers(0, g.n_flav, x.size)].astype(np.int32)
    w = rng.standard_normal(x.size)
    gv = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
    pdf.xfxQ2_backward(cuda(pid), cuda(x), cuda(q2), cuda(w), pointwise=True, grad_values=gv)
    _check(gv.cpu().numpy(), o.dgrid_pw(pid, x, q2, w), o.dgrid_pw(pid, x, q2, w, absval=True),
           "pointwise dL/dvalues near knots")
    pids = np.array([-2, 0, 3], dtype=np.int32)
    gout = rng.standard_normal((x.size, pids.size))
    gv = torch.zeros(g.values.shape[1:], dtype=torch.float64, device="cuda")
    pdf.xfxQ2_backward(pids, cuda(x), cuda(q2), cuda(gout), grad_values=gv)
    _check(gv.cpu().numpy(), o.dgrid(pids, x, q2, gout), o.dgrid(pids, x, q2, gout, absval=True),
           "matrix dL/dvalues near knots")
