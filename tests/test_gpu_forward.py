"""GPU parity of the forward kernels against the FP64 oracle (through the C ABI).

Sizes: the small grid workload in full (1e5 points x 11 flavours), the
NNPDF-shaped workload on 300001 points (many tiles plus a ragged tail) and at
its full 1e7 points in the benchmark's launch configuration, where every
output is checked against the oracle.
"""
import math

import numpy as np
import pytest

from oracle.oracle import OracleGrid
from paper_2012_08221_gb300 import synth
from tests import parity
from tests.golden_io import load as load_golden
from tests.tinygrids import tiny_two_sub

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib_built():
    from paper_2012_08221_gb300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def small(lib_built):
    from paper_2012_08221_gb300.pdf import PDF
    g = synth.grid_small()
    return g, PDF.from_grid(g), OracleGrid.from_synth(g)


@pytest.fixture(scope="module")
def nnpdf(lib_built):
    from paper_2012_08221_gb300.pdf import PDF
    g = synth.grid_nnpdf()
    return g, PDF.from_grid(g), OracleGrid.from_synth(g)


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def test_small_grid_full_workload(small):
    """The small-grid workload in full, as the benchmark runs it: x*f of all
    11 flavours and alpha_s at the same Q^2, in one launch (the same bits as
    the two calls) and against the oracle."""
    g, pdf, o = small
    x, q2 = synth.queries_small()
    X, Q = cuda(x), cuda(q2)
    got = pdf.xfxQ2(g.pids, X, Q)
    ref = o.xfxq2_batch(g.pids, x, q2)
    kap = o.kappa(g.pids, x, q2)
    parity.check(got.cpu().numpy(), ref, kap, what="small grid xfxQ2")
    out, a_s = pdf.xfxQ2_alphasQ2(g.pids, X, Q)
    assert torch.equal(out.view(torch.int64), got.view(torch.int64))
    assert torch.equal(a_s.view(torch.int64), pdf.alphasQ2(Q).view(torch.int64))
    parity.check(a_s.cpu().numpy(), o.alphas_batch(q2), o.alphas_kappa(q2), what="small grid alpha_s")
    assert pdf.status() == 0


def test_nnpdf_many_tiles_ragged_tail(nnpdf):
    """Also counts the outputs that a plain 1e-12 relative test (no kappa)
    would reject: values that nearly cancel, where the two sides' rounding
    orders differ on the scale of the terms, not of the result."""
    g, pdf, o = nnpdf
    x, q2, _ = synth.queries_nnpdf(300_001, seed=12)
    got = pdf.xfxQ2(g.pids, cuda(x), cuda(q2)).cpu().numpy()
    ref = o.xfxq2_batch(g.pids, x, q2)
    kap = o.kappa(g.pids, x, q2)
    worst = parity.check(got, ref, kap, what="nnpdf xfxQ2")
    strict = parity.strict_count(got, ref)
    print(f"\nnnpdf xfxQ2: worst error / scale {worst:.2e}; "
          f"plain 1e-12 relative test would reject {strict} of {ref.size}")
    assert strict <= 1e-4 * ref.size


def test_output_alignment_and_odd_runs(nnpdf):
    """Both exits of the staged output rows give the same values: the bulk
    copy (16-byte aligned runs of a multiple of 16 bytes) and the warp-wide
    stores (an output 8 bytes off a 16-byte boundary; the odd-length run of
    the ragged last warp)."""
    g, pdf, o = nnpdf
    x, q2, _ = synth.queries_nnpdf(100_003, seed=31)
    X, Q = cuda(x), cuda(q2)
    for pids in (g.pids, g.pids[:3], g.pids[:1]):
        k = len(pids)
        aligned = pdf.xfxQ2(pids, X, Q)
        assert aligned.data_ptr() % 16 == 0
        buf = torch.empty(x.size * k + 1, dtype=torch.float64, device="cuda")
        shifted = buf[1:].view(x.size, k)
        assert shifted.data_ptr() % 16 == 8
        pdf.xfxQ2(pids, X, Q, out=shifted)
        assert torch.equal(aligned, shifted)
        ref = o.xfxq2_batch(pids, x, q2)
        parity.check(shifted.cpu().numpy(), ref, o.kappa(pids, x, q2), what=f"shifted output, {k} pids")


def test_host_buffer_path(nnpdf):
    """xfxQ2_host, the end-to-end entry point: several chunks through the
    three staging slots and a ragged last chunk, pinned and pageable host
    buffers; equal bit for bit to the device-resident call, and to the
    oracle on a sample; a domain error gives a NaN row and the status bit."""
    g, pdf, o = nnpdf
    n = 3 * (1 << 18) + 12_345
    x, q2, _ = synth.queries_nnpdf(n, seed=33)
    x[7] = -1.0
    dev = pdf.xfxQ2(g.pids, cuda(x), cuda(q2)).cpu()
    assert pdf.status() == 1
    got = pdf.xfxQ2_host(g.pids, torch.as_tensor(x).pin_memory(), torch.as_tensor(q2).pin_memory())
    assert torch.equal(got[8:], dev[8:]) and torch.equal(got[:7], dev[:7])
    assert torch.isnan(got[7]).all()
    assert pdf.status() == 1
    two = pdf.xfxQ2_host(g.pids[:2], torch.as_tensor(x), torch.as_tensor(q2))
    assert torch.equal(two[8:], dev[8:, :2])
    assert pdf.status() == 1
    idx = np.random.default_rng(33).choice(np.arange(8, n), 2000, replace=False)
    ref = o.xfxq2_batch(g.pids, x[idx], q2[idx])
    parity.check(got.numpy()[idx], ref, o.kappa(g.pids, x[idx], q2[idx]), what="xfxQ2_host")


def test_nnpdf_full_size_every_output(nnpdf):
    """The full 1e7-point workload in one launch, as the benchmark runs it:
    every one of the 1.3e8 x*f outputs and the 1e7 alpha_s values against the
    oracle (compared in chunks of 1e6 points on the host cores)."""
    g, pdf, o = nnpdf
    x, q2, q2a = synth.queries_nnpdf()
    X, Q = cuda(x), cuda(q2)
    out = pdf.xfxQ2(g.pids, X, Q)
    a_s = pdf.alphasQ2(cuda(q2a)).cpu().numpy()
    assert pdf.status() == 0
    step = 1_000_000
    strict = 0
    for s0 in range(0, x.size, step):
        sl = slice(s0, s0 + step)
        got = out[sl].cpu().numpy()
        ref = o.xfxq2_batch(g.pids, x[sl], q2[sl])
        parity.check(got, ref, o.kappa(g.pids, x[sl], q2[sl]), what=f"nnpdf full size, points {s0}+")
        strict += parity.strict_count(got, ref)
    print(f"\nfull size: plain 1e-12 relative test would reject {strict} of {out.numel()}")
    assert strict == 0
    ra = o.alphas_batch(q2a)
    parity.check(a_s, ra, o.alphas_kappa(q2a), what="alphas full size")
    assert parity.strict_count(a_s, ra) == 0


def test_alphas_parity(small, nnpdf):
    for g, pdf, o in (small, nnpdf):
        q2 = np.exp(np.random.default_rng(4).uniform(math.log(0.01), math.log(1e12), 200_003))
        got = pdf.alphasQ2(cuda(q2)).cpu().numpy()
        ref = o.alphas_batch(q2)
        parity.check(got, ref, o.alphas_kappa(q2), what=f"alphas {g.name}")


def test_xfxq_is_xfxq2_of_q_squared(small):
    g, pdf, o = small
    x, q2 = synth.queries_small(10_007, seed=31)
    q = np.sqrt(q2)
    a = pdf.xfxQ(g.pids, cuda(x), cuda(q)).cpu().numpy()
    b = pdf.xfxQ2(g.pids, cuda(x), cuda(q * q)).cpu().numpy()
    assert np.array_equal(a, b)
    qa = pdf.alphasQ(cuda(q)).cpu().numpy()
    qb = pdf.alphasQ2(cuda(q * q)).cpu().numpy()
    assert np.array_equal(qa, qb)


def test_pointwise_parity(lib_built):
    from paper_2012_08221_gb300.pdf import PDF
    g = synth.grid_small(seed=1003, pids=synth.PIDS_13)
    pdf, o = PDF.from_grid(g), OracleGrid.from_synth(g)
    pid, x, q2, _ = synth.queries_pointwise(200_003)
    pid[::7] = 21                               # the gluon under its other name
    pid[::11] = 9                               # a pid not in the grid
    got = pdf.xfxQ2_pw(cuda(pid), cuda(x), cuda(q2)).cpu().numpy()
    ref = o.xfxq2_pw(pid, x, q2)
    kap = o.kappa(pid, x, q2, pointwise=True)
    parity.check(got, ref, kap, what="pointwise")
    assert np.all(got[::11] == 0.0)
    # matrix form, same points: column of the point's pid
    full = pdf.xfxQ2(g.pids, cuda(x), cuda(q2)).cpu().numpy()
    col = {int(p): i for i, p in enumerate(g.pids)}
    sel = np.array([col.get(0 if p == 21 else int(p), -1) for p in pid])
    m = sel >= 0
    assert np.array_equal(full[np.arange(x.size)[m], sel[m]], got[m])


def test_golden_exact_values(lib_built):
    from paper_2012_08221_gb300.pdf import PDF
    g, x, q2, exp, exp_as = load_golden()
    pdf, o = PDF.from_grid(g), OracleGrid.from_synth(g)
    got = pdf.xfxQ2(g.pids, cuda(x), cuda(q2)).cpu().numpy()
    parity.check(got, exp, o.kappa(g.pids, x, q2), what="golden")
    parity.check(pdf.alphasQ2(cuda(q2)).cpu().numpy(), exp_as, o.alphas_kappa(q2), what="golden alphas")


def test_edge_cases(nnpdf):
    g, pdf, o = nnpdf
    pids = np.array([-6, 0, 21, 3, 7, 22], dtype=np.int32)     # 7, 22 absent
    xs, qs = [], []
    for k in range(g.n_x):                       # every knot, several rows
        for r in (0, 7, 8, 19, 20, 39, 40, 49):
            xs.append(g.x_knots[k])
            qs.append(g.q_knots[r] ** 2)
    for v in (1.0, np.nextafter(1.0, 0), 1e-9, np.nextafter(1e-9, 0), 1e-12, 3e-300, 5e-324):
        for q2 in (1.0, np.nextafter(1.0, 0), 0.04, 1e10, 3e10, 1.51 ** 2, 4.92 ** 2, 172.5 ** 2):
            xs.append(v)
            qs.append(q2)
    nan, inf = float("nan"), float("inf")
    bad = [(0.0, 10.0), (-1e-3, 10.0), (1.0 + 2e-16, 10.0), (0.1, 0.0), (0.1, -4.0), (nan, 10.0),
           (0.1, nan), (0.1, inf), (inf, 10.0), (-0.0, 10.0)]
    xs += [b[0] for b in bad]
    qs += [b[1] for b in bad]
    x, q2 = np.array(xs), np.array(qs)
    pdf.status()
    got = pdf.xfxQ2(pids, cuda(x), cuda(q2)).cpu().numpy()
    assert pdf.status() & 1
    assert pdf.status() == 0                     # reading clears
    ref = o.xfxq2_batch(pids, x, q2)
    kap = o.kappa(pids, x, q2)
    parity.check(got, ref, kap, what="edge cases")
    nb = len(bad)
    assert np.all(np.isnan(got[-nb:]))
    assert np.all(got[:-nb, 4] == 0.0) and np.all(got[:-nb, 5] == 0.0)
    assert np.array_equal(got[:, 1], got[:, 2], equal_nan=True)  # pid 0 and 21
    # knots reproduce the stored values (upper subgrid at thresholds)
    n_k = g.n_x * 8
    rows = np.tile([0, 8, 8, 20, 20, 40, 40, 49], g.n_x)
    ks = np.repeat(np.arange(g.n_x), 8)
    want = g.values[0, rows, ks][:, [0, 6, 9]]
    err = np.abs(got[:n_k][:, [0, 1, 3]] - want)
    assert np.all(err <= 1e-13 * (np.abs(want) + 1e-3))


def test_maximum_pid_count(nnpdf):
    """64 requested pids (the limit; repeats allowed): 128 KB of staged rows
    per CTA, above the default shared-memory limit; every column equals the
    same pid's column of a 13-pid call bit for bit."""
    g, pdf, o = nnpdf
    x, q2, _ = synth.queries_nnpdf(20_001, seed=35)
    X, Q = cuda(x), cuda(q2)
    pids = np.array([g.pids[k % g.n_flav] for k in range(64)], dtype=np.int32)
    wide = pdf.xfxQ2(pids, X, Q).cpu().numpy()
    base = pdf.xfxQ2(g.pids, X, Q).cpu().numpy()
    assert np.array_equal(wide, base[:, [k % g.n_flav for k in range(64)]])
    parity.check(wide[:3000], o.xfxq2_batch(pids, x[:3000], q2[:3000]), o.kappa(pids, x[:3000], q2[:3000]),
                 what="64 pids")


def test_empty_and_tiny_batches(small):
    g, pdf, o = small
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    assert pdf.xfxQ2(g.pids, e, e).shape == (0, g.n_flav)
    assert pdf.alphasQ2(e).shape == (0,)
    assert pdf.xfxQ2_pw(torch.empty(0, dtype=torch.int32, device="cuda"), e, e).shape == (0,)
    for n in (1, 31, 255, 257):
        x, q2 = synth.queries_small(n, seed=n)
        got = pdf.xfxQ2(g.pids, cuda(x), cuda(q2)).cpu().numpy()
        parity.check(got, o.xfxq2_batch(g.pids, x, q2), o.kappa(g.pids, x, q2), what=f"n={n}")


def test_two_subgrid_tiny_grid_everywhere(lib_built):
    """A tiny grid with unequal duplicated rows: exercises the threshold rule."""
    from paper_2012_08221_gb300.pdf import PDF
    g = tiny_two_sub(seed=3, dup_equal=False)
    pdf, o = PDF.from_grid(g), OracleGrid.from_synth(g)
    rng = np.random.default_rng(8)
    x = np.exp(rng.uniform(math.log(1e-7), 0, 50_000))
    q2 = np.exp(rng.uniform(math.log(0.2), math.log(1e4), 50_000))
    x[:6] = g.x_knots[[0, 1, 2, 3, 4, 4]]
    q2[:6] = g.q_knots[[2, 3, 3, 2, 0, 5]] ** 2
    got = pdf.xfxQ2(g.pids, cuda(x), cuda(q2)).cpu().numpy()
    parity.check(got, o.xfxq2_batch(g.pids, x, q2), o.kappa(g.pids, x, q2), what="tiny two-subgrid")


def test_table_log_against_cuda_log(small):
    g, pdf, o = small
    rng = np.random.default_rng(5)
    v = np.concatenate([np.exp(rng.uniform(-700, 700, 200_000)), [5e-324, 1e-310, 2.2250738585072014e-308,
                        1.0, np.nextafter(1.0, 2), np.nextafter(1.0, 0), 1.7976931348623157e308]])
    V = cuda(v)
    got = pdf.debug_log(V).cpu().numpy()
    ref = torch.log(V).cpu().numpy()
    # within 3 units in the last place of CUDA's log, or 1e-18 absolute
    ulp = np.spacing(np.abs(ref))
    assert np.all(np.abs(got - ref) <= 3 * ulp + 1e-18)
    assert got[-4] == 0.0                        # ln 1 is exact


def test_concurrent_streams_and_host_threads(nnpdf):
    """Device calls on two streams at once, and host-buffer calls from two
    host threads at once, on the same grid: the same results as one at a
    time (the forward kernels use no grid-owned scratch; the host-buffer
    path serialises its staging buffers per grid)."""
    import threading
    g, pdf, o = nnpdf
    xa, qa, _ = synth.queries_nnpdf(200_003, seed=51)
    xb, qb, _ = synth.queries_nnpdf(150_001, seed=52)
    ref_a = pdf.xfxQ2(g.pids, cuda(xa), cuda(qa))
    ref_b = pdf.xfxQ2(g.pids, cuda(xb), cuda(qb))
    Xa, Qa, Xb, Qb = cuda(xa), cuda(qa), cuda(xb), cuda(qb)
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with torch.cuda.stream(s1):
        a = pdf.xfxQ2(g.pids, Xa, Qa)
    with torch.cuda.stream(s2):
        b = pdf.xfxQ2(g.pids, Xb, Qb)
    torch.cuda.synchronize()
    assert torch.equal(a, ref_a) and torch.equal(b, ref_b)
    out = {}

    def host_call(key, x, q):
        out[key] = pdf.xfxQ2_host(g.pids, torch.as_tensor(x).pin_memory(), torch.as_tensor(q).pin_memory())

    ts = [threading.Thread(target=host_call, args=("a", xa, qa)),
          threading.Thread(target=host_call, args=("b", xb, qb))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert torch.equal(out["a"], ref_a.cpu()) and torch.equal(out["b"], ref_b.cpu())


def test_cuda_graph_capture_and_replay(nnpdf):
    """The headline step (x*f for 13 pids plus alpha_s) captured once in a
    CUDA graph and replayed on new inputs copied into the captured buffers:
    the same results as direct calls."""
    g, pdf, o = nnpdf
    x, q2, qa = synth.queries_nnpdf(100_003, seed=53)
    X, Q, QA = cuda(x), cuda(q2), cuda(qa)
    OUT = torch.empty((x.size, g.n_flav), dtype=torch.float64, device="cuda")
    AS = torch.empty(x.size, dtype=torch.float64, device="cuda")
    pdf.xfxQ2(g.pids, X, Q, out=OUT)            # first calls outside the capture
    pdf.alphasQ2(QA, out=AS)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        pdf.xfxQ2(g.pids, X, Q, out=OUT)
        pdf.alphasQ2(QA, out=AS)
    for seed in (54, 55):
        x2, q22, qa2 = synth.queries_nnpdf(x.size, seed=seed)
        X.copy_(cuda(x2))
        Q.copy_(cuda(q22))
        QA.copy_(cuda(qa2))
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(OUT, pdf.xfxQ2(g.pids, cuda(x2), cuda(q22)))
        assert torch.equal(AS, pdf.alphasQ2(cuda(qa2)))


def test_small_query_kernel_matches_the_per_point_kernel(nnpdf):
    """Queries of at most 2^18 point-flavour pairs run one thread per pair;
    larger ones one thread per point.  The same points give the same bits
    both ways (the value of a point does not depend on the batch it is in),
    and the small launch matches the oracle, for x*f, x*f(Q) and a shorter
    pid list."""
    g, pdf, o = nnpdf
    x, q2, _ = synth.queries_nnpdf(100_003, seed=17)
    X, Q = cuda(x), cuda(q2)
    big = pdf.xfxQ2(g.pids, X, Q)                        # 100003 x 13 pairs: per point
    for n in (1, 31, 1001, (1 << 18) // g.n_flav):       # per pair
        small = pdf.xfxQ2(g.pids, X[:n].clone(), Q[:n].clone())
        assert torch.equal(torch.nan_to_num(small, nan=7.0), torch.nan_to_num(big[:n], nan=7.0)), n
    n = 1001
    got = pdf.xfxQ2(g.pids, X[:n], Q[:n]).cpu().numpy()
    parity.check(got, o.xfxq2_batch(g.pids, x[:n], q2[:n]), o.kappa(g.pids, x[:n], q2[:n]),
                 what="small query xfxQ2")
    q = torch.sqrt(Q)
    assert torch.equal(pdf.xfxQ(g.pids, X[:n], q[:n]), pdf.xfxQ(g.pids, X, q)[:n])
    three = np.array([21, -1, 2], dtype=np.int32)            # 100003 x 3 > 2^18 pairs
    assert torch.equal(pdf.xfxQ2(three, X[:n], Q[:n]), pdf.xfxQ2(three, X, Q)[:n])


def test_more_than_two_to_the_31_outputs(nnpdf):
    """Offsets past 32 bits: x*f over n points with n*13 > 2^31 outputs, and
    alpha_s over more than 2^31 points.  The inputs tile a seeded base set on
    the device, so every sampled output (spread over the array, around the
    2^31 boundary and at the very end) must match the oracle at its base
    point."""
    g, pdf, o = nnpdf
    base = 1_000_003
    x, q2, _ = synth.queries_nnpdf(base, seed=19)
    reps = 166
    X, Q = cuda(x).repeat(reps), cuda(q2).repeat(reps)
    n = X.numel()
    assert n * g.n_flav > 2 ** 31
    out = pdf.xfxQ2(g.pids, X, Q)
    del X, Q
    rng = np.random.default_rng(23)
    edge = 2 ** 31 // g.n_flav
    idx = np.concatenate([rng.choice(n, 400, replace=False), np.arange(edge - 40, edge + 40),
                          np.arange(n - 200, n)])
    got = out[cuda(idx)].cpu().numpy()
    del out
    b = idx % base
    parity.check(got, o.xfxq2_batch(g.pids, x[b], q2[b]), o.kappa(g.pids, x[b], q2[b]),
                 what="x*f beyond 2^31 outputs")
    reps_a = 2 ** 31 // base + 2
    QA = cuda(q2).repeat(reps_a)
    na = QA.numel()
    assert na > 2 ** 31
    a_s = pdf.alphasQ2(QA)
    del QA
    idx = np.concatenate([rng.choice(na, 400, replace=False), np.arange(2 ** 31 - 40, 2 ** 31 + 40),
                          np.arange(na - 200, na)])
    got = a_s[cuda(idx)].cpu().numpy()
    ref = o.alphas_batch(q2[idx % base])
    parity.check(got, ref, o.alphas_kappa(q2[idx % base]), what="alpha_s beyond 2^31 points")


def test_xf_and_alphas_in_one_launch(nnpdf):
    """xfxQ2_alphasQ2 gives what xfxQ2 and alphasQ2 give on the same arrays,
    bit for bit, and matches the oracle: a ragged 3e5-point query with domain
    errors on x alone (alpha_s stays valid), on Q^2, NaN, and points outside
    the grid; also on a grid with the error option and on a short query."""
    from paper_2012_08221_gb300.pdf import PDF
    g, pdf, o = nnpdf
    x, q2, _ = synth.queries_nnpdf(300_001, seed=61)
    x[:6] = [-1.0, 0.3, np.nan, 2.0, 1e-12, 0.01]
    q2[:6] = [50.0, -4.0, 10.0, 1e3, 1e14, 0.2]
    for p, n in ((pdf, x.size), (PDF.from_grid(g, extrap="error"), x.size), (pdf, 777)):
        X, Q = cuda(x[:n]), cuda(q2[:n])
        out, a_s = p.xfxQ2_alphasQ2(g.pids, X, Q)
        # bit for bit, NaNs included (compared as 64-bit integers)
        assert torch.equal(out.view(torch.int64), p.xfxQ2(g.pids, X, Q).view(torch.int64))
        assert torch.equal(a_s.view(torch.int64), p.alphasQ2(Q).view(torch.int64))
    out, a_s = pdf.xfxQ2_alphasQ2(g.pids, cuda(x), cuda(q2))
    assert pdf.status() == 1
    parity.check(out.cpu().numpy(), o.xfxq2_batch(g.pids, x, q2), o.kappa(g.pids, x, q2), what="combined x*f")
    ra = o.alphas_batch(q2)
    assert not np.isnan(ra[0]) and np.isnan(ra[1])
    parity.check(a_s.cpu().numpy(), ra, o.alphas_kappa(q2), what="combined alpha_s")
