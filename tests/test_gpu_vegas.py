"""GPU VEGAS integration of the luminosity against the oracle: one
iteration's sums on the same uniforms and grid edges, the host refinement,
several adapting iterations in lock step, and the closed form on a constant
grid."""
import math

import numpy as np
import pytest

from oracle.oracle import OracleGrid, vegas_accumulate, vegas_map, vegas_refine, vegas_sums
from paper_2012_08221_gb300 import synth
from tests.tinygrids import fill

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LN_TAU_MIN = math.log(1e-6)
LN_S = 2 * math.log(13000.0)
SUM_RTOL = 1e-11          # sums of 1e4-1e5 positive terms in different orders


@pytest.fixture(scope="module")
def nn():
    from paper_2012_08221_gb300 import build
    from paper_2012_08221_gb300.pdf import PDF
    build.build()
    g = synth.grid_nnpdf()
    return g, PDF.from_grid(g), OracleGrid.from_synth(g)


def test_iteration_sums_match_the_oracle(nn):
    from paper_2012_08221_gb300.vegas import VegasLumi
    g, pdf, o = nn
    rng = np.random.default_rng(10)
    for trial in range(2):
        vg = VegasLumi(pdf, LN_TAU_MIN, LN_S, n_bins=40)
        if trial:
            for d in range(2):
                vg.edges[d] = np.concatenate([[0.0], np.sort(rng.uniform(0, 1, 39)), [1.0]])
        edges = vg.edges.copy()
        v = rng.uniform(0, 1, (30_011, 2))
        _, _, s = vg.iteration(torch.as_tensor(v, device="cuda"), refine=False)
        ref = vegas_sums(o, 0, LN_TAU_MIN, LN_S, edges, v)
        assert np.all(np.abs(s - ref) <= SUM_RTOL * np.abs(ref) + 1e-300)


def test_adapting_iterations_in_lock_step(nn):
    from paper_2012_08221_gb300.vegas import VegasLumi
    g, pdf, o = nn
    rng = np.random.default_rng(12)
    vg = VegasLumi(pdf, LN_TAU_MIN, LN_S, n_bins=30)
    edges = vg.edges.copy()
    for it in range(4):
        v = rng.uniform(0, 1, (20_000, 2))
        est, err, s = vg.iteration(torch.as_tensor(v, device="cuda"))
        ref = vegas_sums(o, 0, LN_TAU_MIN, LN_S, edges, v)
        assert abs(s[0] - ref[0]) <= 1e-10 * ref[0]
        for d in range(2):
            edges[d] = vegas_refine(ref[2 + 30 * d: 32 + 30 * d], 1.5, edges[d])
        assert np.allclose(vg.edges, edges, rtol=0, atol=1e-10)


def test_constant_grid_integral_closed_form():
    from paper_2012_08221_gb300.pdf import PDF
    from paper_2012_08221_gb300.vegas import VegasLumi
    g = fill(synth.grid_nnpdf(), lambda U, W: 0.75 + 0 * U * W)
    res = VegasLumi(PDF.from_grid(g), LN_TAU_MIN, LN_S).integrate(n_iter=4, n_per_iter=400_000, seed=5)
    exact = LN_TAU_MIN ** 2 * g.n_flav * 0.75 ** 2 / 2
    assert abs(res.integral - exact) < 4 * res.error
    assert res.error < 1e-3 * exact


def test_full_size_iteration_sums(nn):
    """One iteration at the benchmark's size and shape (1e7 points, 50 bins
    per dimension) on adapted edges: every sum against the oracle, which
    runs on the host cores in chunks (partial sums added in chunk order)."""
    from paper_2012_08221_gb300.vegas import VegasLumi
    from tests.oracle_pool import vegas_sums_parallel
    g, pdf, o = nn
    n_bins = 50
    rng = np.random.default_rng(14)
    # adapted edges from one small oracle iteration and the oracle's refinement
    edges = np.tile(np.linspace(0.0, 1.0, n_bins + 1), (2, 1))
    s0 = vegas_sums(o, 0, LN_TAU_MIN, LN_S, edges, rng.uniform(0, 1, (100_000, 2)))
    for d in range(2):
        edges[d] = vegas_refine(s0[2 + n_bins * d: 2 + n_bins * (d + 1)], 1.5, edges[d])
    v = rng.uniform(0, 1, (10_000_000, 2))
    ref = vegas_sums_parallel("grid_nnpdf", 0, LN_TAU_MIN, LN_S, edges, v)
    vg = VegasLumi(pdf, LN_TAU_MIN, LN_S, n_bins=n_bins)
    vg.edges = edges.copy()
    _, _, s = vg.iteration(torch.as_tensor(v, device="cuda"), refine=False)
    # 1e7 positive terms per sum, summed in different orders on the two sides
    assert np.all(np.abs(s - ref) <= 1e-10 * np.abs(ref) + 1e-300), np.max(np.abs(s - ref) / np.abs(ref))
    assert np.all(ref[2:] > 0.0)



# --------------------------------------------- general VEGAS, user integrand

def _random_edges(rng, dim, nb):
    return np.stack([np.concatenate([[0.0], np.sort(rng.uniform(0, 1, nb - 1)), [1.0]]) for _ in range(dim)])


def test_general_map_and_accumulate_match_the_oracle(nn):
    from paper_2012_08221_gb300.vegas import Vegas
    rng = np.random.default_rng(20)
    vg = Vegas(3, n_bins=20)
    vg.edges = _random_edges(rng, 3, 20)
    v = rng.uniform(0, 1, (50_001, 3))
    r, jac, bins = vg.map(torch.as_tensor(v, device="cuda"))
    rr, rj, rb = vegas_map(vg.edges, v)
    assert np.array_equal(bins.cpu().numpy(), rb)
    assert np.allclose(r.cpu().numpy(), rr, rtol=0, atol=1e-15)
    assert np.allclose(jac.cpu().numpy(), rj, rtol=1e-14, atol=0)
    w = rng.standard_normal(v.shape[0]) * np.exp(rng.uniform(-3, 3, v.shape[0]))
    got = vg.accumulate(torch.as_tensor(w, device="cuda"), torch.as_tensor(rb, device="cuda"))
    ref = vegas_accumulate(20, w, rb)
    scale = np.concatenate([[np.abs(w).sum()], ref[1:]])
    assert np.all(np.abs(got - ref) <= 1e-12 * scale)


def test_general_midpoint_lattice_is_exact_on_the_gpu():
    """A multilinear integrand through random edges: the midpoint lattice
    integrates it exactly (the closed form prod_d (a_d + b_d / 2))."""
    from paper_2012_08221_gb300.vegas import Vegas
    rng = np.random.default_rng(21)
    dim, nb = 3, 8
    vg = Vegas(dim, n_bins=nb)
    vg.edges = _random_edges(rng, dim, nb)
    axes = [(np.arange(k) + 0.5) / k for k in (2 * nb, 3 * nb, nb)]
    v = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, dim)
    a = torch.tensor([0.5, 2.0, -1.0], dtype=torch.float64, device="cuda")
    b = torch.tensor([1.5, -0.7, 3.0], dtype=torch.float64, device="cuda")
    est, _, _ = vg.iteration(lambda r: torch.prod(a + b * r, dim=1), torch.as_tensor(v, device="cuda"),
                             refine=False)
    assert abs(est - float(torch.prod(a + b / 2))) <= 1e-12


# A single-top-like leading-order integrand, written as user code (the shape
# of the paper's example: b quark from one proton, light quarks from the
# other, a t-channel W propagator; toy normalisation).  ``xf(pids, x, q2)``
# is the PDF call and ``lib`` the array module, so that the same function
# runs on the GPU (torch, the library's xfxQ2) and on the CPU (numpy, the
# oracle).
MT, MW, SQRT_S = 173.0, 80.4, 13000.0


def single_top_like(r, xf, lib):
    s = SQRT_S ** 2
    ln_tau_min = math.log(MT * MT / s)
    ln_tau = (1.0 - r[:, 0]) * ln_tau_min
    tau = lib.exp(ln_tau)
    y = (2.0 * r[:, 1] - 1.0) * (-0.5 * ln_tau)
    cos_t = 2.0 * r[:, 2] - 1.0
    x1 = lib.exp(0.5 * ln_tau + y)
    x2 = lib.exp(0.5 * ln_tau - y)
    shat = tau * s
    that = -(shat - MT * MT) * (1.0 - cos_t) / 2.0
    me2 = shat * (shat - MT * MT) / (that - MW * MW) ** 2
    q2 = x1 * 0.0 + MT * MT
    fb = xf([5], x1, q2)[:, 0]
    fq = xf([2, 4, -1, -3], x2, q2).sum(1)
    lum = fb * fq / (x1 * x2)
    jac = (-ln_tau_min) * tau * (-ln_tau) * 2.0
    return jac * me2 * lum / (2.0 * shat)


def test_user_integrand_in_lock_step_with_the_oracle(nn):
    """Three adapting iterations of the single-top-like user integrand: the
    GPU path (library map, torch integrand calling xfxQ2, library
    accumulation and refinement) and the oracle path (oracle map, numpy
    integrand calling the oracle, oracle accumulation and refinement) on the
    same uniforms."""
    from paper_2012_08221_gb300.vegas import Vegas
    g, pdf, o = nn
    gpu_xf = lambda pids, x, q2: pdf.xfxQ2(np.array(pids, np.int32), x, q2)
    cpu_xf = lambda pids, x, q2: o.xfxq2_batch(np.array(pids, np.int32), x, q2)
    vg = Vegas(3, n_bins=30)
    edges = vg.edges.copy()
    rng = np.random.default_rng(22)
    for it in range(3):
        v = rng.uniform(0, 1, (40_000, 3))
        shift = vg.shift
        est, err, s = vg.iteration(lambda r: single_top_like(r, gpu_xf, torch), torch.as_tensor(v, device="cuda"))
        r, jac, bins = vegas_map(edges, v)
        ref = vegas_accumulate(30, single_top_like(r, cpu_xf, np) * jac, bins, shift=shift)
        assert np.all(np.abs(s - ref) <= 1e-10 * np.abs(ref)), it
        for d in range(3):
            edges[d] = vegas_refine(ref[2 + 30 * d: 32 + 30 * d], 1.5, edges[d])
        assert np.allclose(vg.edges, edges, rtol=0, atol=1e-10)
        assert 0 < err < 0.1 * est


def test_user_integrand_converges():
    """Adaptation on a peaked separable integrand whose integral is known:
    prod_d 1 / (1 + 50 (r_d - c_d)^2) over [0, 1]^3."""
    from paper_2012_08221_gb300.vegas import Vegas
    c = torch.tensor([0.3, 0.6, 0.8], dtype=torch.float64, device="cuda")
    k = 50.0
    exact = 1.0
    for cd in (0.3, 0.6, 0.8):
        exact *= (math.atan(math.sqrt(k) * (1 - cd)) + math.atan(math.sqrt(k) * cd)) / math.sqrt(k)
    res = Vegas(3, n_bins=40).integrate(lambda r: torch.prod(1.0 / (1.0 + k * (r - c) ** 2), dim=1),
                                        n_iter=5, n_per_iter=200_000, seed=3, warmup=3)
    assert abs(res.integral - exact) < 4 * res.error
    assert res.error < 2e-3 * exact


def test_nearly_flat_integrand_variance_matches_the_oracle():
    """Weights 1 + 1e-7 g(r): the second iteration takes its variance about
    the first estimate, on the GPU and in the oracle alike; the two agree to
    1e-9 and both agree with a two-pass variance of the same weights (about
    0, E[w^2] - E[w]^2 would cancel to the last digits)."""
    from paper_2012_08221_gb300.vegas import Vegas
    rng = np.random.default_rng(23)
    vg = Vegas(2, n_bins=16)                      # uniform edges: every Jacobian is 1
    f_gpu = lambda r: 1.0 + 1e-7 * torch.sin(6.0 * r[:, 0]) * torch.cos(5.0 * r[:, 1])
    n = 1_000_000
    for it in range(2):
        v = rng.uniform(0, 1, (n, 2))
        shift = vg.shift
        est, err, s = vg.iteration(f_gpu, torch.as_tensor(v, device="cuda"), refine=False)
    r, jac, bins = vegas_map(vg.edges, v)
    w = (1.0 + 1e-7 * np.sin(6.0 * r[:, 0]) * np.cos(5.0 * r[:, 1])) * jac
    ref = vegas_accumulate(16, w, bins, shift=shift)
    mean_r = ref[0] / n
    err_r = math.sqrt(max(ref[1] / n - (mean_r - shift) ** 2, 0.0) / (n - 1))
    assert abs(shift) > 0.5                       # the second iteration ran about the first estimate
    assert abs(err - err_r) <= 1e-9 * err_r, (err, err_r)
    two_pass = math.sqrt(math.fsum((w - math.fsum(w) / n) ** 2) / n / (n - 1))
    assert abs(err - two_pass) <= 1e-6 * two_pass, (err, two_pass)
