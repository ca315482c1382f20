"""GPU VEGAS integration of the luminosity against the oracle: one
iteration's sums on the same uniforms and grid edges, the host refinement,
several adapting iterations in lock step, and the closed form on a constant
grid."""
import math

import numpy as np
import pytest

from oracle.oracle import OracleGrid, vegas_refine, vegas_sums
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
