"""LHAPDF lhagrid1 reader (CPU: the reader makes no GPU call): a grid written
as a set reads back bit for bit; malformed sets are refused."""
import os

import numpy as np
import pytest

from paper_2012_08221_gb300 import _lib, build, lhapdf, synth


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def test_round_trip_multi_subgrid_set(tmp_path):
    g = synth.grid_nnpdf(seeds=(1002, 1005, 1006))
    d = tmp_path / "SYNTH_NNPDF"
    lhapdf.write_set(str(d), g)
    r = lhapdf.read_set(str(d), 0, 3)
    assert np.array_equal(r.x_knots, g.x_knots)
    assert np.array_equal(r.n_q, g.n_q)
    assert np.array_equal(r.q_knots, g.q_knots)
    assert list(r.pids) == [21 if p == 0 else p for p in g.pids]
    assert np.array_equal(r.values, g.values)
    assert np.array_equal(r.alphas, g.alphas)
    one = lhapdf.read_set(str(d), 2, 1)
    assert np.array_equal(one.values[0], g.values[2])


def test_refuses_malformed_sets(tmp_path):
    g = synth.grid_small()
    d = tmp_path / "S"
    lhapdf.write_set(str(d), g)
    with pytest.raises(_lib.PdfError, match="PDF_E_RANGE"):
        lhapdf.read_set(str(d), 0, 2)                       # NumMembers is 1
    with pytest.raises(_lib.PdfError, match="PDF_E_ARG"):
        lhapdf.read_set(str(tmp_path / "missing"), 0, 1)
    dat = d / "S_0000.dat"
    text = dat.read_text().splitlines()
    bad = text[:]
    bad[5] = bad[5] + " 1.0"                                # one value too many
    dat.write_text("\n".join(bad) + "\n")
    with pytest.raises(_lib.PdfError, match="bad value line"):
        lhapdf.read_set(str(d), 0, 1)
    bad = [t.replace("lhagrid1", "lhagrid9") for t in text]
    dat.write_text("\n".join(bad) + "\n")
    with pytest.raises(_lib.PdfError, match="not an lhagrid1"):
        lhapdf.read_set(str(d), 0, 1)


def test_alpha_s_only_when_on_the_grid_knots(tmp_path):
    g = synth.grid_small()
    d = tmp_path / "A"
    lhapdf.write_set(str(d), g)
    info = (d / "A.info").read_text().replace("AlphaS_Qs: [", "AlphaS_Qs: [0.5, ")
    info = info.replace("AlphaS_Vals: [", "AlphaS_Vals: [0.6, ")
    (d / "A.info").write_text(info)
    assert lhapdf.read_set(str(d)).alphas is None


@pytest.mark.parametrize("seed", range(12))
def test_round_trip_random_grids(tmp_path, seed):
    """Randomly shaped grids (2 to 30 x knots, x_max = 1 or below, 1 to 4
    subgrids of 2 to 9 knots, random pids, 1 to 3 members) written as sets
    read back bit for bit, member by member and all at once."""
    from tests.tinygrids import random_grid
    g, _ = random_grid(7200 + seed)
    d = tmp_path / f"RAND{seed}"
    lhapdf.write_set(str(d), g)
    m = g.values.shape[0]
    r = lhapdf.read_set(str(d), 0, m)
    assert np.array_equal(r.x_knots, g.x_knots) and np.array_equal(r.n_q, g.n_q)
    assert np.array_equal(r.q_knots, g.q_knots)
    assert list(r.pids) == [21 if p == 0 else int(p) for p in g.pids]
    assert np.array_equal(r.values, g.values) and np.array_equal(r.alphas, g.alphas)
    for k in range(m):
        assert np.array_equal(lhapdf.read_set(str(d), k, 1).values[0], g.values[k])
