"""A set written in LHAPDF format and loaded through the native reader gives
the same results on the GPU as the same grid loaded from arrays, and matches
the oracle (pid 21 in the files is the gluon)."""
import numpy as np
import pytest

from oracle.oracle import OracleGrid
from paper_2012_08221_gb300 import lhapdf, synth
from tests import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_lhapdf_set_equals_array_grid(tmp_path):
    from paper_2012_08221_gb300 import build
    from paper_2012_08221_gb300.pdf import PDF
    build.build()
    g = synth.grid_nnpdf(seeds=(1002, 1005))
    d = tmp_path / "SYNTH"
    lhapdf.write_set(str(d), g)
    a = PDF.from_grid(g)
    b = lhapdf.load(str(d), 0, 2)
    x, q2, q2a = synth.queries_nnpdf(50_000, seed=9)
    X = torch.as_tensor(x, device="cuda")
    Q = torch.as_tensor(q2, device="cuda")
    pids = np.array([-5, 21, 0, 2], dtype=np.int32)
    for m in (0, 1):
        ra = a.xfxQ2(pids, X, Q, member=m)
        rb = b.xfxQ2(pids, X, Q, member=m)
        assert torch.equal(ra, rb)
    assert torch.equal(a.alphasQ2(Q), b.alphasQ2(Q))
    o = OracleGrid.from_synth(g)
    got = b.xfxQ2(pids, X, Q, member=1).cpu().numpy()
    parity.check(got, o.xfxq2_batch(pids, x, q2, member=1), o.kappa(pids, x, q2, member=1),
                 what="lhapdf member 1")


def test_mkpdf_by_set_name(tmp_path):
    """mkPDF("<set>/<member>", dirname) loads that member of a set on disk:
    the same results as the array grid's member (as the paper's mkPDF)."""
    from paper_2012_08221_gb300 import build
    from paper_2012_08221_gb300.pdf import PDF, mkPDF
    build.build()
    g = synth.grid_nnpdf(seeds=(1002, 1005))
    lhapdf.write_set(str(tmp_path / "SYNTH"), g)
    a = PDF.from_grid(g)
    x, q2, _ = synth.queries_nnpdf(20_000, seed=10)
    X = torch.as_tensor(x, device="cuda")
    Q = torch.as_tensor(q2, device="cuda")
    pids = np.array([-1, 21, 1], dtype=np.int32)
    for name, m in (("SYNTH/1", 1), ("SYNTH", 0)):
        p = mkPDF(name, dirname=str(tmp_path))
        assert torch.equal(p.py_xfxQ2(pids, X, Q), a.xfxQ2(pids, X, Q, member=m))
        assert torch.equal(p.py_alphasQ2(Q), a.alphasQ2(Q))
