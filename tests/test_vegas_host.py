"""The library's host-side VEGAS refinement against the oracle's (CPU)."""
import numpy as np

from oracle.oracle import vegas_refine


def test_refinement_matches_the_oracle():
    from paper_2012_08221_gb300 import build
    build.build()
    import ctypes as C

    from paper_2012_08221_gb300._lib import lib
    rng = np.random.default_rng(11)
    for _ in range(20):
        nb = int(rng.integers(2, 60))
        w2 = rng.exponential(1.0, nb) * rng.uniform(0, 1, nb) ** 3
        old = np.concatenate([[0.0], np.sort(rng.uniform(0, 1, nb - 1)), [1.0]])
        a = old.copy()
        assert lib().pdf_vegas_refine(w2.ctypes.data_as(C.POINTER(C.c_double)), nb, 1.5,
                                      a.ctypes.data_as(C.POINTER(C.c_double))) == 0
        assert np.allclose(a, vegas_refine(w2, 1.5, old), rtol=0, atol=1e-14)
