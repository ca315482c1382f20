"""The FP64 roofline's measured denominators on the GPU: the DFMA-chain peak,
the FP64 tensor instruction (mma.sync f64) of each shape, and DFMA and DMMA
issued together.  These calls compute nothing of the interpolation; the test
checks that they run, return plausible rates, and that the measured fact the
kernels' design rests on holds on this part: the two instruction kinds share
one FP64 pipe, so a mix of them is no faster than the FMA pipe alone."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_fp64_probes():
    from paper_2012_08221_gb300.pdf import MMA_SHAPES, fp64_mixed, fp64_mma_peak, fp64_peak

    dfma = fp64_peak()
    assert 1e11 < dfma < 1e14
    for shape in MMA_SHAPES:
        r = fp64_mma_peak(shape)
        assert math.isfinite(r) and 1e10 < r < 1e14, (shape, r)
    mix = fp64_mixed()
    assert all(math.isfinite(v) and v > 0 for v in mix.values()), mix
    # One shared pipe: the interleaved kernel runs at about the harmonic
    # combination of the two rates, far below their sum.
    assert mix["mixed"] < 0.75 * (mix["dfma"] + mix["dmma"]), mix
    print({k: round(v / 1e12, 3) for k, v in mix.items()}, "TFLOP/s")
