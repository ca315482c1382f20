"""Parity criterion between the CUDA path and the FP64 oracle.

|gpu - oracle| <= rtol * max(|oracle|, kappa) + atol, where kappa is the sum of
|weight * value| over the stencil (computed by the oracle): the size of the
terms the interpolation adds, so that results near zero by cancellation are
judged on the scale of their terms.  rtol = 1e-12, atol = 1e-15 for values.
"""
import numpy as np

RTOL = 1e-12
ATOL = 1e-15


def check(gpu, ref, kappa, rtol=RTOL, atol=ATOL, what=""):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    kappa = np.broadcast_to(np.asarray(kappa, dtype=np.float64), ref.shape)
    nan_ref = np.isnan(ref)
    assert np.array_equal(np.isnan(gpu), nan_ref), f"{what}: NaN pattern differs"
    g, r, k = gpu[~nan_ref], ref[~nan_ref], kappa[~nan_ref]
    scale = np.maximum(np.abs(r), np.nan_to_num(k))
    err = np.abs(g - r)
    bound = rtol * scale + atol
    bad = err > bound
    if bad.any():
        i = np.argmax(err / bound)
        raise AssertionError(
            f"{what}: {bad.sum()} of {bad.size} outside tolerance; worst gpu={g[i]!r} "
            f"ref={r[i]!r} kappa={k[i]!r} err={err[i]:.3e} bound={bound[i]:.3e}")
    return float(np.max(err / np.maximum(scale, 1e-300))) if err.size else 0.0


def strict_count(gpu, ref, rtol=RTOL, atol=ATOL):
    """Number of outputs that would fail with kappa replaced by |oracle|."""
    gpu = np.asarray(gpu)
    ref = np.asarray(ref)
    m = ~np.isnan(ref)
    return int(np.sum(np.abs(gpu[m] - ref[m]) > rtol * np.abs(ref[m]) + atol))
