"""Small hand-made grids for the oracle pins and the GPU edge cases, and
randomly shaped grids for the fuzz tests."""
import math

import numpy as np

from paper_2012_08221_gb300 import synth


def tiny_single(seed=7, n_flav=2):
    """4 x knots (non-uniform in ln x) x one subgrid of 4 Q knots."""
    rng = np.random.default_rng(seed)
    x = np.array([1e-4, 5e-4, 8e-3, 0.3])
    nq = np.array([4], dtype=np.int32)
    q = np.array([1.2, 2.0, 5.5, 30.0])
    pids = np.array([0, 2], dtype=np.int32)[:n_flav]
    v = rng.uniform(-1.0, 2.0, size=(1, 4, 4, n_flav))
    a = rng.uniform(0.1, 0.4, size=4)
    return synth.Grid(x, nq, q, pids, v, a, "tiny4x4")


def tiny_two_sub(seed=11, n_flav=3, dup_equal=True):
    """5 x knots x two Q subgrids (3 + 3 knots, threshold knot duplicated)."""
    rng = np.random.default_rng(seed)
    x = np.array([2e-5, 1e-4, 3e-3, 0.04, 1.0])
    nq = np.array([3, 3], dtype=np.int32)
    q = np.array([1.0, 1.4, 2.3, 2.3, 6.0, 40.0])
    pids = np.array([-1, 0, 1], dtype=np.int32)[:n_flav]
    v = rng.uniform(-1.0, 2.0, size=(1, 6, 5, n_flav))
    if dup_equal:
        v[:, 3] = v[:, 2]
    a = rng.uniform(0.1, 0.4, size=6)
    if dup_equal:
        a[3] = a[2]
    return synth.Grid(x, nq, q, pids, v, a, "tiny5x6")


def fill(grid, fn):
    """Replace every flavour's values by fn(u, w) on the knots (all members)."""
    U = np.log(grid.x_knots)
    W = np.log(grid.q_knots * grid.q_knots)
    vals = fn(U[None, :], W[:, None])
    v = np.broadcast_to(vals[None, :, :, None], grid.values.shape).copy()
    return synth.Grid(grid.x_knots, grid.n_q, grid.q_knots, grid.pids, v, grid.alphas, grid.name)


def _spaced(rng, lo, hi, n):
    """n ascending values from lo to hi whose neighbouring gaps differ by at
    most a factor e^1.6 (non-uniform, as real grids are, but not so uneven
    that the finite-difference slopes become ill-conditioned)."""
    if n == 1:
        return np.array([lo])
    gaps = np.exp(rng.uniform(-0.8, 0.8, n - 1))
    v = lo + (hi - lo) * np.concatenate([[0.0], np.cumsum(gaps) / np.sum(gaps)])
    v[-1] = hi
    return v


def random_grid(seed):
    rng = np.random.default_rng(seed)
    nx = int(rng.integers(2, 31))
    u_hi = 0.0 if rng.random() < 0.6 else float(rng.uniform(-3.0, -0.5))
    x = np.exp(_spaced(rng, float(rng.uniform(-21.0, -8.0)), u_hi, nx))
    if u_hi == 0.0:
        x[-1] = 1.0
    nsub = int(rng.integers(1, 5))
    bounds = np.exp(_spaced(rng, 0.0, float(rng.uniform(3.0, 11.5)), nsub + 1))
    nq = rng.integers(2, 10, nsub).astype(np.int32)
    q = np.concatenate([np.exp(_spaced(rng, math.log(bounds[s]), math.log(bounds[s + 1]), int(nq[s])))
                        for s in range(nsub)])
    F = int(rng.integers(1, 15))
    pids = rng.choice(np.arange(-6, 7), size=min(F, 13), replace=False).astype(np.int32)
    if rng.random() < 0.5 and 0 in pids:
        pids[pids == 0] = 21
    nmem = int(rng.integers(1, 4))
    rows = q.size
    v = rng.uniform(-1.0, 2.0, size=(nmem, rows, nx, pids.size))
    a = rng.uniform(0.1, 0.4, size=rows)
    if rng.random() < 0.5:                     # equal duplicated threshold rows
        r = np.cumsum(nq)[:-1]
        v[:, r] = v[:, r - 1]
        a[r] = a[r - 1]
    return synth.Grid(x, nq, q, pids, v, a, f"fuzz{seed}"), rng
