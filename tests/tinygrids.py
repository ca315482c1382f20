"""Small hand-made grids for the oracle pins and the GPU edge cases."""
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
