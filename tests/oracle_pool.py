"""The oracle spread over the host cores, for full-size parity checks.

Where the oracle sums over many points in one serial loop (the VEGAS sums),
the points are split into chunks that spawned worker processes evaluate;
the partial sums are added in chunk order.  Spawned, not forked: the parent
already holds a CUDA context, which a forked child must not inherit."""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def _oracle(grid_factory, kwargs=None):
    from oracle.oracle import OracleGrid
    from paper_2012_08221_gb300 import synth
    return OracleGrid.from_synth(getattr(synth, grid_factory)(**(kwargs or {})))


def _vegas_chunk(args):
    grid_factory, member, ln_tau_min, ln_s, edges, v = args
    from oracle.oracle import vegas_sums
    return vegas_sums(_oracle(grid_factory), member, ln_tau_min, ln_s, edges, v)


def _dgrid_chunk(args):
    grid_factory, kwargs, pid, x, q2, w, absval = args
    return _oracle(grid_factory, kwargs).dgrid_pw(pid, x, q2, w, absval=absval)


def _dgrid_matrix_chunk(args):
    grid_factory, kwargs, pids, x, q2, gout, absval = args
    return _oracle(grid_factory, kwargs).dgrid(pids, x, q2, gout, absval=absval)


def workers(limit: int = 16) -> int:
    return max(1, min(limit, len(os.sched_getaffinity(0))))


def vegas_sums_parallel(grid_factory: str, member: int, ln_tau_min: float, ln_s: float,
                        edges: np.ndarray, v: np.ndarray, n_workers: int | None = None) -> np.ndarray:
    """``vegas_sums`` of the grid ``synth.<grid_factory>()`` over all of
    ``v``, chunked over ``n_workers`` processes."""
    n_workers = n_workers or workers()
    chunks = np.array_split(np.ascontiguousarray(v), n_workers)
    jobs = [(grid_factory, member, ln_tau_min, ln_s, edges, c) for c in chunks]
    with mp.get_context("spawn").Pool(n_workers) as pool:
        parts = pool.map(_vegas_chunk, jobs)
    return np.sum(np.stack(parts), axis=0)


def dgrid_pw_parallel(grid_factory: str, kwargs: dict, pid, x, q2, w, absval: bool = False,
                      n_workers: int | None = None) -> np.ndarray:
    """The oracle's grid gradient of L = sum_i w_i xf_{pid_i}(x_i, Q^2_i)
    over all points, chunked over ``n_workers`` processes (member 0 of
    ``synth.<grid_factory>(**kwargs)``); with ``absval`` the sums of |terms|."""
    n_workers = n_workers or workers()
    parts = np.array_split(np.arange(len(x)), n_workers)
    jobs = [(grid_factory, kwargs, pid[p], x[p], q2[p], w[p], absval) for p in parts]
    with mp.get_context("spawn").Pool(n_workers) as pool:
        grads = pool.map(_dgrid_chunk, jobs)
    return np.sum(np.stack(grads), axis=0)


def dgrid_parallel(grid_factory: str, kwargs: dict, pids, x, q2, gout, absval: bool = False,
                   n_workers: int | None = None) -> np.ndarray:
    """The oracle's grid gradient of L = sum_i sum_a gout[i][a] xf_{pids[a]}(x_i, Q^2_i)
    (the matrix form) over all points, chunked over ``n_workers`` processes
    (member 0 of ``synth.<grid_factory>(**kwargs)``); with ``absval`` the sums
    of |terms|."""
    n_workers = n_workers or workers()
    parts = np.array_split(np.arange(len(x)), n_workers)
    jobs = [(grid_factory, kwargs, pids, x[p], q2[p], gout[p], absval) for p in parts]
    with mp.get_context("spawn").Pool(n_workers) as pool:
        grads = pool.map(_dgrid_matrix_chunk, jobs)
    return np.sum(np.stack(grads), axis=0)
