"""Seeded synthetic PDF grids and query batches.

This module only *generates inputs*: knot layouts, knot values from a smooth
parametric x*f(x, Q^2), alpha_s knot values from one-loop running, and the
query points of each workload.  It contains none of the interpolation
arithmetic; both the CUDA path and the CPU oracle receive the arrays it makes.

The workloads stand in for the real NNPDF/LHAPDF sets and Monte Carlo phase
space of the paper (Sec. 2.2 benchmarks, Sec. 3 examples), which are not
available here.  Shapes follow an NNPDF-like grid: log-spaced x knots down to
1e-9, Q knots split into subgrids at the charm, bottom and top thresholds.

Random numbers: numpy ``Generator(PCG64(seed))``.  Grid parameters use seed
``1000 + workload`` (replica k of set j: seed ``[1000 + workload, j, k]``),
queries use ``2000 + workload``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

Q0 = 1.65            # reference scale of the parametric knot values (GeV)
MZ = 91.19           # alpha_s anchor scale (GeV)
ALPHAS_MZ = 0.118
THRESHOLDS = (1.51, 4.92, 172.5)   # charm, bottom, top (GeV)
SQRT_S = 13000.0     # LHC Run-2 energy for the Monte Carlo workload (GeV)


@dataclass
class Grid:
    """One PDF set in memory: knots, subgrid split, flavours and values.

    ``q_knots`` lists Q (GeV) subgrid by subgrid; the last knot of subgrid s
    equals the first knot of subgrid s+1 (the threshold is duplicated), so
    the number of Q rows is ``sum(n_q)``.  ``values`` is
    ``[n_members][rows][n_x][n_flav]`` of x*f; ``alphas`` is ``[rows]``.
    """
    x_knots: np.ndarray
    n_q: np.ndarray
    q_knots: np.ndarray
    pids: np.ndarray
    values: np.ndarray
    alphas: np.ndarray | None
    name: str = ""
    params: dict = field(default_factory=dict)

    @property
    def n_x(self) -> int:
        return int(self.x_knots.size)

    @property
    def n_flav(self) -> int:
        return int(self.pids.size)

    @property
    def n_members(self) -> int:
        return int(self.values.shape[0])

    @property
    def n_rows(self) -> int:
        return int(self.q_knots.size)

    def member(self, k: int) -> "Grid":
        return Grid(self.x_knots, self.n_q, self.q_knots, self.pids,
                    self.values[k:k + 1].copy(), self.alphas, f"{self.name}/{k}")


def log_knots(lo: float, hi: float, n: int) -> np.ndarray:
    """n knots log-spaced over [lo, hi], endpoints exactly lo and hi."""
    k = np.exp(np.linspace(math.log(lo), math.log(hi), n))
    k[0], k[-1] = lo, hi
    return k


def subgrid_knots(edges, counts) -> tuple[np.ndarray, np.ndarray]:
    """Concatenate log-spaced subgrids [edges[s], edges[s+1]] with counts[s]
    knots each; shared edges appear in both neighbours (duplicated rows)."""
    parts = [log_knots(edges[s], edges[s + 1], counts[s]) for s in range(len(counts))]
    return np.concatenate(parts), np.asarray(counts, dtype=np.int32)


def flavour_params(rng: np.random.Generator, n_flav: int) -> np.ndarray:
    """(A, alpha, beta, c) per flavour, drawn in ascending pid order."""
    out = np.empty((n_flav, 4))
    for a in range(n_flav):
        out[a, 0] = rng.uniform(0.1, 2.0)
        out[a, 1] = rng.uniform(-0.3, 0.8)
        out[a, 2] = rng.uniform(2.0, 6.0)
        out[a, 3] = rng.uniform(-0.1, 0.1)
    return out


def parametric_values(x_knots, q_knots, params) -> np.ndarray:
    """x*f = A x^alpha (1-x)^beta (1 + c ln(Q^2/Q0^2)) on every knot.

    Returns ``[rows][n_x][n_flav]``.  Values cross zero where
    1 + c ln(Q^2/Q0^2) < 0 and vanish at x = 1."""
    x = x_knots[None, :, None]
    lq = np.log(q_knots * q_knots / (Q0 * Q0))[:, None, None]
    A, al, be, c = (params[:, i][None, None, :] for i in range(4))
    return A * x ** al * (1.0 - x) ** be * (1.0 + c * lq)


def b0(nf: int) -> float:
    return (33.0 - 2.0 * nf) / (12.0 * math.pi)


def alphas_one_loop(q: np.ndarray, nf_fixed: int | None = None) -> np.ndarray:
    """One-loop alpha_s(Q) anchored at alpha_s(MZ) = 0.118.

    1/alpha_s is continuous and piecewise linear in ln Q^2 with slope b0(nf);
    nf = 3, 4, 5, 6 below 1.51, 4.92, 172.5 GeV and above (or ``nf_fixed``)."""
    q = np.asarray(q, dtype=np.float64)
    lz = math.log(MZ * MZ)
    if nf_fixed is not None:
        inv = 1.0 / ALPHAS_MZ + b0(nf_fixed) * (np.log(q * q) - lz)
        return 1.0 / inv
    t = [math.log(th * th) for th in THRESHOLDS]
    out = np.empty_like(q)
    for i, qi in enumerate(q.ravel()):
        L = math.log(qi * qi)
        inv = 1.0 / ALPHAS_MZ
        # integrate b0(nf(l)) dl from lz to L across the threshold segments
        lo, hi, sign = (lz, L, 1.0) if L >= lz else (L, lz, -1.0)
        bounds = [-math.inf] + t + [math.inf]
        acc = 0.0
        for j in range(4):
            a, b = max(lo, bounds[j]), min(hi, bounds[j + 1])
            if b > a:
                acc += b0(3 + j) * (b - a)
        out.ravel()[i] = inv + sign * acc
    return 1.0 / out


def _grid(name, x_knots, q_knots, n_q, pids, seeds, nf_fixed=None) -> Grid:
    vals = []
    plist = []
    for s in seeds:
        rng = np.random.default_rng(s)
        p = flavour_params(rng, len(pids))
        plist.append(p)
        vals.append(parametric_values(x_knots, q_knots, p))
    return Grid(np.ascontiguousarray(x_knots, dtype=np.float64),
                np.ascontiguousarray(n_q, dtype=np.int32),
                np.ascontiguousarray(q_knots, dtype=np.float64),
                np.ascontiguousarray(pids, dtype=np.int32),
                np.ascontiguousarray(np.stack(vals)),
                alphas_one_loop(q_knots, nf_fixed), name,
                {"flavour_params": np.stack(plist)})


PIDS_11 = np.arange(-5, 6, dtype=np.int32)
PIDS_13 = np.arange(-6, 7, dtype=np.int32)


def grid_small(seed: int = 1001, pids=PIDS_11) -> Grid:
    """Single-member grid: 50 x knots in [1e-7, 1], one subgrid of 20 Q knots
    in [1.65, 1e4] GeV, one-loop alpha_s with nf = 5."""
    xk = log_knots(1e-7, 1.0, 50)
    qk, nq = subgrid_knots([1.65, 1e4], [20])
    return _grid("small-50x20", xk, qk, nq, pids, [seed], nf_fixed=5)


def grid_nnpdf(seeds=(1002,)) -> Grid:
    """NNPDF-shaped grid: 196 x knots in [1e-9, 1]; Q subgrids
    [1.0, 1.51] 8, [1.51, 4.92] 12, [4.92, 172.5] 20, [172.5, 1e5] 10 knots;
    13 flavours; one member per seed."""
    xk = log_knots(1e-9, 1.0, 196)
    qk, nq = subgrid_knots([1.0, 1.51, 4.92, 172.5, 1e5], [8, 12, 20, 10])
    return _grid("nnpdf-196x50", xk, qk, nq, PIDS_13, list(seeds))


def grid_set_a(n_rep: int = 101) -> Grid:
    xk = log_knots(1e-7, 1.0, 50)
    qk, nq = subgrid_knots([1.65, 1e4], [20])
    return _grid("setA-50x20", xk, qk, nq, PIDS_11,
                 [[1004, 0, k] for k in range(n_rep)], nf_fixed=5)


def grid_set_b() -> Grid:
    xk = log_knots(1e-8, 1.0, 100)
    qk, nq = subgrid_knots([1.65, 4.92, 172.5, 1e5], [10, 10, 10])
    return _grid("setB-100x30", xk, qk, nq, PIDS_11, [[1004, 1, 0]])


def grid_set_c(n_rep: int = 50) -> Grid:
    xk = log_knots(1e-9, 1.0, 150)
    qk, nq = subgrid_knots([1.0, 1.51, 4.92, 172.5, 1e5], [8, 10, 15, 12])
    return _grid("setC-150x45", xk, qk, nq, PIDS_13,
                 [[1004, 2, k] for k in range(n_rep)])


# ---------------------------------------------------------------- queries

def _loguniform(rng, lo, hi, n):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), n))


def queries_small(n: int = 100_000, seed: int = 2001):
    """x log-uniform in [1e-6, 0.9], Q^2 log-uniform in [4, 2.5e7] GeV^2.
    The same Q^2 serve the alpha_s queries."""
    rng = np.random.default_rng(seed)
    x = _loguniform(rng, 1e-6, 0.9, n)
    q2 = _loguniform(rng, 4.0, 2.5e7, n)
    return x, q2


def queries_nnpdf(n: int = 10_000_000, seed: int = 2002):
    """x log-uniform in [1e-8, 1), Q^2 log-uniform in [1, 1e10] GeV^2,
    plus an independent set of alpha_s Q^2 drawn the same way."""
    rng = np.random.default_rng(seed)
    x = np.exp(rng.uniform(math.log(1e-8), 0.0, n))
    x = np.minimum(x, np.nextafter(1.0, 0.0))
    q2 = np.exp(rng.uniform(0.0, math.log(1e10), n))
    q2a = np.exp(rng.uniform(0.0, math.log(1e10), n))
    return x, q2, q2a


def queries_pointwise(n: int = 10_000_000, seed: int = 2003, pids=PIDS_13):
    """Pointwise queries on the small grid: one pid per point, uniform over
    the flavours, and a N(0,1) weight per point for L = sum w_i xf_i."""
    rng = np.random.default_rng(seed)
    x = _loguniform(rng, 1e-6, 0.9, n)
    q2 = _loguniform(rng, 4.0, 2.5e7, n)
    pid = rng.choice(np.asarray(pids, dtype=np.int32), size=n).astype(np.int32)
    w = rng.standard_normal(n)
    return pid, x, q2, w


@dataclass
class Batch:
    set_index: int
    member: int
    pids: np.ndarray
    x: np.ndarray
    q2: np.ndarray


def batches_uneven(grids, n_batches: int = 400, seed: int = 2004,
                   nmin: float = 1e3, nmax: float = 1e6, scale: float = 1.0):
    """Request batches for the batched workload: size log-uniform in
    [nmin, nmax] (times ``scale``), a uniformly drawn set and member, and a
    flavour subset of 1, 2 or 3 pids.  Points are log-uniform inside the
    chosen grid's x and Q^2 range."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_batches):
        s = int(rng.integers(0, len(grids)))
        g = grids[s]
        m = int(rng.integers(0, g.n_members))
        k = int(rng.integers(1, 4))
        pids = np.sort(rng.choice(g.pids, size=k, replace=False)).astype(np.int32)
        n = max(1, int(round(scale * math.exp(rng.uniform(math.log(nmin), math.log(nmax))))))
        x = np.exp(rng.uniform(math.log(g.x_knots[0]), math.log(g.x_knots[-1]), n))
        qlo, qhi = g.q_knots[0] ** 2, g.q_knots[-1] ** 2
        q2 = np.exp(rng.uniform(math.log(qlo), math.log(qhi), n))
        out.append(Batch(s, m, pids, x, q2))
    return out


@dataclass
class Events:
    """Hadron-collider events in log variables.

    ln tau ~ U[ln 1e-6, 0]; y uniform within |y| <= -ln(tau)/2, so that
    ln x1 = ln(tau)/2 + y and ln x2 = ln(tau)/2 - y never exceed 0, and
    ln Q^2 = ln tau + ln s.  ``flags`` marks the injected low tail:
    bit 0 -> ln Q^2 replaced by ``ln_mu2`` (mu_F^2 log-uniform in
    [0.04, 1) GeV^2), bit 1 -> ln x1 replaced by ``ln_x1`` (x1 log-uniform in
    [1e-11, 1e-9))."""
    ln_tau: np.ndarray
    y: np.ndarray
    flags: np.ndarray
    ln_mu2: np.ndarray
    ln_x1: np.ndarray
    ln_s: float


def events_lhc(n: int, seed: int = 2005, tail: float = 0.05) -> Events:
    rng = np.random.default_rng(seed)
    ln_tau = rng.uniform(math.log(1e-6), 0.0, n)
    half = -0.5 * ln_tau
    y = (2.0 * rng.uniform(0.0, 1.0, n) - 1.0) * half
    r_tail = rng.uniform(0.0, 1.0, n)
    r_half = rng.uniform(0.0, 1.0, n)
    ln_mu2 = rng.uniform(math.log(0.04), 0.0, n)
    ln_x1 = rng.uniform(math.log(1e-11), math.log(1e-9), n)
    flags = np.zeros(n, dtype=np.uint8)
    t = r_tail < tail
    flags[t] |= 1
    flags[t & (r_half < 0.5)] |= 2
    return Events(ln_tau, y, flags, ln_mu2, ln_x1, 2.0 * math.log(SQRT_S))


def paper_usage_example():
    """The query of the paper's usage example (Fig. 1): pids -1, 21, 1;
    x = 1e-6 .. 1e-2 and Q = 10 .. 1e5 GeV, five points."""
    pids = np.array([-1, 21, 1], dtype=np.int32)
    x = np.array([10.0 ** i for i in range(-6, -1)])
    q = np.array([10.0 ** i for i in range(1, 6)])
    return pids, x, q
