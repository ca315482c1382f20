"""Exact-rational brute force of the interpolation definition, for tiny grids.

TEST INFRASTRUCTURE ONLY (pins the FP64 oracle; never called by the library).

It evaluates the same definition as ``pdf_oracle.c`` (PDFFlow Sec. 2.1 and
Sec. 4: LHAPDF-style log-bicubic interpolation with Q subgrids), but by a
different route and in exact arithmetic (``fractions.Fraction``), so that a
slip in the oracle's Hermite basis, derivative rule, indexing or subgrid
handling shows up as a mismatch:

* knot derivatives are computed for *every* knot of a row or subgrid first
  (one-sided secant at the two ends, mean of the adjacent secants inside);
* the cubic on an interval is found by solving the 4x4 linear system
  p(z_k) = g_k, p(z_{k+1}) = g_{k+1}, p'(z_k) = D_k, p'(z_{k+1}) = D_{k+1}
  by exact Gaussian elimination, not by the Hermite basis functions;
* all rows of the chosen subgrid are interpolated in u before the w step;
* outside the grid: linear continuation from the two edge knots, in u from
  the edge columns (each interpolated in w), in w from the edge rows of the
  lowest or highest subgrid.

Inputs are log coordinates: knot logs U (x) and W (Q^2, per subgrid), the
query (u, w), all as exact rationals of the given floats.
"""
from __future__ import annotations

from fractions import Fraction as Fr


def _fr(v):
    return v if isinstance(v, Fr) else Fr(v)


def knot_derivatives(z, g):
    n = len(z)
    out = []
    for k in range(n):
        if k == 0:
            out.append((g[1] - g[0]) / (z[1] - z[0]))
        elif k == n - 1:
            out.append((g[n - 1] - g[n - 2]) / (z[n - 1] - z[n - 2]))
        else:
            left = (g[k] - g[k - 1]) / (z[k] - z[k - 1])
            right = (g[k + 1] - g[k]) / (z[k + 1] - z[k])
            out.append((left + right) / 2)
    return out


def _solve4(A, b):
    """Exact Gaussian elimination with row pivoting on nonzero entries."""
    M = [row[:] + [bb] for row, bb in zip(A, b)]
    n = 4
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [a - f * bb for a, bb in zip(M[r], M[c])]
    return [M[r][n] / M[r][r] for r in range(n)]


def cubic_on_interval(z0, z1, g0, g1, d0, d1):
    """Coefficients (a, b, c, d) of p(s) = a + b s + c s^2 + d s^3, s = z - z0."""
    h = z1 - z0
    A = [[Fr(1), Fr(0), Fr(0), Fr(0)],
         [Fr(1), h, h * h, h * h * h],
         [Fr(0), Fr(1), Fr(0), Fr(0)],
         [Fr(0), Fr(1), 2 * h, 3 * h * h]]
    return _solve4(A, [g0, g1, d0, d1])


def _cubic_eval(c, s):
    v = c[0] + c[1] * s + c[2] * s * s + c[3] * s * s * s
    dv = c[1] + 2 * c[2] * s + 3 * c[3] * s * s
    return v, dv


def _interval(z, v):
    k = 0
    for j in range(len(z)):
        if z[j] <= v:
            k = j
    return min(k, len(z) - 2)


def interp_1d(z, g, v):
    """Piecewise cubic through (z, g) with finite-difference knot derivatives,
    evaluated at v inside [z_0, z_last].  Returns (value, d/dv)."""
    D = knot_derivatives(z, g)
    k = _interval(z, v)
    c = cubic_on_interval(z[k], z[k + 1], g[k], g[k + 1], D[k], D[k + 1])
    return _cubic_eval(c, v - z[k])


def linear_1d(z0, z1, g0, g1, v):
    slope = (g1 - g0) / (z1 - z0)
    return g0 + (v - z0) * slope, slope


def line_1d(z, g, v):
    """Straight line between the two knots of the interval containing v."""
    k = _interval(z, v)
    return linear_1d(z[k], z[k + 1], g[k], g[k + 1], v)


class ExactGrid:
    """values[s][j][k]: subgrid s, local Q row j, x knot k (one flavour).

    interp: 0 cubic on both axes, 1 straight lines on both axes, 2 cubic but
    straight lines on an axis or subgrid with fewer than 4 knots.
    extrap: 0 linear continuation, 1 frozen at the edge (u, w clamped)."""

    def __init__(self, U, W_sub, values_sub, interp=0, extrap=0):
        self.U = [_fr(v) for v in U]
        self.W = [[_fr(v) for v in Ws] for Ws in W_sub]
        self.V = [[[_fr(v) for v in row] for row in sub] for sub in values_sub]
        self.interp, self.extrap = interp, extrap

    def _lin(self, n):
        return self.interp == 1 or (self.interp == 2 and n < 4)

    def _row_u(self, s, j, u, column=None):
        row = self.V[s][j]
        if column is not None:
            return row[column], Fr(0)
        if self._lin(len(self.U)):
            return line_1d(self.U, row, u)
        return interp_1d(self.U, row, u)

    def _w_step(self, u, w, column=None):
        W = self.W
        lo, hi = W[0][0], W[-1][-1]
        if w < lo or w > hi:
            s = 0 if w < lo else len(W) - 1
            j0 = 0 if w < lo else len(W[s]) - 2
            (b0, du0), (b1, du1) = self._row_u(s, j0, u, column), self._row_u(s, j0 + 1, u, column)
            v, dw = linear_1d(W[s][j0], W[s][j0 + 1], b0, b1, w)
            t = (w - W[s][j0]) / (W[s][j0 + 1] - W[s][j0])
            return v, du0 + t * (du1 - du0), dw
        s = 0
        for j in range(len(W)):
            if W[j][0] <= w:
                s = j
        rows = [self._row_u(s, j, u, column) for j in range(len(W[s]))]
        R = [r[0] for r in rows]
        dR = [r[1] for r in rows]
        one_d = line_1d if self._lin(len(W[s])) else interp_1d
        v, dw = one_d(W[s], R, w)
        du, _ = one_d(W[s], dR, w)
        return v, du, dw

    def eval(self, u, w):
        """Exact (value, d/du, d/dw) at log coordinates (u, w)."""
        u, w = _fr(u), _fr(w)
        U = self.U
        if self.extrap == 1:
            lo, hi = self.W[0][0], self.W[-1][-1]
            cu, cw = min(max(u, U[0]), U[-1]), min(max(w, lo), hi)
            v, du, dw = self._eval_in(cu, cw)
            return v, (du if cu == u else Fr(0)), (dw if cw == w else Fr(0))
        return self._eval_in(u, w)

    def _eval_in(self, u, w):
        U = self.U
        if u < U[0] or u > U[-1]:
            k0 = 0 if u < U[0] else len(U) - 2
            a0, _, dw0 = self._w_step(u, w, column=k0)
            a1, _, dw1 = self._w_step(u, w, column=k0 + 1)
            v, du = linear_1d(U[k0], U[k0 + 1], a0, a1, u)
            t = (u - U[k0]) / (U[k0 + 1] - U[k0])
            return v, du, dw0 + t * (dw1 - dw0)
        return self._w_step(u, w)


def exact_alphas(W_sub, alphas_sub, w):
    """alpha_s at w: subgrid cubic with finite-difference derivatives inside,
    linear continuation from the edge knots outside."""
    w = _fr(w)
    W = [[_fr(v) for v in Ws] for Ws in W_sub]
    A = [[_fr(v) for v in As] for As in alphas_sub]
    if w < W[0][0]:
        return linear_1d(W[0][0], W[0][1], A[0][0], A[0][1], w)[0]
    if w > W[-1][-1]:
        return linear_1d(W[-1][-2], W[-1][-1], A[-1][-2], A[-1][-1], w)[0]
    s = 0
    for j in range(len(W)):
        if W[j][0] <= w:
            s = j
    return interp_1d(W[s], A[s], w)[0]
