// Device helpers shared by the adjoints that accumulate a grid gradient in
// the monomial basis of the interpolation patch (the grid gradients of
// bwd.cu and the luminosity adjoint of lumi.cu): per bin of sorted points a
// half-warp holds G[n][m] = sum over the bin's points of (weight) bq_n bx_m
// and maps it back to the 16 stencil values once per run of the bin; and
// the pointwise bin of a point, which the forward pass also writes into the
// derivative tape.
#pragma once

#include "pdf_common.cuh"

namespace pdfgpu {

// Maps a half-warp's 16 accumulators back to the 16 stencil values of their
// bin.  Lane 4n + m passes G[n][m] in g; lane 4j + i gets
// sum_{n,m} Mq[n][j] G[n][m] Mx[m][i], in two stages through the half-warp's
// 16 shared slots buf: T[j][m] = sum_n Mq[n][j] G[n][m] (lane 4j + m), then
// sum_m T[j][m] Mx[m][i] -- 8 FMAs per lane.
__device__ __forceinline__ double map_back(double g, double *buf, const double *__restrict__ Mq,
                                           const double *__restrict__ Mx, int sn, int sm, unsigned hmask)
{
    buf[4 * sn + sm] = g;
    __syncwarp(hmask);
    double t = 0.0;
#pragma unroll
    for (int n = 0; n < 4; ++n) t = fma(Mq[n * 4 + sn], buf[4 * n + sm], t);
    __syncwarp(hmask);
    buf[4 * sn + sm] = t;
    __syncwarp(hmask);
    double dv = 0.0;
#pragma unroll
    for (int m = 0; m < 4; ++m) dv = fma(buf[4 * sn + m], Mx[m * 4 + sm], dv);
    __syncwarp(hmask);
    return dv;
}

// Half of a cell a point lies in along each axis: bit 0 set when t_x > 1/2,
// bit 1 when t_q > 1/2.  In an upper half the accumulation runs in powers of
// s = 1 - t (and maps back with the cell's matrix in s), so that the weights
// that vanish at the near knot come out of small powers, not of cancelling
// ones: a bin holds the points of one cell (and flavour) and one half pair.
// (The tape records the same two bits, from the same t, for the counting
// pass.)
__device__ __forceinline__ int half_pair(const Axis &X, const Axis &Q)
{
    return (upper_half(X.t) ? 1 : 0) | (upper_half(Q.t) ? 2 : 0);
}

// The local coordinate the accumulation uses: t, or 1 - t in an upper half
// (exact: t lies in [1/2, 1] there).
__device__ __forceinline__ double near_coord(double t) { return upper_half(t) ? 1.0 - t : t; }

// Bin of a point in the pointwise sorted accumulation, ((cell * F + flavour
// column) * 4 + half pair), or -1 for a point that adds nothing there: a
// domain error, outside the grid under the error option, an absent pid, or
// outside the knot range on either axis (see k_bwd_rec).  The counting pass
// and the record pass both take the bin from this one function, on the same
// tape values (or both read the one the forward pass wrote from them into
// the derivative tape), so that every record placed was counted.
__device__ __forceinline__ int sorted_bin(const GridDev &g, const Axis &X, const Axis &Q, bool bad, int col,
                                          int halves, int nbins)
{
    if (bad || col < 0 || !(X.in && Q.in)) return -1;
    return checked_index(g.status, ((Q.cell * g.nxc + X.cell) * g.nflav + col) * 4 + halves, nbins);
}

}  // namespace pdfgpu
