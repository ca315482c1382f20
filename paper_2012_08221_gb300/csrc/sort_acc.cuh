// Device helper shared by the adjoints that accumulate a grid gradient in
// the monomial basis of the interpolation patch (the grid gradients of
// bwd.cu and the luminosity adjoint of lumi.cu): per bin of sorted points a
// half-warp holds G[n][m] = sum over the bin's points of (weight) bq_n bx_m
// and maps it back to the 16 stencil values once per run of the bin.
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

}  // namespace pdfgpu
