// Adjoint of the interpolation: dL/dx, dL/dQ^2 and dL/d(grid values).
//
// For L = sum_i sum_p gout[i][p] xf_p(x_i, Q^2_i):
//   dL/dx_i   = sum_p gout[i][p] (dP/dtx) / dU / x_i
//   dL/dQ^2_i = sum_p gout[i][p] (dP/dtq) / dW / Q^2_i
// with the patch derivatives taken from the same bicubic coefficients, and
//   dL/dv[row][knot][p] += gout[i][p] Wq_j(tq) Wx_k(tx)
// over the 4x4 stencil, where W are the stencil weights of the Hermite
// cubics with finite-difference slopes (the interpolant is linear in v, so
// these weights are exactly its derivative).  Outside the grid the same
// formulas with the linear basis give the derivatives of the linear
// continuation.  The grid gradient is accumulated with FP64 atomics, either
// into a shared-memory copy per CTA (flushed once at the end) when the
// member's gradient fits, or straight into global memory.  Given the tape of
// the forward pass over the same points, the adjoint rebuilds each point's
// cells and local coordinates from it instead of searching the knots and
// taking the two logarithms again; the arithmetic that follows is the same.
#include <math.h>

#include <algorithm>

#include "pdf_internal.h"

using namespace pdfgpu;

namespace {

constexpr int kBlock = 256;
constexpr size_t kSmemGradMax = 200 * 1024;

__device__ __forceinline__ double qnan() { return __longlong_as_double(0x7FF8000000000000ll); }

template <bool PW, bool SMEM, bool TAPE>
__global__ void __launch_bounds__(kBlock) k_bwd(GridDev g, Cols cols, int npid, int member,
                                                const int *__restrict__ pid,
                                                const double *__restrict__ x,
                                                const double *__restrict__ q2, int64_t n,
                                                const double *__restrict__ tape,
                                                const double *__restrict__ gout,
                                                double *__restrict__ gx, double *__restrict__ gq,
                                                double *__restrict__ gval)
{
    extern __shared__ double sgrad[];
    __shared__ signed char scol[PDF_MAX_PIDS];
    const int gsize = g.nrows * g.nx * g.nflav;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < PDF_MAX_PIDS; ++k) scol[k] = cols.c[k];
    }
    if (SMEM)
        for (int k = threadIdx.x; k < gsize; k += blockDim.x) sgrad[k] = 0.0;
    __syncthreads();
    double *acc = SMEM ? sgrad : gval;
    const size_t cell_stride = (size_t)g.nflav * 16;
    const double *cm = g.coef + (size_t)member * g.nqc * g.nxc * cell_stride;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double xi = x[i], qi = q2[i];
        Axis X, Q;
        if (TAPE) {
            if (tape_get(g, tape, i, X, Q)) {
                if (gx) gx[i] = qnan();
                if (gq) gq[i] = qnan();
                continue;
            }
        } else {
            bool bad = !(x_ok(dbits(xi)) && q2_ok(dbits(qi)));
            if (bad) {
                if (gx) gx[i] = qnan();
                if (gq) gq[i] = qnan();
                continue;
            }
            double u, w;
            X = axis_x(g, xi, &u);
            Q = axis_q2(g, qi, &w);
            if (out_of_range(g, X, Q)) {
                if (gx) gx[i] = qnan();
                if (gq) gq[i] = qnan();
                continue;
            }
        }
        // derivative bases: (0, 1, 2t, 3t^2) inside; outside (0, 1, 1, 1) for
        // the linear continuation, and no derivative across a frozen edge
        double dx2 = X.in ? 2.0 * X.t : 1.0, dx3 = X.in ? 3.0 * X.t * X.t : 1.0;
        double dq2 = Q.in ? 2.0 * Q.t : 1.0, dq3 = Q.in ? 3.0 * Q.t * Q.t : 1.0;
        const bool fzx = !X.in && g.extrap == PDF_EXTRAP_FREEZE;
        const bool fzq = !Q.in && g.extrap == PDF_EXTRAP_FREEZE;
        const double *cell = cm + ((size_t)Q.cell * g.nxc + X.cell) * cell_stride;
        double Wx[4], Wq[4];
        int qmask = 0, r0 = 0, k0 = 0;
        if (gval) {
            stencil_weights(g.mx + (size_t)X.cell * 16, X, Wx);
            stencil_weights(g.mq + (size_t)Q.cell * 16, Q, Wq);
            qmask = g.qmask[Q.cell];
            r0 = g.qrow[Q.cell] - 1;
            k0 = X.cell - 1;
        }
        double sx = 0.0, sq = 0.0;
        const int na = PW ? 1 : npid;
        for (int a = 0; a < na; ++a) {
            int col = PW ? pid_col(g, pid[i]) : scol[a];
            if (col >= 0) col = checked_index(g.status, col, g.nflav);
            if (col < 0) continue;
            double ga = PW ? gout[i] : gout[i * npid + a];
            double dtx, dtq;
            patch_d(cell + col * 16, X, Q, dx2, dx3, dq2, dq3, &dtx, &dtq);
            if (fzx) dtx = 0.0;
            if (fzq) dtq = 0.0;
            sx = fma(ga, dtx, sx);
            sq = fma(ga, dtq, sq);
            if (gval) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (!((qmask >> j) & 1)) continue;
                    double gj = ga * Wq[j];
                    const int row = checked_index(g.status, r0 + j, g.nrows);
                    double *rowp = acc + ((size_t)row * g.nx) * g.nflav + col;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        int kk = k0 + k;
                        if (kk < 0 || kk >= g.nx) continue;
                        atomicAdd(rowp + (size_t)kk * g.nflav, gj * Wx[k]);
                    }
                }
            }
        }
        if (gx) gx[i] = sx * g.xcell[X.cell].y * __drcp_rn(xi);
        if (gq) gq[i] = sq * g.qcell[Q.cell].y * __drcp_rn(qi);
    }
    if (SMEM) {
        __syncthreads();
        for (int k = threadIdx.x; k < gsize; k += blockDim.x) {
            double v = sgrad[k];
            if (dbits(v) << 1) atomicAdd(gval + k, v);
        }
    }
}

template <bool PW, bool TAPE>
int launch(pdfgpu_grid *g, const Cols &cols, int npid, int member, const int *pid, const double *x,
           const double *q2, int64_t n, const double *tape, const double *gout, double *gx, double *gq,
           double *gval, cudaStream_t s)
{
    size_t gbytes = (size_t)g->d.nrows * g->d.nx * g->d.nflav * sizeof(double);
    if (gval && gbytes <= kSmemGradMax) {
        const void *kern = (const void *)k_bwd<PW, true, TAPE>;
        int rc = allow_dynamic_smem(kern, gbytes);
        if (rc) return rc;
        int grid = wave_grid(g, kern, kBlock, gbytes, n);
        k_bwd<PW, true, TAPE><<<grid, kBlock, gbytes, s>>>(g->d, cols, npid, member, pid, x, q2, n, tape, gout,
                                                            gx, gq, gval);
    } else {
        const void *kern = (const void *)k_bwd<PW, false, TAPE>;
        int grid = wave_grid(g, kern, kBlock, 0, n);
        k_bwd<PW, false, TAPE><<<grid, kBlock, 0, s>>>(g->d, cols, npid, member, pid, x, q2, n, tape, gout, gx,
                                                        gq, gval);
    }
    PDF_CUDA(cudaGetLastError());
    return PDF_OK;
}

int backward(pdfgpu_grid_t g, int32_t member, const int32_t *pids, int32_t n_pid, int32_t pointwise,
             const double *x, const double *q2, int64_t n, const double *tape, const double *grad_out,
             double *grad_x, double *grad_q2, double *grad_values, cudaStream_t s)
{
    clear_error();
    int rc = check_grid(g, true);
    if (rc) return rc;
    if (g->d.extrap == PDF_EXTRAP_CONTINUATION)
        return fail(PDF_E_ARG, "the adjoint needs linear, freeze or error extrapolation (continuation is not linear "
                               "in the grid values)");
    if (n < 0) return fail(PDF_E_ARG, "negative n");
    if (member < 0 || member >= g->d.nmem) return fail(PDF_E_ARG, "member out of range");
    if (tape && (uintptr_t)tape % 32) return fail(PDF_E_ARG, "tape must be 32-byte aligned");
    Cols cols;
    memset(&cols, -1, sizeof(cols));
    if (!pointwise) {
        rc = resolve_cols(g, pids, n_pid, &cols);
        if (rc) return rc;
    }
    if (n == 0) return PDF_OK;
    if (!x || !q2 || !grad_out || !pids) return fail(PDF_E_ARG, "null array");
    if (pointwise)
        return tape ? launch<true, true>(g, cols, 1, member, pids, x, q2, n, tape, grad_out, grad_x, grad_q2,
                                         grad_values, s)
                    : launch<true, false>(g, cols, 1, member, pids, x, q2, n, nullptr, grad_out, grad_x, grad_q2,
                                          grad_values, s);
    return tape ? launch<false, true>(g, cols, n_pid, member, nullptr, x, q2, n, tape, grad_out, grad_x, grad_q2,
                                      grad_values, s)
                : launch<false, false>(g, cols, n_pid, member, nullptr, x, q2, n, nullptr, grad_out, grad_x,
                                       grad_q2, grad_values, s);
}

}  // namespace

extern "C" int xfxQ2_backward(pdfgpu_grid_t g, int32_t member, const int32_t *pids, int32_t n_pid,
                              int32_t pointwise, const double *x, const double *q2, int64_t n,
                              const double *grad_out, double *grad_x, double *grad_q2,
                              double *grad_values, pdfgpu_stream_t stream)
{
    PDF_TRACE("xfxQ2_backward");
    return backward(g, member, pids, n_pid, pointwise, x, q2, n, nullptr, grad_out, grad_x, grad_q2, grad_values,
                    (cudaStream_t)stream);
}

extern "C" int xfxQ2_backward_tape(pdfgpu_grid_t g, int32_t member, const int32_t *pids, int32_t n_pid,
                                   int32_t pointwise, const double *x, const double *q2, int64_t n,
                                   const double *tape, const double *grad_out, double *grad_x, double *grad_q2,
                                   double *grad_values, pdfgpu_stream_t stream)
{
    PDF_TRACE("xfxQ2_backward_tape");
    if (!tape && n != 0) {
        clear_error();
        return fail(PDF_E_ARG, "null tape");
    }
    return backward(g, member, pids, n_pid, pointwise, x, q2, n, tape, grad_out, grad_x, grad_q2, grad_values,
                    (cudaStream_t)stream);
}
