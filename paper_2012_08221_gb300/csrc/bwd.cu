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
// continuation.  Given the tape of the forward pass over the same points,
// the adjoint rebuilds each point's cells and local coordinates from it
// instead of searching the knots and taking the two logarithms again; the
// arithmetic that follows is the same.  A pointwise forward pass may also
// keep each point's two patch derivatives (the derivative tape), computed
// with its value by the same routine the adjoint would use, so that the
// adjoint reads them instead of reloading the coefficients.
//
// Grid gradient: the points are counting-sorted into bins of one cell, one
// flavour (pointwise form; the matrix form bins by cell and keeps every
// column of the call in the same bin) and one half of the cell along each
// axis -- a counting pass over the tape's cells (the forward's tape, or one
// made here), a scan, and the record pass placing each point's record in its
// bin -- and the gradient is accumulated per bin in the monomial basis of
// the patch,
//   G[n][m] = sum over the bin's points of g bq_n bx_m,
// one FMA per term with no stencil weights, then mapped back to the 16
// stencil values once per bin run: dL/dv[j][i] = sum_n,m Mq[n][j] G[n][m]
// Mx[m][i] (the transpose of the map that builds the patch from the
// values, so the result is the same derivative).  In the upper half of an
// axis the basis is in powers of s = 1 - t, with the cell's matrix in s.
// Beyond 16 columns the matrix form scatters the 16 stencil weights per
// flavour with FP64 atomics, into a shared-memory copy per CTA when the
// member's gradient fits, or straight into global memory.
#include <math.h>
#include <stdlib.h>

#include <algorithm>

#include "pdf_internal.h"
#include "sort_acc.cuh"

using namespace pdfgpu;

namespace {

constexpr int kBlock = 256;
constexpr size_t kSmemGradMax = 200 * 1024;

__device__ __forceinline__ double qnan() { return __longlong_as_double(0x7FF8000000000000ll); }

// Chain rule from the local coordinates to x and Q^2: given sx = g dP/dtx
// and sq = g dP/dtq, dL/dx = sx (1/dU) / x and dL/dQ^2 = sq (1/dW) / Q^2,
// with one reciprocal of x Q^2 for both (1/x = Q^2 / (x Q^2), 1/Q^2 =
// x / (x Q^2)); where the product leaves the normal range the two
// reciprocals are taken apart.  Every adjoint goes through here, so their
// dL/dx and dL/dQ^2 stay the same bits.
__device__ __forceinline__ void chain_rule(double sx, double sq, double ydu, double ydw, double x, double q2,
                                           double *__restrict__ gx, double *__restrict__ gq, int64_t i)
{
    const double xq = x * q2;
    double rx, rq;
    if (dbits(xq) - 0x0010000000000000ull < 0x7FE0000000000000ull) {   // normal and finite
        const double r = __drcp_rn(xq);
        rx = q2 * r;
        rq = x * r;
    } else {
        rx = __drcp_rn(x);
        rq = __drcp_rn(q2);
    }
    if (gx) gx[i] = sx * ydu * rx;
    if (gq) gq[i] = sq * ydw * rq;
}

template <bool PW, bool SMEM, bool TAPE>
__global__ void __launch_bounds__(kBlock) k_bwd(GridDev g, Cols cols, int npid, int member,
                                                const int *__restrict__ pid,
                                                const double *__restrict__ x,
                                                const double *__restrict__ q2, int64_t n,
                                                const double *__restrict__ tape,
                                                const double *__restrict__ dtape,
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
        // derivatives of the patch: (0, 1, 2t, 3t^2) inside; outside (0, 1, 1, 1)
        // for the linear continuation, and none across a frozen edge
        const bool fzx = !X.in && g.extrap == PDF_EXTRAP_FREEZE;
        const bool fzq = !Q.in && g.extrap == PDF_EXTRAP_FREEZE;
        const double *cell = cm + ((size_t)Q.cell * g.nxc + X.cell) * cell_stride;
        double Wx[4], Wq[4];
        int qmask = 0, r0 = 0, k0 = 0;
        if (gval) {
            stencil_weights(g.mx + (size_t)X.cell * 16, g.mxs + (size_t)X.cell * 16, X, Wx);
            stencil_weights(g.mq + (size_t)Q.cell * 16, g.mqs + (size_t)Q.cell * 16, Q, Wq);
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
            if (PW && TAPE && dtape) {
                const double2 d = __ldg(reinterpret_cast<const double2 *>(dtape) + i);
                dtx = d.x;
                dtq = d.y;
            } else {
                patch_vd(cell + col * 16, X, Q, &dtx, &dtq);
            }
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
        chain_rule(sx, sq, g.xcell[X.cell].y, g.qcell[Q.cell].y, xi, qi, gx, gq, i);
    }
    if (SMEM) {
        __syncthreads();
        for (int k = threadIdx.x; k < gsize; k += blockDim.x) {
            double v = sgrad[k];
            if (dbits(v) << 1) atomicAdd(gval + k, v);
        }
    }
}

// ------------------------------------------- sorted pointwise grid gradient

constexpr int kMaxSmemBins = 50 * 1024;   // bin counters in shared memory (200 KB, one block per SM)
constexpr int kCountBlock = 1024;         // one such block per SM counts
constexpr int kCountIlp = 4;
constexpr int kAccWarps = 4;
constexpr int kSegment = 1024;            // sorted points per warp of the accumulation
constexpr int kSegmentM = 128;            // the same for the matrix form (npid FMAs per point
                                          // and lane: shorter runs keep enough warps busy)
constexpr int64_t kSortChunk = (int64_t)1 << 24;

// Sorted record of one point (32 bytes): t of the x axis, t of the Q axis
// (as the tape holds them), g = dL/d(x*f) of the point, and the bits of
// bin (low 32) | x inside (bit 32) | Q inside (bit 33).
__device__ __forceinline__ void put_rec(double *__restrict__ rec, int pos, double tx, double tq, double ga,
                                        int b, bool xin, bool qin)
{
    const uint64_t bits = (uint64_t)(uint32_t)b | ((uint64_t)xin << 32) | ((uint64_t)qin << 33);
    double2 *d = reinterpret_cast<double2 *>(rec + 4 * (size_t)pos);
    d[0] = make_double2(tx, tq);
    d[1] = make_double2(ga, dfrom(bits));
}

// Bin of a point in the matrix form's sorted accumulation: its cell and
// half pair (all the call's flavours accumulate together), (cell * 4 + half
// pair), or -1 as for sorted_bin.
__device__ __forceinline__ int sorted_cell(const GridDev &g, const Axis &X, const Axis &Q, bool bad, int halves,
                                           int nbins)
{
    if (bad || !(X.in && Q.in)) return -1;
    return checked_index(g.status, (Q.cell * g.nxc + X.cell) * 4 + halves, nbins);
}

// Without a forward tape: the tape records of the chunk's points (domain
// check, both knot searches and logarithms), into chunk-local scratch.
__global__ void __launch_bounds__(kBlock) k_bwd_axes(GridDev g, const double *__restrict__ x,
                                                     const double *__restrict__ q2, int64_t i0, int m,
                                                     double *__restrict__ tape)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
        const double xi = x[i0 + k], qi = q2[i0 + k];
        bool bad = !(x_ok(dbits(xi)) && q2_ok(dbits(qi)));
        double u, w;
        Axis X = axis_x(g, bad ? 0.5 : xi, &u);
        Axis Q = axis_q2(g, bad ? 10.0 : qi, &w);
        bad |= out_of_range(g, X, Q);
        tape_put(tape, k, X, Q, bad);
    }
}

// Histogram of the chunk's bins from the tape records' cells, flags and
// halves and the pids (20 bytes read per point, no FP64 work).  One block of kCountBlock threads
// per SM, so that flushing the shared-memory counters costs one pass over
// the bins per SM, not per small block.  `tape` is the chunk's view.
template <bool PW>
__global__ void __launch_bounds__(kCountBlock) k_bwd_count(GridDev g, const int *__restrict__ pid,
                                                           const double *__restrict__ tape, int64_t i0, int m,
                                                           int *__restrict__ hist, int nbins)
{
    extern __shared__ int shist[];
    const bool sh = nbins <= kMaxSmemBins;
    if (sh) {
        for (int k = threadIdx.x; k < nbins; k += blockDim.x) shist[k] = 0;
        __syncthreads();
    }
    // kCountIlp points per thread at a time: the pass is bound by memory
    // latency, so each thread keeps that many loads in flight
    // (all of a group's loads, the tape records' cells and flags and the
    // pids, are issued before any is used)
    const int stride = gridDim.x * blockDim.x;
    for (int k0 = blockIdx.x * blockDim.x + threadIdx.x; k0 < m; k0 += kCountIlp * stride) {
        int b[kCountIlp], pv[kCountIlp];
        double2 r[kCountIlp];
#pragma unroll
        for (int u = 0; u < kCountIlp; ++u) {
            const int k = k0 + u * stride;
            if (k < m) {
                r[u] = tape_cells_raw(tape, k);
                if (PW) pv[u] = __ldg(pid + i0 + k);
            }
        }
#pragma unroll
        for (int u = 0; u < kCountIlp; ++u) {
            const int k = k0 + u * stride;
            b[u] = -1;
            if (k < m) {
                Axis X, Q;
                unsigned halves;
                const bool bad = tape_decode(g, r[u].x, r[u].y, X, Q, &halves);
                b[u] = PW ? sorted_bin(g, X, Q, bad, bad ? -1 : pid_col(g, pv[u]), (int)halves, nbins)
                          : sorted_cell(g, X, Q, bad, (int)halves, nbins);
            }
        }
#pragma unroll
        for (int u = 0; u < kCountIlp; ++u) {
            if (b[u] < 0) continue;
            if (sh) atomicAdd(&shist[b[u]], 1);
            else atomicAdd(&hist[b[u]], 1);
        }
    }
    if (sh) {
        __syncthreads();
        for (int k = threadIdx.x; k < nbins; k += blockDim.x)
            if (shist[k]) atomicAdd(&hist[k], shist[k]);
    }
}

// Per point (chunk-local index k of point i0 + k, tape record k of the
// chunk's view): dL/dx and dL/dQ^2 as in k_bwd, and the point's record,
// placed in the next free slot of its bin (cursor[b], from the scan of
// k_bwd_count's histogram): the scattered store overlaps the FP64 work.  A
// point outside the knot range on either axis has no record: it adds its
// exact stencil weights of the extrapolation, (1 - t, t) on the edge cell's
// two knots, to the gradient here with global atomics (rare points; through
// the monomial basis the two knots that carry no weight would receive
// rounding-sized terms instead of zeros).
template <bool DT>
__global__ void __launch_bounds__(kBlock, 5) k_bwd_rec(GridDev g, int member, const int *__restrict__ pid,
                                                    const double *__restrict__ x,
                                                    const double *__restrict__ q2, int64_t i0, int m,
                                                    const double *__restrict__ tape,
                                                    const double *__restrict__ dtape,
                                                    const int *__restrict__ dbins,
                                                    const double *__restrict__ gout,
                                                    double *__restrict__ gx, double *__restrict__ gq,
                                                    double *__restrict__ gval, int nbins,
                                                    int *__restrict__ cursor, double *__restrict__ rec)
{
    const size_t cell_stride = (size_t)g.nflav * 16;
    const double *cm = g.coef + (size_t)member * g.nqc * g.nxc * cell_stride;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
        const int64_t i = i0 + k;
        Axis X, Q;
        if (tape_get(g, tape, k, X, Q)) {
            if (gx) gx[i] = qnan();
            if (gq) gq[i] = qnan();
            continue;
        }
        const int col = pid_col(g, pid[i]);
        if (col < 0) {
            if (gx) gx[i] = 0.0;
            if (gq) gq[i] = 0.0;
            continue;
        }
        const double ga = gout[i];
        if (gx || gq) {
            double dtx, dtq;
            if (DT) {
                const double2 d = __ldg(reinterpret_cast<const double2 *>(dtape) + i);
                dtx = d.x;
                dtq = d.y;
            } else {
                patch_vd(cm + ((size_t)Q.cell * g.nxc + X.cell) * cell_stride + col * 16, X, Q, &dtx, &dtq);
            }
            if (!X.in && g.extrap == PDF_EXTRAP_FREEZE) dtx = 0.0;
            if (!Q.in && g.extrap == PDF_EXTRAP_FREEZE) dtq = 0.0;
            chain_rule(ga * dtx, ga * dtq, g.xcell[X.cell].y, g.qcell[Q.cell].y, x[i], q2[i], gx, gq, i);
        }
        if (!(X.in && Q.in)) {
            double Wx[4], Wq[4];
            stencil_weights(g.mx + (size_t)X.cell * 16, g.mxs + (size_t)X.cell * 16, X, Wx);
            stencil_weights(g.mq + (size_t)Q.cell * 16, g.mqs + (size_t)Q.cell * 16, Q, Wq);
            const int qmask = g.qmask[Q.cell], r0 = g.qrow[Q.cell] - 1, k0 = X.cell - 1;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (!((qmask >> j) & 1)) continue;
                const double gj = ga * Wq[j];
                const int row = checked_index(g.status, r0 + j, g.nrows);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int kk = k0 + c;
                    const double t = gj * Wx[c];
                    if (kk >= 0 && kk < g.nx && (dbits(t) << 1))
                        atomicAdd(gval + ((size_t)row * g.nx + kk) * g.nflav + col, t);
                }
            }
            continue;
        }
        const int b = DT ? checked_index(g.status, __ldg(dbins + i), nbins)
                         : sorted_bin(g, X, Q, false, col, half_pair(X, Q), nbins);
        put_rec(rec, atomicAdd(&cursor[b], 1), near_coord(X.t), near_coord(Q.t), ga, b, X.in, Q.in);
    }
}

// Accumulation over the sorted records.  Each warp takes a segment of
// kSegment records and each half-warp half of it, in steps of 16: lane s of
// the half stages record p + s (g times the Q basis, and the x basis) in
// shared memory, then, for each of the 16 staged records in order, lane
// s = 4 n + m adds g bq_n bx_m to its accumulator G[n][m] of the current
// bin (one FMA).  When the bin changes the half-warp maps its 16
// accumulators back to the 16 stencil values (map_back), each lane adding
// its value to the gradient with one atomic.
__global__ void __launch_bounds__(kAccWarps * 32) k_bwd_accum(GridDev g, const double *__restrict__ rec,
                                                              const int *__restrict__ offs, int nbins,
                                                              double *__restrict__ gval)
{
    __shared__ double sV[kAccWarps][32][9];      // per staged record: g bq[4], bx[4] (padded)
    __shared__ int sK[kAccWarps][32];
    __shared__ double sG[kAccWarps][32];         // accumulators handed over at a flush
    const int F = g.nflav;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nvalid = offs[nbins];
    const int64_t wbeg = ((int64_t)blockIdx.x * kAccWarps + wid) * kSegment;
    if (wbeg >= nvalid) return;
    const int wend = (int)min((int64_t)nvalid, wbeg + kSegment);
    const int h = lane >> 4, s = lane & 15, sn = s >> 2, sm = s & 3;
    const unsigned hmask = 0xFFFFu << (16 * h);
    const int half = (wend - (int)wbeg + 1) / 2;
    const int beg = (int)wbeg + h * half;
    const int end = h ? wend : (int)wbeg + half;
    const int row0 = h * 16;
    double acc = 0.0;
    int cur = -1;
    auto flush = [&](int b) {
        const int cb = b >> 2, cell = cb / F, col = cb - cell * F;
        const int qc = cell / g.nxc, xc = cell - qc * g.nxc;
        const double *Mq = ((b & 2) ? g.mqs : g.mq) + (size_t)qc * 16;
        const double *Mx = ((b & 1) ? g.mxs : g.mx) + (size_t)xc * 16;
        const double dv = map_back(acc, &sG[wid][row0], Mq, Mx, sn, sm, hmask);   // lane (j, i) = (sn, sm)
        acc = 0.0;
        const int kk = xc - 1 + sm;
        if (((g.qmask[qc] >> sn) & 1) && kk >= 0 && kk < g.nx && (dbits(dv) << 1)) {
            const int row = checked_index(g.status, g.qrow[qc] - 1 + sn, g.nrows);
            atomicAdd(gval + ((size_t)row * g.nx + kk) * F + col, dv);
        }
    };
    const int steps = (half + 15) / 16;
    for (int step = 0; step < steps; ++step) {
        const int p = beg + step * 16;
        const int r = p + s;
        int kr = -1;
        if (r < end) {
            const D4 t = ld4(rec + 4 * (size_t)r);
            const uint64_t bits = dbits(t.w);
            kr = (int)(uint32_t)bits;
            const bool xin = (bits >> 32) & 1, qin = (bits >> 33) & 1;
            const double tx2 = t.x * t.x, tq2 = t.y * t.y;
            const double gq1 = t.z * t.y;
            double *v = sV[wid][row0 + s];
            v[0] = t.z;
            v[1] = gq1;
            v[2] = qin ? gq1 * t.y : gq1;
            v[3] = qin ? gq1 * tq2 : gq1;
            v[4] = 1.0;
            v[5] = t.x;
            v[6] = xin ? tx2 : t.x;
            v[7] = xin ? tx2 * t.x : t.x;
        }
        sK[wid][row0 + s] = kr;
        __syncwarp();
        const int nb = min(16, end - p);
        for (int q = 0; q < nb; ++q) {
            const int kq = sK[wid][row0 + q];
            if (kq != cur) {
                if (cur >= 0) flush(cur);
                cur = kq;
            }
            acc = fma(sV[wid][row0 + q][sn], sV[wid][row0 + q][4 + sm], acc);
        }
        __syncwarp();
    }
    if (cur >= 0) flush(cur);
}

// ------------------------------------------ sorted matrix-form grid gradient
//
// The matrix form (a shared list of up to kMaxSortedPids flavour columns,
// gout [n][npid]) sorts the points by cell only: every column of a point
// accumulates in the same bin, lane 4n + m of a half-warp keeping
// G_a[n][m] for every column a.  dL/dx and dL/dQ^2 take the derivative of
// one combined patch, sum_a g_a C_a (16 FMA per column), instead of one
// derivative per column (the result is linear in the coefficients).

constexpr int kMaxSortedPids = 16;

// Derivatives of a patch held in registers (as patch_vd).
__device__ __forceinline__ void patch_d_regs(const double C[16], const Axis &X, const Axis &Q, double *dtx,
                                             double *dtq)
{
    D4 r[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) r[n] = D4{C[4 * n], C[4 * n + 1], C[4 * n + 2], C[4 * n + 3]};
    patch_vd_rows(r, X, Q, dtx, dtq);
}

// Per point: dL/dx and dL/dQ^2 from the combined patch, and the point's
// record (t_x, t_q, bits of cell | x inside << 32 | Q inside << 33, point
// index) placed in its cell's range; points outside the knot range add
// their exact extrapolation weights per column with global atomics.
__global__ void __launch_bounds__(kBlock) k_bwd_rec_m(GridDev g, Cols cols, int npid, int member,
                                                      const double *__restrict__ x,
                                                      const double *__restrict__ q2, int64_t i0, int m,
                                                      const double *__restrict__ tape,
                                                      const double *__restrict__ gout,
                                                      double *__restrict__ gx, double *__restrict__ gq,
                                                      double *__restrict__ gval, int nbins,
                                                      int *__restrict__ cursor, double *__restrict__ rec)
{
    __shared__ signed char scol[PDF_MAX_PIDS];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < PDF_MAX_PIDS; ++k) scol[k] = cols.c[k];
    }
    __syncthreads();
    const size_t cell_stride = (size_t)g.nflav * 16;
    const double *cm = g.coef + (size_t)member * g.nqc * g.nxc * cell_stride;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
        const int64_t i = i0 + k;
        Axis X, Q;
        if (tape_get(g, tape, k, X, Q)) {
            if (gx) gx[i] = qnan();
            if (gq) gq[i] = qnan();
            continue;
        }
        const double *cell = cm + ((size_t)Q.cell * g.nxc + X.cell) * cell_stride;
        const double *go = gout + (size_t)i * npid;
        if (gx || gq) {
            double C[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) C[c] = 0.0;
            for (int a = 0; a < npid; ++a) {
                int col = scol[a];
                if (col < 0) continue;
                col = checked_index(g.status, col, g.nflav);
                const double ga = go[a];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const D4 v = ld4(cell + col * 16 + 4 * r);
                    C[4 * r] = fma(ga, v.x, C[4 * r]);
                    C[4 * r + 1] = fma(ga, v.y, C[4 * r + 1]);
                    C[4 * r + 2] = fma(ga, v.z, C[4 * r + 2]);
                    C[4 * r + 3] = fma(ga, v.w, C[4 * r + 3]);
                }
            }
            double dtx, dtq;
            patch_d_regs(C, X, Q, &dtx, &dtq);
            if (!X.in && g.extrap == PDF_EXTRAP_FREEZE) dtx = 0.0;
            if (!Q.in && g.extrap == PDF_EXTRAP_FREEZE) dtq = 0.0;
            chain_rule(dtx, dtq, g.xcell[X.cell].y, g.qcell[Q.cell].y, x[i], q2[i], gx, gq, i);
        }
        if (!(X.in && Q.in)) {
            double Wx[4], Wq[4];
            stencil_weights(g.mx + (size_t)X.cell * 16, g.mxs + (size_t)X.cell * 16, X, Wx);
            stencil_weights(g.mq + (size_t)Q.cell * 16, g.mqs + (size_t)Q.cell * 16, Q, Wq);
            const int qmask = g.qmask[Q.cell], r0 = g.qrow[Q.cell] - 1, k0 = X.cell - 1;
            for (int a = 0; a < npid; ++a) {
                int col = scol[a];
                if (col < 0) continue;
                col = checked_index(g.status, col, g.nflav);
                const double ga = go[a];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (!((qmask >> j) & 1)) continue;
                    const double gj = ga * Wq[j];
                    const int row = checked_index(g.status, r0 + j, g.nrows);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int kk = k0 + c;
                        const double t = gj * Wx[c];
                        if (kk >= 0 && kk < g.nx && (dbits(t) << 1))
                            atomicAdd(gval + ((size_t)row * g.nx + kk) * g.nflav + col, t);
                    }
                }
            }
            continue;
        }
        const int b = sorted_cell(g, X, Q, false, half_pair(X, Q), nbins);
        const int pos = atomicAdd(&cursor[b], 1);
        const uint64_t bits = (uint64_t)(uint32_t)b | ((uint64_t)X.in << 32) | ((uint64_t)Q.in << 33);
        double2 *d = reinterpret_cast<double2 *>(rec + 4 * (size_t)pos);
        d[0] = make_double2(near_coord(X.t), near_coord(Q.t));
        d[1] = make_double2(dfrom(bits), dfrom((uint64_t)i));
    }
}

// Accumulation over the cell-sorted records of the matrix form: as
// k_bwd_accum, but each staged record carries the point's whole gout row,
// and lane 4n + m adds w g_a to G_a[n][m] for every column a, with
// w = bq_n bx_m (one multiply and npid FMAs per record).  At a cell change
// the half-warp maps G_a back to the 16 stencil values of column a, one
// column after another.
__global__ void __launch_bounds__(kAccWarps * 32) k_bwd_accum_m(GridDev g, Cols cols, int npid,
                                                                const double *__restrict__ rec,
                                                                const int *__restrict__ offs, int nbins,
                                                                const double *__restrict__ gout,
                                                                double *__restrict__ gval)
{
    __shared__ double sV[kAccWarps][32][9];                   // bq[4], bx[4] (padded)
    __shared__ double sGo[kAccWarps][32][kMaxSortedPids + 1]; // the record's gout row (padded)
    __shared__ int sK[kAccWarps][32];
    __shared__ double sG[kAccWarps][32];
    __shared__ signed char scol[PDF_MAX_PIDS];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < PDF_MAX_PIDS; ++k) scol[k] = cols.c[k];
    }
    __syncthreads();
    const int F = g.nflav;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nvalid = offs[nbins];
    const int64_t wbeg = ((int64_t)blockIdx.x * kAccWarps + wid) * kSegmentM;
    if (wbeg >= nvalid) return;
    const int wend = (int)min((int64_t)nvalid, wbeg + kSegmentM);
    const int h = lane >> 4, s = lane & 15, sn = s >> 2, sm = s & 3;
    const unsigned hmask = 0xFFFFu << (16 * h);
    const int half = (wend - (int)wbeg + 1) / 2;
    const int beg = (int)wbeg + h * half;
    const int end = h ? wend : (int)wbeg + half;
    const int row0 = h * 16;
    double acc[kMaxSortedPids];
#pragma unroll
    for (int a = 0; a < kMaxSortedPids; ++a) acc[a] = 0.0;
    int cur = -1;
    auto flush = [&](int b) {
        const int cell = b >> 2, qc = cell / g.nxc, xc = cell - qc * g.nxc;
        const double *Mq = ((b & 2) ? g.mqs : g.mq) + (size_t)qc * 16;
        const double *Mx = ((b & 1) ? g.mxs : g.mx) + (size_t)xc * 16;
        const int kk = xc - 1 + sm;
        const bool ok = ((g.qmask[qc] >> sn) & 1) && kk >= 0 && kk < g.nx;
        const int row = ok ? checked_index(g.status, g.qrow[qc] - 1 + sn, g.nrows) : 0;
#pragma unroll
        for (int a = 0; a < kMaxSortedPids; ++a) {
            if (a < npid && scol[a] >= 0) {
                const double dv = map_back(acc[a], &sG[wid][row0], Mq, Mx, sn, sm, hmask);
                if (ok && (dbits(dv) << 1)) {
                    const int col = checked_index(g.status, scol[a], F);
                    atomicAdd(gval + ((size_t)row * g.nx + kk) * F + col, dv);
                }
            }
            acc[a] = 0.0;
        }
    };
    const int steps = (half + 15) / 16;
    for (int step = 0; step < steps; ++step) {
        const int p = beg + step * 16;
        const int r = p + s;
        int kr = -1;
        if (r < end) {
            const D4 t = ld4(rec + 4 * (size_t)r);
            const uint64_t bits = dbits(t.z);
            const int64_t i = (int64_t)dbits(t.w);
            kr = (int)(uint32_t)bits;
            const bool xin = (bits >> 32) & 1, qin = (bits >> 33) & 1;
            const double tx2 = t.x * t.x, tq2 = t.y * t.y;
            double *v = sV[wid][row0 + s];
            v[0] = 1.0;
            v[1] = t.y;
            v[2] = qin ? tq2 : t.y;
            v[3] = qin ? tq2 * t.y : t.y;
            v[4] = 1.0;
            v[5] = t.x;
            v[6] = xin ? tx2 : t.x;
            v[7] = xin ? tx2 * t.x : t.x;
            const double *go = gout + (size_t)i * npid;
            for (int a = 0; a < npid; ++a) sGo[wid][row0 + s][a] = go[a];
        }
        sK[wid][row0 + s] = kr;
        __syncwarp();
        const int nb = min(16, end - p);
        for (int q = 0; q < nb; ++q) {
            const int kq = sK[wid][row0 + q];
            if (kq != cur) {
                if (cur >= 0) flush(cur);
                cur = kq;
            }
            const double w = sV[wid][row0 + q][sn] * sV[wid][row0 + q][4 + sm];
#pragma unroll
            for (int a = 0; a < kMaxSortedPids; ++a)
                if (a < npid) acc[a] = fma(w, sGo[wid][row0 + q][a], acc[a]);
        }
        __syncwarp();
    }
    if (cur >= 0) flush(cur);
}

// The same accumulation with the columns split between the two halves of a
// warp (for 5 or more columns): the whole warp walks its segment's records
// together, 16 at a time -- lanes 0-15 stage a record's 16 basis products
// bq_n bx_m (9 multiplies, the rest are copies), lanes 16-31 its gout row --
// and half h accumulates columns [h C, min(npid, (h + 1) C)), C = ceil(npid
// / 2), lane s owning G[s >> 2][s & 3] of each.  Every record reaches both
// halves, so a bin's run can span the whole segment and each half maps back
// half of the columns: half as many map-backs per record as with the
// records split between the halves, the same FMAs.
constexpr int kHalfPids = kMaxSortedPids / 2;

__global__ void __launch_bounds__(kAccWarps * 32) k_bwd_accum_mc(GridDev g, Cols cols, int npid,
                                                                 const double *__restrict__ rec,
                                                                 const int *__restrict__ offs, int nbins,
                                                                 const double *__restrict__ gout,
                                                                 double *__restrict__ gval)
{
    __shared__ double sW[kAccWarps][16][17];                   // a record's basis products (padded)
    __shared__ double sGo[kAccWarps][16][kMaxSortedPids + 1];  // its gout row (padded)
    __shared__ int sK[kAccWarps][16];
    __shared__ double sG[kAccWarps][32];
    __shared__ signed char scol[PDF_MAX_PIDS];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < PDF_MAX_PIDS; ++k) scol[k] = cols.c[k];
    }
    __syncthreads();
    const int F = g.nflav;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nvalid = offs[nbins];
    const int64_t wbeg = ((int64_t)blockIdx.x * kAccWarps + wid) * kSegmentM;
    if (wbeg >= nvalid) return;
    const int wend = (int)min((int64_t)nvalid, wbeg + kSegmentM);
    const int h = lane >> 4, s = lane & 15, sn = s >> 2, sm = s & 3;
    const unsigned hmask = 0xFFFFu << (16 * h);
    const int row0 = h * 16;
    const int C = (npid + 1) / 2;
    const int a0 = h * C;
    const int na = min(npid - a0, C);
    double acc[kHalfPids];
#pragma unroll
    for (int a = 0; a < kHalfPids; ++a) acc[a] = 0.0;
    int cur = -1;
    auto flush = [&](int b) {
        const int cell = b >> 2, qc = cell / g.nxc, xc = cell - qc * g.nxc;
        const double *Mq = ((b & 2) ? g.mqs : g.mq) + (size_t)qc * 16;
        const double *Mx = ((b & 1) ? g.mxs : g.mx) + (size_t)xc * 16;
        const int kk = xc - 1 + sm;
        const bool ok = ((g.qmask[qc] >> sn) & 1) && kk >= 0 && kk < g.nx;
        const int row = ok ? checked_index(g.status, g.qrow[qc] - 1 + sn, g.nrows) : 0;
#pragma unroll
        for (int a = 0; a < kHalfPids; ++a) {
            if (a < na && scol[a0 + a] >= 0) {   // the same for the 16 lanes of a half
                const double dv = map_back(acc[a], &sG[wid][row0], Mq, Mx, sn, sm, hmask);
                if (ok && (dbits(dv) << 1)) {
                    const int col = checked_index(g.status, scol[a0 + a], F);
                    atomicAdd(gval + ((size_t)row * g.nx + kk) * F + col, dv);
                }
            }
            acc[a] = 0.0;
        }
    };
    for (int p = (int)wbeg; p < wend; p += 16) {
        const int r = p + s;
        int kr = -1;
        if (r < wend) {
            const D4 t = ld4(rec + 4 * (size_t)r);
            const uint64_t bits = dbits(t.z);
            kr = (int)(uint32_t)bits;
            if (h == 0) {
                const bool xin = (bits >> 32) & 1, qin = (bits >> 33) & 1;
                const double tq2 = t.y * t.y, tx2 = t.x * t.x;
                const double bq[4] = {1.0, t.y, qin ? tq2 : t.y, qin ? tq2 * t.y : t.y};
                const double bx[4] = {1.0, t.x, xin ? tx2 : t.x, xin ? tx2 * t.x : t.x};
                double *w = sW[wid][s];
#pragma unroll
                for (int m = 0; m < 4; ++m) w[m] = bx[m];
#pragma unroll
                for (int n = 1; n < 4; ++n) {
                    w[4 * n] = bq[n];
#pragma unroll
                    for (int m = 1; m < 4; ++m) w[4 * n + m] = bq[n] * bx[m];
                }
                sK[wid][s] = kr;
            } else {
                const double *go = gout + (size_t)(int64_t)dbits(t.w) * npid;
                for (int a = 0; a < npid; ++a) sGo[wid][s][a] = go[a];
            }
        } else if (h == 0) {
            sK[wid][s] = -1;
        }
        __syncwarp();
        const int nb = min(16, wend - p);
        for (int q = 0; q < nb; ++q) {
            const int kq = sK[wid][q];
            if (kq != cur) {
                if (cur >= 0) flush(cur);
                cur = kq;
            }
            const double w = sW[wid][q][s];
#pragma unroll
            for (int a = 0; a < kHalfPids; ++a)
                if (a < na) acc[a] = fma(w, sGo[wid][q][a0 + a], acc[a]);
        }
        __syncwarp();
    }
    if (cur >= 0) flush(cur);
}

// The sorted adjoint, pointwise (PW: bins by cell and flavour) or matrix
// form (bins by cell, up to kMaxSortedPids columns): per chunk of points, the
// coordinates (without a forward tape), the counting pass, the scan, the
// record pass and the accumulation.
template <bool PW>
int backward_sorted(pdfgpu_grid *g, int member, const Cols &cols, int npid, const int *pid, const double *x,
                    const double *q2, int64_t n, const double *tape, const double *dtape, const double *gout,
                    double *gx, double *gq, double *gval, cudaStream_t st)
{
    const int64_t nbins64 = (int64_t)g->d.nqc * g->d.nxc * (PW ? g->d.nflav : 1) * 4;
    if (nbins64 >= (int64_t)1 << 30) return fail(PDF_E_RANGE, "grid too large for the sorted adjoint");
    const int nbins = (int)nbins64;
    // the derivative tape's bin words (pointwise form): after the n derivative pairs
    const int *dbins = PW && dtape ? reinterpret_cast<const int *>(dtape + 2 * n) : nullptr;
    // points per round of count, records and accumulation ($PDFGPU_SORT_CHUNK
    // overrides the default; the scratch grows with it)
    int64_t chunk_max = kSortChunk;
    if (const char *e = getenv("PDFGPU_SORT_CHUNK")) {
        long long v = atoll(e);
        if (v > 0) chunk_max = std::min<int64_t>(v, (int64_t)1 << 30);
    }
    const int64_t chunk = std::min<int64_t>(n, chunk_max);
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t brec = al((size_t)chunk * 32);
    const size_t btape = tape ? 0 : brec;        // tape records made here when the caller has none
    const size_t bbins = al((size_t)(nbins + 1) * sizeof(int));
    const size_t need = brec + btape + 3 * bbins;
    if (g->bwd_scratch_bytes < need) {
        if (g->bwd_scratch) cudaFree(g->bwd_scratch);
        g->bwd_scratch = nullptr;
        g->bwd_scratch_bytes = 0;
        if (dev_malloc(&g->bwd_scratch, need, "sorted adjoint scratch")) return PDF_E_NOMEM;
        g->bwd_scratch_bytes = need;
    }
    char *base = (char *)g->bwd_scratch;
    double *rec = (double *)base;
    double *tape_s = tape ? nullptr : (double *)(base + brec);
    int *hist = (int *)(base + brec + btape);
    int *offs = (int *)(base + brec + btape + bbins);
    int *cursor = (int *)(base + brec + btape + 2 * bbins);
    const size_t hsmem = nbins <= kMaxSmemBins ? (size_t)nbins * sizeof(int) : 0;
    int rc = allow_dynamic_smem((const void *)k_bwd_count<PW>, hsmem);
    if (rc) return rc;
    for (int64_t i0 = 0; i0 < n; i0 += chunk) {
        const int m = (int)std::min(chunk, n - i0);
        const double *tv = tape ? tape + 4 * i0 : tape_s;     // the chunk's tape records
        if (!tape) {
            k_bwd_axes<<<wave_grid(g, (const void *)k_bwd_axes, kBlock, 0, m), kBlock, 0, st>>>(g->d, x, q2, i0, m,
                                                                                                tape_s);
            PDF_CUDA(cudaGetLastError());
        }
        PDF_CUDA(cudaMemsetAsync(hist, 0, (size_t)(nbins + 1) * sizeof(int), st));
        if (dbins) {   // the bins the forward pass wrote: 4 bytes per point to count
            rc = key_histogram(dbins + i0, m, hist, nbins, g->d.status, g->sm_count, st);
            if (rc) return rc;
        } else {
            const int gc =
                std::min(g->sm_count, std::max(1, (m + kCountIlp * kCountBlock - 1) / (kCountIlp * kCountBlock)));
            k_bwd_count<PW><<<gc, kCountBlock, hsmem, st>>>(g->d, pid, tv, i0, m, hist, nbins);
            PDF_CUDA(cudaGetLastError());
        }
        rc = exclusive_scan(hist, nbins, offs, cursor, st);
        if (rc) return rc;
        const int seg = PW ? kSegment : kSegmentM;
        const int64_t warps = (m + seg - 1) / seg;
        const int blocks = (int)((warps + kAccWarps - 1) / kAccWarps);
        if constexpr (PW) {
            auto krec = dtape ? k_bwd_rec<true> : k_bwd_rec<false>;
            krec<<<wave_grid(g, (const void *)krec, kBlock, 0, m), kBlock, 0, st>>>(
                g->d, member, pid, x, q2, i0, m, tv, dtape, dbins, gout, gx, gq, gval, nbins, cursor, rec);
            PDF_CUDA(cudaGetLastError());
            k_bwd_accum<<<blocks, kAccWarps * 32, 0, st>>>(g->d, rec, offs, nbins, gval);
        } else {
            k_bwd_rec_m<<<wave_grid(g, (const void *)k_bwd_rec_m, kBlock, 0, m), kBlock, 0, st>>>(
                g->d, cols, npid, member, x, q2, i0, m, tv, gout, gx, gq, gval, nbins, cursor, rec);
            PDF_CUDA(cudaGetLastError());
            if (npid >= 5)
                k_bwd_accum_mc<<<blocks, kAccWarps * 32, 0, st>>>(g->d, cols, npid, rec, offs, nbins, gout,
                                                                   gval);
            else
                k_bwd_accum_m<<<blocks, kAccWarps * 32, 0, st>>>(g->d, cols, npid, rec, offs, nbins, gout, gval);
        }
        PDF_CUDA(cudaGetLastError());
    }
    return PDF_OK;
}

template <bool PW, bool TAPE>
int launch(pdfgpu_grid *g, const Cols &cols, int npid, int member, const int *pid, const double *x,
           const double *q2, int64_t n, const double *tape, const double *dtape, const double *gout, double *gx,
           double *gq, double *gval, cudaStream_t s)
{
    if (gval && (PW || npid <= kMaxSortedPids))
        return backward_sorted<PW>(g, member, cols, npid, pid, x, q2, n, tape, dtape, gout, gx, gq, gval, s);
    size_t gbytes = (size_t)g->d.nrows * g->d.nx * g->d.nflav * sizeof(double);
    if constexpr (!PW) {
        if (gval && gbytes <= kSmemGradMax) {
            const void *kern = (const void *)k_bwd<PW, true, TAPE>;
            int rc = allow_dynamic_smem(kern, gbytes);
            if (rc) return rc;
            int grid = wave_grid(g, kern, kBlock, gbytes, n);
            k_bwd<PW, true, TAPE><<<grid, kBlock, gbytes, s>>>(g->d, cols, npid, member, pid, x, q2, n, tape,
                                                                dtape, gout, gx, gq, gval);
            PDF_CUDA(cudaGetLastError());
            return PDF_OK;
        }
    }
    {
        const void *kern = (const void *)k_bwd<PW, false, TAPE>;
        int grid = wave_grid(g, kern, kBlock, 0, n);
        k_bwd<PW, false, TAPE><<<grid, kBlock, 0, s>>>(g->d, cols, npid, member, pid, x, q2, n, tape, dtape,
                                                        gout, gx, gq, gval);
    }
    PDF_CUDA(cudaGetLastError());
    return PDF_OK;
}

int backward(pdfgpu_grid_t g, int32_t member, const int32_t *pids, int32_t n_pid, int32_t pointwise,
             const double *x, const double *q2, int64_t n, const double *tape, const double *dtape,
             const double *grad_out, double *grad_x, double *grad_q2, double *grad_values, cudaStream_t s)
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
    if (dtape && !pointwise) return fail(PDF_E_ARG, "a derivative tape serves the pointwise form only");
    if (dtape && !tape) return fail(PDF_E_ARG, "a derivative tape goes with the tape of the same forward call");
    if (dtape && (uintptr_t)dtape % 16) return fail(PDF_E_ARG, "derivative tape must be 16-byte aligned");
    Cols cols;
    memset(&cols, -1, sizeof(cols));
    if (!pointwise) {
        rc = resolve_cols(g, pids, n_pid, &cols);
        if (rc) return rc;
    }
    if (n == 0) return PDF_OK;
    if (!x || !q2 || !grad_out || !pids) return fail(PDF_E_ARG, "null array");
    if (pointwise)
        return tape ? launch<true, true>(g, cols, 1, member, pids, x, q2, n, tape, dtape, grad_out, grad_x,
                                         grad_q2, grad_values, s)
                    : launch<true, false>(g, cols, 1, member, pids, x, q2, n, nullptr, nullptr, grad_out, grad_x,
                                          grad_q2, grad_values, s);
    return tape ? launch<false, true>(g, cols, n_pid, member, nullptr, x, q2, n, tape, nullptr, grad_out, grad_x,
                                      grad_q2, grad_values, s)
                : launch<false, false>(g, cols, n_pid, member, nullptr, x, q2, n, nullptr, nullptr, grad_out,
                                       grad_x, grad_q2, grad_values, s);
}

}  // namespace

extern "C" int xfxQ2_backward(pdfgpu_grid_t g, int32_t member, const int32_t *pids, int32_t n_pid,
                              int32_t pointwise, const double *x, const double *q2, int64_t n,
                              const double *grad_out, double *grad_x, double *grad_q2,
                              double *grad_values, pdfgpu_stream_t stream)
{
    PDF_TRACE("xfxQ2_backward");
    return backward(g, member, pids, n_pid, pointwise, x, q2, n, nullptr, nullptr, grad_out, grad_x, grad_q2,
                    grad_values, (cudaStream_t)stream);
}

extern "C" int xfxQ2_backward_tape(pdfgpu_grid_t g, int32_t member, const int32_t *pids, int32_t n_pid,
                                   int32_t pointwise, const double *x, const double *q2, int64_t n,
                                   const double *tape, const double *dtape, const double *grad_out,
                                   double *grad_x, double *grad_q2, double *grad_values, pdfgpu_stream_t stream)
{
    PDF_TRACE("xfxQ2_backward_tape");
    if (!tape && n != 0) {
        clear_error();
        return fail(PDF_E_ARG, "null tape");
    }
    return backward(g, member, pids, n_pid, pointwise, x, q2, n, tape, dtape, grad_out, grad_x, grad_q2,
                    grad_values, (cudaStream_t)stream);
}
