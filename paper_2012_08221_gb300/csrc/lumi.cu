// Fused parton-luminosity workload (PDFFlow Sec. 3.1-3.2: the integrand maps
// random numbers to x1, x2 and the scale, calls xfxQ2 twice and multiplies
// the PDFs into the luminosity).  One thread per event does the kinematics
// in log variables, one Q search shared by both partons and by alpha_s, two
// x searches, 2 x F patch contractions and the flavour-paired product sum.
#include <math.h>

#include <algorithm>

#include "pdf_internal.h"
#include "sort_acc.cuh"

using namespace pdfgpu;

namespace {

constexpr int kBlock = 256;
constexpr int kMaxLumiFlav = 16;

__device__ __forceinline__ double qnan() { return __longlong_as_double(0x7FF8000000000000ll); }

struct Event {
    double u1, u2, w;
    bool bad;
};

// ln x1 = ln(tau)/2 + y, ln x2 = ln(tau)/2 - y, ln Q^2 = ln tau + ln s, with
// the overrides of the flags; bad if ln x > 0 or any value is not finite.
__device__ __forceinline__ Event event(int64_t e, const double *ln_tau, const double *y,
                                       const uint8_t *flags, const double *ln_mu2,
                                       const double *ln_x1, double ln_s)
{
    Event E;
    double lt = ln_tau[e], yy = y[e];
    unsigned f = flags ? flags[e] : 0u;
    double h = 0.5 * lt;
    E.u1 = h + yy;
    E.u2 = h - yy;
    E.w = lt + ln_s;
    if (f & 1u) E.w = ln_mu2[e];
    if (f & 2u) E.u1 = ln_x1[e];
    auto finite = [](double v) { return (dbits(v) & 0x7FF0000000000000ull) != 0x7FF0000000000000ull; };
    E.bad = !(finite(E.u1) && finite(E.u2) && finite(E.w)) || dkey(E.u1) > 0 || dkey(E.u2) > 0;
    if (E.bad) {
        E.u1 = -1.0;
        E.u2 = -1.0;
        E.w = 4.0;
    }
    return E;
}

// At most 64 registers (4 CTAs per SM): with the 32-byte coefficient loads
// the unbounded build takes 80 and runs 1 % slower at 3 CTAs per SM.
template <bool SAVE, bool CONT>
__global__ void __launch_bounds__(kBlock, 4) k_lumi(GridDev g, Cols anti, int member,
                                                    const double *__restrict__ ln_tau,
                                                    const double *__restrict__ y,
                                                    const uint8_t *__restrict__ flags,
                                                    const double *__restrict__ ln_mu2,
                                                    const double *__restrict__ ln_x1, double ln_s,
                                                    int64_t n, double *__restrict__ lum,
                                                    double *__restrict__ as, double *__restrict__ partials,
                                                    double *__restrict__ save_p)
{
    __shared__ signed char santi[PDF_MAX_PIDS];
    __shared__ double red[kBlock / 32];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < PDF_MAX_PIDS; ++k) santi[k] = anti.c[k];
    }
    __syncthreads();
    const size_t cell_stride = (size_t)g.nflav * 16;
    const double *cm = g.coef + (size_t)member * g.nqc * g.nxc * cell_stride;
    double acc = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        Event E = event(e, ln_tau, y, flags, ln_mu2, ln_x1, ln_s);
        flag_status(g, E.bad);
        Axis Q = axis_w(g, E.w);
        Axis X1 = axis_u(g, E.u1);
        Axis X2 = axis_u(g, E.u2);
        const bool oor = !E.bad && (out_of_range(g, X1, Q) || out_of_range(g, X2, Q));
        flag_status(g, oor, PDF_S_RANGE);
        E.bad |= oor;
        const double *c1 = cm + ((size_t)Q.cell * g.nxc + X1.cell) * cell_stride;
        const double *c2 = cm + ((size_t)Q.cell * g.nxc + X2.cell) * cell_stride;
        double s = 0.0;
        for (int a = 0; a < g.nflav; ++a) {
            int b = santi[a];
            if (b < 0) continue;
            double p1 = patch_any<CONT>(g, c1 + a * 16, X1, Q);
            double p2 = patch_any<CONT>(g, c2 + b * 16, X2, Q);
            s = fma(p1, p2, s);
            if (SAVE) {
                // the partner factors the adjoint needs: [event][parton][flavour]
                double *pe = save_p + (size_t)e * 2 * g.nflav;
                pe[a] = p1;
                pe[g.nflav + b] = p2;
            }
        }
        if (E.bad) s = qnan();
        if (lum) lum[e] = s;
        acc += s;
        if (as) {
            double v = alphas_any(g, ld4(g.acoef + (size_t)Q.cell * 4), Q);
            as[e] = E.bad ? qnan() : v;
        }
    }
    // fixed-order block reduction of the per-thread sums
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        partials[blockIdx.x] = t;
    }
}

__global__ void k_lumi_final(const double *__restrict__ partials, int nb, double inv_n, double *L)
{
    __shared__ double red[256];
    double t = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) t += partials[k];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *L = red[0] * inv_n;
}

// ---------------------------------------------------------------- adjoint
//
// dL/dv for L = (1/n) sum_e sum_a f_a(x1) f_{-a}(x2), times dL:
//   dL/dv[row][knot][b] = scale sum over partons p of all events of
//                         Wq_j(p) Wx_i(p) f_{-b}(other parton)
// over each parton's 4x4 stencil.  Instead of 16 x F global atomics per
// parton, partons are grouped by grid cell and accumulated in registers:
//   1. k_lumi_rec: per event the two partons' F values (the partner factors)
//      and, per parton, its bin key, local coordinates and range flags;
//   2. key_histogram: a histogram of the keys; exclusive_scan: bin offsets;
//      k_scatter_tiled: parton ids in bin order;
//   3. k_lumi_accum: each half-warp walks half of a warp's run of sorted
//      partons in batches of 16 (one parton per lane stages its 16 basis
//      products and its partner factors, already paired, in shared
//      memory); lane s of a half owns slot s of the current bin for all F
//      flavours and adds F FMAs per parton; when the bin changes the
//      accumulators go to the gradient with one atomic per output.
// A bin is one cell and one kind: a parton inside the knot range on both
// axes accumulates in the monomial basis of the patch, bq_n bx_m in the
// near-knot coordinate of each axis (t, or 1 - t in the upper half of the
// cell; kinds 0-3 by the two halves), and the bin maps its accumulators back
// to the stencil values once per run (as the grid gradients of the x*f
// adjoint do); a parton outside the range on either axis (kind 4) takes its
// exact stencil weights, whose products are accumulated directly.
// Events are processed in chunks so that the scratch stays bounded.

constexpr int kAccWarps = 4;
constexpr int kSegment = 1024;        // partons per warp
constexpr int kKinds = 5;             // bin kinds per cell: 4 half pairs inside, 1 outside
constexpr int kScatterSmemBins = 50 * 1024;  // bin counters of the scatter in shared memory
constexpr int kScatterBlock = 1024;         // (one 1024-thread block per SM)

__device__ __forceinline__ int parton_kind(const Axis &X, const Axis &Q)
{
    if (!(X.in && Q.in)) return 4;
    return (upper_half(X.t) ? 1 : 0) | (upper_half(Q.t) ? 2 : 0);
}

template <bool PATCHES>
__global__ void __launch_bounds__(kBlock) k_lumi_rec(GridDev g, int member,
                                                     const double *__restrict__ ln_tau,
                                                     const double *__restrict__ y,
                                                     const uint8_t *__restrict__ flags,
                                                     const double *__restrict__ ln_mu2,
                                                     const double *__restrict__ ln_x1, double ln_s,
                                                     int64_t e0, int m, int *__restrict__ key,
                                                     double *__restrict__ tx, double *__restrict__ tq,
                                                     uint8_t *__restrict__ fin, double *__restrict__ P)
{
    const int F = g.nflav;
    const size_t cell_stride = (size_t)F * 16;
    const double *cm = g.coef + (size_t)member * g.nqc * g.nxc * cell_stride;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        Event E = event(e0 + i, ln_tau, y, flags, ln_mu2, ln_x1, ln_s);
        if (E.bad) {
            key[2 * i] = -1;
            key[2 * i + 1] = -1;
            continue;
        }
        Axis Q = axis_w(g, E.w);
        Axis X1 = axis_u(g, E.u1);
        Axis X2 = axis_u(g, E.u2);
        if (out_of_range(g, X1, Q) || out_of_range(g, X2, Q)) {
            key[2 * i] = -1;
            key[2 * i + 1] = -1;
            continue;
        }
        const double *c1 = cm + ((size_t)Q.cell * g.nxc + X1.cell) * cell_stride;
        const double *c2 = cm + ((size_t)Q.cell * g.nxc + X2.cell) * cell_stride;
        if (PATCHES) {
            double *p1 = P + (size_t)i * 2 * F;
            double *p2 = p1 + F;
            for (int a = 0; a < F; ++a) {
                p1[a] = patch(c1 + a * 16, X1, Q);
                p2[a] = patch(c2 + a * 16, X2, Q);
            }
        }
        const int cq = Q.cell * g.nxc;
        key[2 * i] = (cq + X1.cell) * kKinds + parton_kind(X1, Q);
        key[2 * i + 1] = (cq + X2.cell) * kKinds + parton_kind(X2, Q);
        tx[2 * i] = X1.t;
        tx[2 * i + 1] = X2.t;
        tq[i] = Q.t;
        fin[2 * i] = (uint8_t)(Q.in | (X1.in << 1));
        fin[2 * i + 1] = (uint8_t)(Q.in | (X2.in << 1));
    }
}

__global__ void k_scatter(const int *__restrict__ key, int nrec, int *__restrict__ cursor,
                          int *__restrict__ perm)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrec; r += gridDim.x * blockDim.x) {
        int k = key[r];
        if (k >= 0) perm[atomicAdd(&cursor[k], 1)] = r;
    }
}

// The same scatter with one global atomic per (tile, bin) instead of one
// per record: a block counts its tile's records per bin in shared memory,
// reserves a range for each bin present, then places the records in their
// ranges with shared-memory atomics.  The order inside a bin is free (the
// accumulation sums the bin's records).  nbins <= kScatterSmemBins; one block
// of kScatterBlock threads per SM.
constexpr int kScatterTile = 32768;

__global__ void __launch_bounds__(kScatterBlock) k_scatter_tiled(const int *__restrict__ key, int nrec, int nbins,
                                                          int *__restrict__ cursor, int *__restrict__ perm)
{
    extern __shared__ int sc[];
    const int r0 = blockIdx.x * kScatterTile, r1 = min(nrec, r0 + kScatterTile);
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) sc[b] = 0;
    __syncthreads();
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        const int k = key[r];
        if (k >= 0) atomicAdd(&sc[k], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        const int c = sc[b];
        if (c) sc[b] = atomicAdd(&cursor[b], c);
    }
    __syncthreads();
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        const int k = key[r];
        if (k >= 0) perm[atomicAdd(&sc[k], 1)] = r;
    }
}

// Rebuild an axis from its stored local coordinate (t and range flag).  The
// stored t is the effective one (0 or 1 when frozen at an edge), for which
// the outside basis (1, t, t, t) and weights (1 - t, t) are the right ones.
__device__ __forceinline__ Axis axis_from(int cell, double t, bool in)
{
    Axis A;
    A.cell = cell;
    A.in = in;
    A.below = false;
    make_basis(A, t, PDF_EXTRAP_LINEAR);
    return A;
}

template <int kF>
__global__ void __launch_bounds__(kAccWarps * 32) k_lumi_accum(GridDev g, Cols anti,
                                                               const int *__restrict__ perm,
                                                               const int *__restrict__ offs, int nbins,
                                                               const int *__restrict__ key,
                                                               const double *__restrict__ tx,
                                                               const double *__restrict__ tq,
                                                               const uint8_t *__restrict__ fin,
                                                               const double *__restrict__ P, double scale,
                                                               double *__restrict__ gval)
{
    // per warp: 32 staged partons (16 per half-warp), their 16 basis products
    // (or stencil weights) and their partner factors already paired: sP[.][b]
    // is the partner parton's value of the flavour paired with b (0 if none)
    __shared__ double sW[kAccWarps][32][17];
    __shared__ double sP[kAccWarps][32][kF + 1];
    __shared__ int sK[kAccWarps][32];
    __shared__ double sG[kAccWarps][32];                      // map-back slots, 16 per half
    __shared__ signed char santi[PDF_MAX_PIDS];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < PDF_MAX_PIDS; ++k) santi[k] = anti.c[k];
    }
    __syncthreads();
    const int F = g.nflav;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nvalid = offs[nbins];
    const int64_t wbeg = ((int64_t)blockIdx.x * kAccWarps + wid) * kSegment;
    if (wbeg >= nvalid) return;
    const int wend = (int)min((int64_t)nvalid, wbeg + kSegment);
    // the two half-warps walk the two halves of the warp's segment; a lane
    // owns slot s = 4 j + i of its half's current bin for every flavour
    const int h = lane >> 4, s = lane & 15, j = s >> 2, i = s & 3;
    const unsigned hmask = 0xFFFFu << (16 * h);
    const int half = (wend - (int)wbeg + 1) / 2;
    const int beg = (int)wbeg + h * half;
    const int end = h ? wend : (int)wbeg + half;
    const int row0 = h * 16;
    double acc[kF];
#pragma unroll
    for (int b = 0; b < kF; ++b) acc[b] = 0.0;
    int cur = -1;
    auto flush = [&](int bin) {
        const int cell = bin / kKinds, kind = bin - cell * kKinds;
        const int qc = cell / g.nxc, xc = cell - qc * g.nxc;
        int row = g.qrow[qc] - 1 + j;
        const int col = xc - 1 + i;
        const bool ok = ((g.qmask[qc] >> j) & 1) && col >= 0 && col < g.nx;
        if (ok) row = checked_index(g.status, row, g.nrows);
        const double *Mq = ((kind & 2) ? g.mqs : g.mq) + (size_t)qc * 16;
        const double *Mx = ((kind & 1) ? g.mxs : g.mx) + (size_t)xc * 16;
#pragma unroll
        for (int b = 0; b < kF; ++b) {
            if (kF == kMaxLumiFlav && b >= F) break;       // the same for the whole warp
            double v = acc[b];
            if (kind < 4) v = map_back(v, &sG[wid][row0], Mq, Mx, j, i, hmask);   // the same for the half
            if (ok && santi[b] >= 0 && (dbits(v) << 1))
                atomicAdd(gval + ((size_t)row * g.nx + col) * F + b, scale * v);
            acc[b] = 0.0;
        }
    };
    const int steps = (half + 15) / 16;
    for (int step = 0; step < steps; ++step) {
        const int p = beg + step * 16;
        // one parton per lane: basis products (or stencil weights) and the
        // paired partner factors
        int r = p + s;
        int kr = -1;
        if (r < end) {
            int rec = perm[r];
            int e = rec >> 1, side = rec & 1;
            kr = checked_index(g.status, key[rec], nbins);
            const int cell = kr / kKinds, kind = kr - cell * kKinds;
            const int qc = cell / g.nxc, xc = cell - qc * g.nxc;
            double *w = sW[wid][row0 + s];
            if (kind < 4) {
                // the near-knot coordinates of the bin's halves and the
                // products of their powers
                const double a = (kind & 1) ? 1.0 - tx[rec] : tx[rec];
                const double c = (kind & 2) ? 1.0 - tq[e] : tq[e];
                const double a2 = a * a, c2 = c * c;
                const double bx[4] = {1.0, a, a2, a2 * a};
                const double bq[4] = {1.0, c, c2, c2 * c};
#pragma unroll
                for (int m = 0; m < 4; ++m) w[m] = bx[m];
#pragma unroll
                for (int n = 1; n < 4; ++n) {
                    w[4 * n] = bq[n];
#pragma unroll
                    for (int m = 1; m < 4; ++m) w[4 * n + m] = bq[n] * bx[m];
                }
            } else {
                uint8_t f = fin[rec];
                Axis Q = axis_from(qc, tq[e], f & 1);
                Axis X = axis_from(xc, tx[rec], (f >> 1) & 1);
                double Wq[4], Wx[4];
                stencil_weights(g.mq + (size_t)qc * 16, g.mqs + (size_t)qc * 16, Q, Wq);
                stencil_weights(g.mx + (size_t)xc * 16, g.mxs + (size_t)xc * 16, X, Wx);
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
#pragma unroll
                    for (int ii = 0; ii < 4; ++ii) w[jj * 4 + ii] = Wq[jj] * Wx[ii];
            }
            const double *po = P + (size_t)e * 2 * F + (size_t)(1 - side) * F;
            for (int b = 0; b < F; ++b) {
                int a = santi[b];
                sP[wid][row0 + s][b] = a >= 0 ? po[a] : 0.0;
            }
        }
        sK[wid][row0 + s] = kr;
        __syncwarp();
        const int nb = min(16, end - p);
        for (int q = 0; q < 16; ++q) {
            if (q < nb) {
                int kq = sK[wid][row0 + q];
                if (kq != cur) {
                    if (cur >= 0) flush(cur);
                    cur = kq;
                }
                double wv = sW[wid][row0 + q][s];
#pragma unroll
                for (int b = 0; b < kF; ++b)
                    if (kF == kMaxLumiFlav ? b < F : true) acc[b] = fma(wv, sP[wid][row0 + q][b], acc[b]);
            }
        }
        __syncwarp();
    }
    if (cur >= 0) flush(cur);
}

int lumi_common(pdfgpu_grid *g, int32_t member, const double *ln_tau, const double *y,
                int64_t n, Cols *anti)
{
    int rc = check_grid(g, true);
    if (rc) return rc;
    if (n < 0) return fail(PDF_E_ARG, "negative n");
    if (member < 0 || member >= g->d.nmem) return fail(PDF_E_ARG, "member out of range");
    if (g->d.nflav > kMaxLumiFlav) return fail(PDF_E_RANGE, "luminosity supports at most 16 flavours");
    if (n > 0 && (!ln_tau || !y)) return fail(PDF_E_ARG, "null array");
    memset(anti, -1, sizeof(*anti));
    for (int a = 0; a < g->d.nflav; ++a) {
        int p = -g->pids[a];
        for (int b = 0; b < g->d.nflav; ++b)
            if (g->pids[b] == p) anti->c[a] = (signed char)b;
    }
    return PDF_OK;
}

}  // namespace

extern "C" int pdf_lumi(pdfgpu_grid_t g, int32_t member, const double *ln_tau, const double *y,
                        const uint8_t *flags, const double *ln_mu2, const double *ln_x1, double ln_s,
                        int64_t n, double *lum, double *alphas, double *L, double *save_p,
                        pdfgpu_stream_t stream)
{
    PDF_TRACE("pdf_lumi");
    clear_error();
    Cols anti;
    int rc = lumi_common(g, member, ln_tau, y, n, &anti);
    if (rc) return rc;
    if (!L) return fail(PDF_E_ARG, "null L");
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        PDF_CUDA(cudaMemsetAsync(L, 0, sizeof(double), s));
        return PDF_OK;
    }
    if (alphas && !g->has_alphas) alphas = nullptr;
    using Kern = void (*)(GridDev, Cols, int, const double *, const double *, const uint8_t *, const double *,
                          const double *, double, int64_t, double *, double *, double *, double *);
    const bool cont = g->d.extrap == PDF_EXTRAP_CONTINUATION;
    Kern k = save_p ? (cont ? k_lumi<true, true> : k_lumi<true, false>)
                    : (cont ? k_lumi<false, true> : k_lumi<false, false>);
    int grid = wave_grid(g, (const void *)k, kBlock, 0, n);
    if (g->partials_cap < grid) {
        if (g->partials) cudaFree(g->partials);
        g->partials = nullptr;
        g->partials_cap = 0;
        rc = dev_malloc((void **)&g->partials, (size_t)grid * sizeof(double), "luminosity partial sums");
        if (rc) return rc;
        g->partials_cap = grid;
    }
    k<<<grid, kBlock, 0, s>>>(g->d, anti, member, ln_tau, y, flags, ln_mu2, ln_x1, ln_s, n, lum, alphas,
                              g->partials, save_p);
    PDF_CUDA(cudaGetLastError());
    k_lumi_final<<<1, 256, 0, s>>>(g->partials, grid, 1.0 / (double)n, L);
    PDF_CUDA(cudaGetLastError());
    return PDF_OK;
}

extern "C" int pdf_lumi_backward(pdfgpu_grid_t g, int32_t member, const double *ln_tau, const double *y,
                                 const uint8_t *flags, const double *ln_mu2, const double *ln_x1,
                                 double ln_s, int64_t n, double dL, const double *saved_p,
                                 double *grad_values, pdfgpu_stream_t stream)
{
    PDF_TRACE("pdf_lumi_backward");
    clear_error();
    Cols anti;
    int rc = lumi_common(g, member, ln_tau, y, n, &anti);
    if (rc) return rc;
    if (g->d.extrap == PDF_EXTRAP_CONTINUATION)
        return fail(PDF_E_ARG, "the adjoint needs linear, freeze or error extrapolation (continuation is not linear "
                               "in the grid values)");
    if (!grad_values) return fail(PDF_E_ARG, "null grad_values");
    if (n == 0) return PDF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int F = g->d.nflav;
    const int64_t nbins64 = (int64_t)g->d.nqc * g->d.nxc * kKinds;
    if (nbins64 >= (int64_t)1 << 30) return fail(PDF_E_RANGE, "grid too large for the luminosity adjoint");
    const int nbins = (int)nbins64;
    const int64_t chunk = std::min<int64_t>(n, (int64_t)1 << 23);
    // scratch layout per chunk of m events
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t bP = saved_p ? 0 : al((size_t)chunk * 2 * F * sizeof(double));
    const size_t btq = al((size_t)chunk * sizeof(double));
    const size_t btx = al((size_t)chunk * 2 * sizeof(double));
    const size_t bkey = al((size_t)chunk * 2 * sizeof(int));
    const size_t bfin = al((size_t)chunk * 2);
    const size_t bperm = bkey;
    const size_t bbins = al((size_t)(nbins + 1) * sizeof(int));
    const size_t need = bP + btq + btx + bkey + bfin + bperm + 3 * bbins;
    if (g->lumi_scratch_bytes < need) {
        if (g->lumi_scratch) cudaFree(g->lumi_scratch);
        g->lumi_scratch = nullptr;
        g->lumi_scratch_bytes = 0;
        if (dev_malloc(&g->lumi_scratch, need, "luminosity adjoint scratch")) return PDF_E_NOMEM;
        g->lumi_scratch_bytes = need;
    }
    char *base = (char *)g->lumi_scratch;
    double *P = saved_p ? nullptr : (double *)base;
    double *tq = (double *)(base += bP);
    double *tx = (double *)(base += btq);
    int *key = (int *)(base += btx);
    uint8_t *fin = (uint8_t *)(base += bkey);
    int *perm = (int *)(base += bfin);
    int *hist = (int *)(base += bperm);
    int *offs = (int *)(base += bbins);
    int *cursor = (int *)(base += bbins);
    const double scale = dL / (double)n;
    const size_t hsmem = nbins <= kScatterSmemBins ? (size_t)nbins * sizeof(int) : 0;
    const void *krec = saved_p ? (const void *)k_lumi_rec<false> : (const void *)k_lumi_rec<true>;
    rc = allow_dynamic_smem((const void *)k_scatter_tiled, hsmem);
    if (rc) return rc;
    for (int64_t e0 = 0; e0 < n; e0 += chunk) {
        const int m = (int)std::min(chunk, n - e0);
        PDF_CUDA(cudaMemsetAsync(hist, 0, (size_t)(nbins + 1) * sizeof(int), st));
        int grid = wave_grid(g, krec, kBlock, 0, m);
        const double *Pc = saved_p ? saved_p + (size_t)e0 * 2 * F : P;
        if (saved_p)
            k_lumi_rec<false><<<grid, kBlock, 0, st>>>(g->d, member, ln_tau, y, flags, ln_mu2, ln_x1, ln_s,
                                                       e0, m, key, tx, tq, fin, nullptr);
        else
            k_lumi_rec<true><<<grid, kBlock, 0, st>>>(g->d, member, ln_tau, y, flags, ln_mu2, ln_x1, ln_s,
                                                      e0, m, key, tx, tq, fin, P);
        PDF_CUDA(cudaGetLastError());
        rc = key_histogram(key, 2 * (int64_t)m, hist, nbins, g->d.status, g->sm_count, st);
        if (rc) return rc;
        rc = exclusive_scan(hist, nbins, offs, cursor, st);
        if (rc) return rc;
        if (hsmem) {
            const int tiles = (int)((2 * (int64_t)m + kScatterTile - 1) / kScatterTile);
            k_scatter_tiled<<<tiles, kScatterBlock, hsmem, st>>>(key, 2 * m, nbins, cursor, perm);
        } else {
            int gs = wave_grid(g, (const void *)k_scatter, kBlock, 0, 2 * (int64_t)m);
            k_scatter<<<gs, kBlock, 0, st>>>(key, 2 * m, cursor, perm);
        }
        PDF_CUDA(cudaGetLastError());
        int64_t warps = (2 * (int64_t)m + kSegment - 1) / kSegment;
        int blocks = (int)((warps + kAccWarps - 1) / kAccWarps);
        if (F == 13)
            k_lumi_accum<13><<<blocks, kAccWarps * 32, 0, st>>>(g->d, anti, perm, offs, nbins, key, tx, tq, fin,
                                                                Pc, scale, grad_values);
        else if (F == 11)
            k_lumi_accum<11><<<blocks, kAccWarps * 32, 0, st>>>(g->d, anti, perm, offs, nbins, key, tx, tq, fin,
                                                                Pc, scale, grad_values);
        else
            k_lumi_accum<kMaxLumiFlav><<<blocks, kAccWarps * 32, 0, st>>>(g->d, anti, perm, offs, nbins, key, tx,
                                                                          tq, fin, Pc, scale, grad_values);
        PDF_CUDA(cudaGetLastError());
    }
    return PDF_OK;
}
