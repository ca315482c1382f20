// Fused parton-luminosity workload (PDFFlow Sec. 3.1-3.2: the integrand maps
// random numbers to x1, x2 and the scale, calls xfxQ2 twice and multiplies
// the PDFs into the luminosity).  One thread per event does the kinematics
// in log variables, one Q search shared by both partons and by alpha_s, two
// x searches, 2 x F patch contractions and the flavour-paired product sum.
#include <math.h>

#include <algorithm>

#include "pdf_internal.h"

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

__global__ void __launch_bounds__(kBlock) k_lumi(GridDev g, Cols anti, int member,
                                                 const double *__restrict__ ln_tau,
                                                 const double *__restrict__ y,
                                                 const uint8_t *__restrict__ flags,
                                                 const double *__restrict__ ln_mu2,
                                                 const double *__restrict__ ln_x1, double ln_s,
                                                 int64_t n, double *__restrict__ lum,
                                                 double *__restrict__ as, double *__restrict__ partials)
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
        const double *c1 = cm + ((size_t)Q.cell * g.nxc + X1.cell) * cell_stride;
        const double *c2 = cm + ((size_t)Q.cell * g.nxc + X2.cell) * cell_stride;
        double s = 0.0;
        for (int a = 0; a < g.nflav; ++a) {
            int b = santi[a];
            if (b < 0) continue;
            double p1 = patch(c1 + a * 16, X1, Q);
            double p2 = patch(c2 + b * 16, X2, Q);
            s = fma(p1, p2, s);
        }
        if (E.bad) s = qnan();
        if (lum) lum[e] = s;
        acc += s;
        if (as) {
            const double2 *A = reinterpret_cast<const double2 *>(g.acoef + (size_t)Q.cell * 4);
            double2 a01 = __ldg(A), a23 = __ldg(A + 1);
            double v = fma(Q.b3, a23.y, fma(Q.b2, a23.x, fma(Q.t, a01.y, a01.x)));
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

// dL/dv for L = (1/n) sum_e sum_a f_a(x1) f_{-a}(x2), times `scale`:
//   d/dv[.][b] gets W(x1) f_{-b}(x2) + W(x2) f_{-b}(x1).
__global__ void __launch_bounds__(kBlock) k_lumi_bwd(GridDev g, Cols anti, int member,
                                                     const double *__restrict__ ln_tau,
                                                     const double *__restrict__ y,
                                                     const uint8_t *__restrict__ flags,
                                                     const double *__restrict__ ln_mu2,
                                                     const double *__restrict__ ln_x1, double ln_s,
                                                     int64_t n, double scale,
                                                     double *__restrict__ gval)
{
    __shared__ signed char santi[PDF_MAX_PIDS];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < PDF_MAX_PIDS; ++k) santi[k] = anti.c[k];
    }
    __syncthreads();
    const int F = g.nflav;
    const size_t cell_stride = (size_t)F * 16;
    const double *cm = g.coef + (size_t)member * g.nqc * g.nxc * cell_stride;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        Event E = event(e, ln_tau, y, flags, ln_mu2, ln_x1, ln_s);
        if (E.bad) continue;
        Axis Q = axis_w(g, E.w);
        Axis X1 = axis_u(g, E.u1);
        Axis X2 = axis_u(g, E.u2);
        const double *c1 = cm + ((size_t)Q.cell * g.nxc + X1.cell) * cell_stride;
        const double *c2 = cm + ((size_t)Q.cell * g.nxc + X2.cell) * cell_stride;
        double P1[kMaxLumiFlav], P2[kMaxLumiFlav];
#pragma unroll
        for (int a = 0; a < kMaxLumiFlav; ++a) {
            P1[a] = a < F ? patch(c1 + a * 16, X1, Q) : 0.0;
            P2[a] = a < F ? patch(c2 + a * 16, X2, Q) : 0.0;
        }
        double Wq[4], Wx1[4], Wx2[4];
        stencil_weights(g.mq + (size_t)Q.cell * 16, Q, Wq);
        stencil_weights(g.mx + (size_t)X1.cell * 16, X1, Wx1);
        stencil_weights(g.mx + (size_t)X2.cell * 16, X2, Wx2);
        int qmask = g.qmask[Q.cell];
        int r0 = g.qrow[Q.cell] - 1;
        int k1 = X1.cell - 1, k2 = X2.cell - 1;
#pragma unroll
        for (int b = 0; b < kMaxLumiFlav; ++b) {
            if (b >= F) break;
            int ab = santi[b];
            if (ab < 0) continue;
            double o2 = 0.0, o1 = 0.0;
#pragma unroll
            for (int a = 0; a < kMaxLumiFlav; ++a)
                if (a == ab) {
                    o2 = P2[a];
                    o1 = P1[a];
                }
            double G1 = scale * o2, G2 = scale * o1;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (!((qmask >> j) & 1)) continue;
                double *rowp = gval + ((size_t)(r0 + j) * g.nx) * F + b;
                double g1 = G1 * Wq[j], g2 = G2 * Wq[j];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    int kk = k1 + k;
                    if (kk >= 0 && kk < g.nx) atomicAdd(rowp + (size_t)kk * F, g1 * Wx1[k]);
                    kk = k2 + k;
                    if (kk >= 0 && kk < g.nx) atomicAdd(rowp + (size_t)kk * F, g2 * Wx2[k]);
                }
            }
        }
    }
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
                        int64_t n, double *lum, double *alphas, double *L, pdfgpu_stream_t stream)
{
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
    int grid = wave_grid(g, (const void *)k_lumi, kBlock, 0, n);
    if (g->partials_cap < grid) {
        if (g->partials) cudaFree(g->partials);
        g->partials = nullptr;
        g->partials_cap = 0;
        PDF_CUDA(cudaMalloc(&g->partials, (size_t)grid * sizeof(double)));
        g->partials_cap = grid;
    }
    k_lumi<<<grid, kBlock, 0, s>>>(g->d, anti, member, ln_tau, y, flags, ln_mu2, ln_x1, ln_s, n, lum,
                                   alphas, g->partials);
    PDF_CUDA(cudaGetLastError());
    k_lumi_final<<<1, 256, 0, s>>>(g->partials, grid, 1.0 / (double)n, L);
    PDF_CUDA(cudaGetLastError());
    return PDF_OK;
}

extern "C" int pdf_lumi_backward(pdfgpu_grid_t g, int32_t member, const double *ln_tau, const double *y,
                                 const uint8_t *flags, const double *ln_mu2, const double *ln_x1,
                                 double ln_s, int64_t n, double dL, double *grad_values,
                                 pdfgpu_stream_t stream)
{
    clear_error();
    Cols anti;
    int rc = lumi_common(g, member, ln_tau, y, n, &anti);
    if (rc) return rc;
    if (!grad_values) return fail(PDF_E_ARG, "null grad_values");
    if (n == 0) return PDF_OK;
    int grid = wave_grid(g, (const void *)k_lumi_bwd, kBlock, 0, n);
    k_lumi_bwd<<<grid, kBlock, 0, (cudaStream_t)stream>>>(g->d, anti, member, ln_tau, y, flags, ln_mu2,
                                                          ln_x1, ln_s, n, dL / (double)n, grad_values);
    PDF_CUDA(cudaGetLastError());
    return PDF_OK;
}
