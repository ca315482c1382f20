// Adaptive Monte Carlo integration of the parton luminosity (the VegasFlow
// use of the PDFs, PDFFlow Sec. 3.1, with the matrix element set to 1):
//
//   I = int_0^1 dr1 dr2 F(r1, r2),
//   ln tau = (1 - r1) ln tau_min,  y = (2 r2 - 1)(-ln tau / 2),
//   ln x1,2 = ln tau / 2 +- y,  ln Q^2 = ln tau + ln s,
//   F = (-ln tau_min)(-ln tau) sum_a xf_a(x1) xf_{-a}(x2),
//
// sampled through the VEGAS map (Lepage, J. Comput. Phys. 27 (1978) 192):
// per dimension n_bins bins with edges e_0 = 0 < ... < e_n = 1; a uniform v
// lands in bin i = floor(v n) at fraction d = v n - i and is mapped to
// r = e_i + d (e_{i+1} - e_i) with Jacobian n (e_{i+1} - e_i).  One kernel
// launch evaluates an iteration's points and accumulates sum w, the sum of
// (w - c)^2 about a shift c the caller passes (the previous iteration's
// estimate, so that the variance is a sum of small squares rather than the
// difference of two large sums) and the per-bin sums of w^2 that drive the
// next grid; the refinement itself is a few hundred flops on the host.
#include <math.h>

#include <algorithm>
#include <vector>

#include "pdf_internal.h"

using namespace pdfgpu;

namespace {

constexpr int kBlock = 256;
constexpr int kMaxBins = 1024;

template <bool CONT>
__global__ void __launch_bounds__(kBlock) k_vegas(GridDev g, Cols anti, int member, double ln_tau_min,
                                                  double ln_s, int n_bins, const double *__restrict__ edges,
                                                  const double *__restrict__ v, int64_t n, double shift,
                                                  double *__restrict__ partials, double *__restrict__ bins)
{
    extern __shared__ double sbin[];          // [2][n_bins] sums of w^2
    __shared__ signed char santi[PDF_MAX_PIDS];
    __shared__ double red[2][kBlock / 32];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < PDF_MAX_PIDS; ++k) santi[k] = anti.c[k];
    }
    for (int k = threadIdx.x; k < 2 * n_bins; k += blockDim.x) sbin[k] = 0.0;
    __syncthreads();
    const size_t cell_stride = (size_t)g.nflav * 16;
    const double *cm = g.coef + (size_t)member * g.nqc * g.nxc * cell_stride;
    const double nb = (double)n_bins;
    double s1 = 0.0, s2 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 vv = reinterpret_cast<const double2 *>(v)[i];
        double r[2], jac = 1.0;
        int bin[2];
#pragma unroll
        for (int d = 0; d < 2; ++d) {
            const double *e = edges + (size_t)d * (n_bins + 1);
            double vn = (d ? vv.y : vv.x) * nb;
            int b = min(max((int)vn, 0), n_bins - 1);    // uniforms outside [0, 1) stay in range
            double lo = __ldg(e + b), width = __ldg(e + b + 1) - lo;
            r[d] = fma(vn - (double)b, width, lo);
            jac *= nb * width;
            bin[d] = b;
        }
        const double ln_tau = (1.0 - r[0]) * ln_tau_min;
        const double h = 0.5 * ln_tau;
        const double y = (2.0 * r[1] - 1.0) * (-h);
        Axis Q = axis_w(g, ln_tau + ln_s);
        Axis X1 = axis_u(g, h + y);
        Axis X2 = axis_u(g, h - y);
        const double *c1 = cm + ((size_t)Q.cell * g.nxc + X1.cell) * cell_stride;
        const double *c2 = cm + ((size_t)Q.cell * g.nxc + X2.cell) * cell_stride;
        double lum = 0.0;
        for (int a = 0; a < g.nflav; ++a) {
            int b = santi[a];
            if (b < 0) continue;
            lum = fma(patch_any<CONT>(g, c1 + a * 16, X1, Q), patch_any<CONT>(g, c2 + b * 16, X2, Q), lum);
        }
        const double w = (-ln_tau_min) * (-ln_tau) * lum * jac;
        const double dw = w - shift;
        s1 += w;
        s2 = fma(dw, dw, s2);
        atomicAdd(&sbin[bin[0]], w * w);
        atomicAdd(&sbin[n_bins + bin[1]], w * w);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = s1;
        red[1][threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            t1 += red[0][k];
            t2 += red[1][k];
        }
        partials[2 * blockIdx.x] = t1;
        partials[2 * blockIdx.x + 1] = t2;
    }
    for (int k = threadIdx.x; k < 2 * n_bins; k += blockDim.x)
        if (dbits(sbin[k]) << 1) atomicAdd(&bins[k], sbin[k]);
}

// Fixed-order sum of the block partials into out[0..1].
__global__ void k_vegas_final(const double *__restrict__ partials, int nb, double *__restrict__ out)
{
    __shared__ double r1[256], r2[256];
    double t1 = 0.0, t2 = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        t1 += partials[2 * k];
        t2 += partials[2 * k + 1];
    }
    r1[threadIdx.x] = t1;
    r2[threadIdx.x] = t2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            r1[threadIdx.x] += r1[threadIdx.x + o];
            r2[threadIdx.x] += r2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = r1[0];
        out[1] = r2[0];
    }
}

constexpr int kMaxVegasDim = 16;

// The VEGAS map for an integrand the caller evaluates: one point per
// thread, every dimension through its own bin edges.
// TABLE: the block first tabulates each bin's lower edge, width and
// n_bins x width in shared memory (the same operations as computing them
// per point, so the same bits), which the points then read.
template <bool TABLE>
__global__ void __launch_bounds__(kBlock) k_vegas_map(int dim, int n_bins, const double *__restrict__ edges,
                                                      const double *__restrict__ v, int64_t n,
                                                      double *__restrict__ r, double *__restrict__ jac,
                                                      int *__restrict__ bins)
{
    extern __shared__ double tab[];          // [dim * n_bins][3]: lower edge, width, n_bins x width
    const double nb = (double)n_bins;
    if (TABLE) {
        for (int k = threadIdx.x; k < dim * n_bins; k += blockDim.x) {
            const int d = k / n_bins, b = k - d * n_bins;
            const double *e = edges + (size_t)d * (n_bins + 1);
            const double lo = e[b], width = e[b + 1] - lo;
            tab[3 * k] = lo;
            tab[3 * k + 1] = width;
            tab[3 * k + 2] = nb * width;
        }
        __syncthreads();
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double j = 1.0;
        for (int d = 0; d < dim; ++d) {
            double vn = v[i * dim + d] * nb;
            int b = min(max((int)vn, 0), n_bins - 1);    // uniforms outside [0, 1) stay in range
            if (TABLE) {
                const double *t = tab + 3 * (d * n_bins + b);
                r[i * dim + d] = fma(vn - (double)b, t[1], t[0]);
                j *= t[2];
            } else {
                const double *e = edges + (size_t)d * (n_bins + 1);
                double lo = __ldg(e + b), width = __ldg(e + b + 1) - lo;
                r[i * dim + d] = fma(vn - (double)b, width, lo);
                j *= nb * width;
            }
            bins[i * dim + d] = b;
        }
        jac[i] = j;
    }
}

// Sums of one iteration from the caller's weights: per block, sum w and
// sum (w - shift)^2 by shuffles and the per-bin sums of w^2 in shared
// memory, then one atomic per nonzero block total.
// PER_WARP: each warp adds into its own copy of the per-bin sums (fewer
// lanes of different warps waiting on one shared-memory address), the
// copies summed per block at the end.
template <bool PER_WARP>
__global__ void __launch_bounds__(kBlock) k_vegas_accumulate(int dim, int n_bins, const double *__restrict__ w,
                                                             const int *__restrict__ bins, int64_t n,
                                                             double shift, double *__restrict__ sums)
{
    extern __shared__ double sb_all[];       // [copies][dim][n_bins]
    __shared__ double red[2][kBlock / 32];
    const int nsb = dim * n_bins;
    const int copies = PER_WARP ? kBlock / 32 : 1;
    for (int k = threadIdx.x; k < copies * nsb; k += blockDim.x) sb_all[k] = 0.0;
    __syncthreads();
    double *sb = sb_all + (PER_WARP ? (threadIdx.x >> 5) * nsb : 0);
    double s1 = 0.0, s2 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double wi = w[i], w2 = wi * wi, dw = wi - shift;
        s1 += wi;
        s2 = fma(dw, dw, s2);
        for (int d = 0; d < dim; ++d) {
            int b = bins[i * dim + d];
            if (b >= 0 && b < n_bins) atomicAdd(&sb[d * n_bins + b], w2);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = s1;
        red[1][threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            t1 += red[0][k];
            t2 += red[1][k];
        }
        atomicAdd(&sums[0], t1);
        atomicAdd(&sums[1], t2);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nsb; k += blockDim.x) {
        double t = sb_all[k];
        for (int c = 1; c < copies; ++c) t += sb_all[c * nsb + k];
        if (dbits(t) << 1) atomicAdd(&sums[2 + k], t);
    }
}

int vegas_grid(int64_t n)
{
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + kBlock - 1) / kBlock, (int64_t)sms * 8));
}

}  // namespace

extern "C" int pdf_vegas_lumi_iteration(pdfgpu_grid_t g, int32_t member, double ln_tau_min, double ln_s,
                                        int32_t n_bins, const double *edges, const double *v, int64_t n,
                                        double shift, double *sums, pdfgpu_stream_t stream)
{
    PDF_TRACE("pdf_vegas_lumi_iteration");
    clear_error();
    int rc = check_grid(g, true);
    if (rc) return rc;
    if (member < 0 || member >= g->d.nmem) return fail(PDF_E_ARG, "member out of range");
    if (n_bins < 2 || n_bins > kMaxBins) return fail(PDF_E_RANGE, "n_bins must be in [2, 1024]");
    if (!(ln_tau_min < 0.0)) return fail(PDF_E_ARG, "ln_tau_min must be negative");
    if (!(shift > -INFINITY && shift < INFINITY)) return fail(PDF_E_ARG, "shift must be finite");
    if (n < 0) return fail(PDF_E_ARG, "negative n");
    if (!edges || !sums || (n > 0 && !v)) return fail(PDF_E_ARG, "null array");
    if (g->d.nflav > PDF_MAX_PIDS) return fail(PDF_E_RANGE, "too many flavours");
    Cols anti;
    memset(&anti, -1, sizeof(anti));
    for (int a = 0; a < g->d.nflav; ++a)
        for (int b = 0; b < g->d.nflav; ++b)
            if (g->pids[b] == -g->pids[a]) anti.c[a] = (signed char)b;
    cudaStream_t s = (cudaStream_t)stream;
    PDF_CUDA(cudaMemsetAsync(sums, 0, (2 + 2 * (size_t)n_bins) * sizeof(double), s));
    if (n == 0) return PDF_OK;
    size_t smem = 2 * (size_t)n_bins * sizeof(double);
    auto k = g->d.extrap == PDF_EXTRAP_CONTINUATION ? k_vegas<true> : k_vegas<false>;
    rc = allow_dynamic_smem((const void *)k, smem);
    if (rc) return rc;
    int grid = wave_grid(g, (const void *)k, kBlock, smem, n);
    if (g->partials_cap < 2 * grid) {
        if (g->partials) cudaFree(g->partials);
        g->partials = nullptr;
        g->partials_cap = 0;
        rc = dev_malloc((void **)&g->partials, (size_t)2 * grid * sizeof(double), "VEGAS partial sums");
        if (rc) return rc;
        g->partials_cap = 2 * grid;
    }
    k<<<grid, kBlock, smem, s>>>(g->d, anti, member, ln_tau_min, ln_s, n_bins, edges, v, n, shift,
                                 g->partials, sums + 2);
    PDF_CUDA(cudaGetLastError());
    k_vegas_final<<<1, 256, 0, s>>>(g->partials, grid, sums);
    PDF_CUDA(cudaGetLastError());
    return PDF_OK;
}

// Lepage's refinement of one dimension (host): smooth the per-bin sums of
// w^2 with their neighbours, damp them to r_i = ((1 - d_i)/ln(1/d_i))^alpha
// (d_i the normalised smoothed sums), and move the edges so that each new bin
// carries an equal share of sum r_i, the old bins' shares spread uniformly.
extern "C" int pdf_vegas_refine(const double *bin_w2, int32_t n_bins, double alpha, double *edges)
{
    PDF_TRACE("pdf_vegas_refine");
    clear_error();
    if (!bin_w2 || !edges) return fail(PDF_E_ARG, "null array");
    if (n_bins < 2 || n_bins > kMaxBins) return fail(PDF_E_RANGE, "n_bins must be in [2, 1024]");
    std::vector<double> sm(n_bins), damp(n_bins), old(edges, edges + n_bins + 1);
    sm[0] = 0.5 * (bin_w2[0] + bin_w2[1]);
    sm[n_bins - 1] = 0.5 * (bin_w2[n_bins - 2] + bin_w2[n_bins - 1]);
    for (int i = 1; i + 1 < n_bins; ++i) sm[i] = (bin_w2[i - 1] + bin_w2[i] + bin_w2[i + 1]) / 3.0;
    double total = 0.0;
    for (double v : sm) total += v;
    if (!(total > 0.0)) return PDF_OK;                 // nothing to learn from
    double dsum = 0.0;
    for (int i = 0; i < n_bins; ++i) {
        double di = sm[i] / total;
        damp[i] = (di > 0.0 && di < 1.0) ? pow((1.0 - di) / log(1.0 / di), alpha) : 0.0;
        dsum += damp[i];
    }
    if (!(dsum > 0.0)) return PDF_OK;
    const double share = dsum / n_bins;
    double acc = 0.0;
    int k = 0;
    for (int j = 1; j < n_bins; ++j) {
        const double target = j * share;
        while (acc + damp[k] <= target) acc += damp[k++];
        edges[j] = old[k] + (target - acc) / damp[k] * (old[k + 1] - old[k]);
    }
    edges[0] = 0.0;
    edges[n_bins] = 1.0;
    return PDF_OK;
}

extern "C" int pdf_vegas_map(int32_t dim, int32_t n_bins, const double *edges, const double *v, int64_t n,
                             double *r, double *jac, int32_t *bins, pdfgpu_stream_t stream)
{
    PDF_TRACE("pdf_vegas_map");
    clear_error();
    if (dim < 1 || dim > kMaxVegasDim) return fail(PDF_E_RANGE, "dim must be in [1, 16]");
    if (n_bins < 2 || n_bins > kMaxBins) return fail(PDF_E_RANGE, "n_bins must be in [2, 1024]");
    if (n < 0) return fail(PDF_E_ARG, "negative n");
    if (n == 0) return PDF_OK;
    if (!edges || !v || !r || !jac || !bins) return fail(PDF_E_ARG, "null array");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t tsmem = (size_t)dim * n_bins * 3 * sizeof(double);
    if (tsmem <= 48 * 1024)
        k_vegas_map<true><<<vegas_grid(n), kBlock, tsmem, s>>>(dim, n_bins, edges, v, n, r, jac, bins);
    else
        k_vegas_map<false><<<vegas_grid(n), kBlock, 0, s>>>(dim, n_bins, edges, v, n, r, jac, bins);
    PDF_CUDA(cudaGetLastError());
    return PDF_OK;
}

extern "C" int pdf_vegas_accumulate(int32_t dim, int32_t n_bins, const double *w, const int32_t *bins,
                                    int64_t n, double shift, double *sums, pdfgpu_stream_t stream)
{
    PDF_TRACE("pdf_vegas_accumulate");
    clear_error();
    if (dim < 1 || dim > kMaxVegasDim) return fail(PDF_E_RANGE, "dim must be in [1, 16]");
    if (n_bins < 2 || n_bins > kMaxBins) return fail(PDF_E_RANGE, "n_bins must be in [2, 1024]");
    if (n < 0) return fail(PDF_E_ARG, "negative n");
    if (!sums || (n > 0 && (!w || !bins))) return fail(PDF_E_ARG, "null array");
    if (!(shift > -INFINITY && shift < INFINITY)) return fail(PDF_E_ARG, "shift must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    PDF_CUDA(cudaMemsetAsync(sums, 0, (2 + (size_t)dim * n_bins) * sizeof(double), s));
    if (n == 0) return PDF_OK;
    const size_t one = (size_t)dim * n_bins * sizeof(double);
    const bool per_warp = one * (kBlock / 32) <= 48 * 1024;
    const void *kern = per_warp ? (const void *)k_vegas_accumulate<true> : (const void *)k_vegas_accumulate<false>;
    const size_t smem = per_warp ? one * (kBlock / 32) : one;
    int rc = allow_dynamic_smem(kern, smem);
    if (rc) return rc;
    if (per_warp)
        k_vegas_accumulate<true><<<vegas_grid(n), kBlock, smem, s>>>(dim, n_bins, w, bins, n, shift, sums);
    else
        k_vegas_accumulate<false><<<vegas_grid(n), kBlock, smem, s>>>(dim, n_bins, w, bins, n, shift, sums);
    PDF_CUDA(cudaGetLastError());
    return PDF_OK;
}
