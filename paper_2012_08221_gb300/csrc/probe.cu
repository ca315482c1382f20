// FP64 peak probe: the denominator of the FP64-pipe roofline.
//
// Eight independent fused multiply-add chains per thread, one full wave of
// CTAs on every SM, timed with CUDA events after a warm-up launch.
#include "pdf_internal.h"

namespace {

__global__ void k_dfma_chains(double *out, int iters, double b, double c)
{
    double a0 = threadIdx.x * 1e-3, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
    double a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
    for (int it = 0; it < iters; ++it) {
        a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
        a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

}  // namespace

extern "C" int pdf_probe_fp64_peak(double *flops)
{
    PDF_TRACE("pdf_probe_fp64_peak");
    pdfgpu::clear_error();
    if (!flops) return pdfgpu::fail(PDF_E_ARG, "null output");
    int dev = 0, sms = 0;
    PDF_CUDA(cudaGetDevice(&dev));
    PDF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int block = 256, per_sm = 4, iters = 4096;
    const int blocks = sms * per_sm;
    double *buf = nullptr;
    int rc = pdfgpu::dev_malloc((void **)&buf, (size_t)blocks * block * sizeof(double), "probe buffer");
    if (rc) return rc;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_dfma_chains<<<blocks, block>>>(buf, 64, 0.999, 1e-3);
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0);
        k_dfma_chains<<<blocks, block>>>(buf, iters, 0.999, 1e-3);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (err != cudaSuccess) return pdfgpu::cuda_fail(err, "probe kernel");
    *flops = 2.0 * 8.0 * (double)iters * blocks * block / (best * 1e-3);
    return PDF_OK;
}

// ------------------------------------------------------------ FP64 MMA probe
//
// Throughput of the FP64 tensor instructions (mma.sync with f64 operands, the
// only FP64 matrix path of sm_103a: tcgen05 has no f64 kind) against the DFMA
// chains above.  Each warp runs kChains independent accumulator chains of one
// shape; a warp-wide mma of shape MxNxK counts 2 M N K flops.

namespace {

constexpr int kChains = 8;

template <int SHAPE>
struct MmaShape;
template <>
struct MmaShape<0> {   // m8n8k4: A 1, B 1, C/D 2 doubles per thread
    static constexpr int M = 8, N = 8, K = 4, NA = 1, NB = 1, NC = 2;
};
template <>
struct MmaShape<1> {   // m16n8k4: A 2, B 1, C/D 4
    static constexpr int M = 16, N = 8, K = 4, NA = 2, NB = 1, NC = 4;
};
template <>
struct MmaShape<2> {   // m16n8k8: A 4, B 2, C/D 4
    static constexpr int M = 16, N = 8, K = 8, NA = 4, NB = 2, NC = 4;
};
template <>
struct MmaShape<3> {   // m16n8k16: A 8, B 4, C/D 4
    static constexpr int M = 16, N = 8, K = 16, NA = 8, NB = 4, NC = 4;
};

template <int SHAPE>
__device__ __forceinline__ void mma_f64(double *d, const double *a, const double *b);

template <>
__device__ __forceinline__ void mma_f64<0>(double *d, const double *a, const double *b)
{
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                 : "+d"(d[0]), "+d"(d[1])
                 : "d"(a[0]), "d"(b[0]));
}
template <>
__device__ __forceinline__ void mma_f64<1>(double *d, const double *a, const double *b)
{
    asm volatile("mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0, %1, %2, %3}, {%4, %5}, {%6}, "
                 "{%0, %1, %2, %3};"
                 : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
                 : "d"(a[0]), "d"(a[1]), "d"(b[0]));
}
template <>
__device__ __forceinline__ void mma_f64<2>(double *d, const double *a, const double *b)
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f64.f64.f64.f64 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                 "{%8, %9}, {%0, %1, %2, %3};"
                 : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
                 : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(b[0]), "d"(b[1]));
}
template <>
__device__ __forceinline__ void mma_f64<3>(double *d, const double *a, const double *b)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0, %1, %2, %3}, "
                 "{%4, %5, %6, %7, %8, %9, %10, %11}, {%12, %13, %14, %15}, {%0, %1, %2, %3};"
                 : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
                 : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]),
                   "d"(b[0]), "d"(b[1]), "d"(b[2]), "d"(b[3]));
}

template <int SHAPE>
__global__ void k_dmma_chains(double *out, int iters)
{
    using S = MmaShape<SHAPE>;
    double a[S::NA], b[S::NB], acc[kChains][S::NC];
#pragma unroll
    for (int k = 0; k < S::NA; ++k) a[k] = 1e-3 * (threadIdx.x + k);
#pragma unroll
    for (int k = 0; k < S::NB; ++k) b[k] = 0.5 - 1e-4 * k;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
#pragma unroll
        for (int k = 0; k < S::NC; ++k) acc[c][k] = c + k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) mma_f64<SHAPE>(acc[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
#pragma unroll
        for (int k = 0; k < S::NC; ++k) s += acc[c][k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int SHAPE>
int time_dmma(double *buf, int blocks, int block, double *flops)
{
    using S = MmaShape<SHAPE>;
    const int iters = 2048;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_dmma_chains<SHAPE><<<blocks, block>>>(buf, 32);
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0);
        k_dmma_chains<SHAPE><<<blocks, block>>>(buf, iters);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return pdfgpu::cuda_fail(err, "mma probe kernel");
    const double warps = (double)blocks * (block / 32);
    *flops = 2.0 * S::M * S::N * S::K * (double)kChains * iters * warps / (best * 1e-3);
    return PDF_OK;
}

}  // namespace

extern "C" int pdf_probe_fp64_mma_peak(int32_t shape, double *flops)
{
    PDF_TRACE("pdf_probe_fp64_mma_peak");
    pdfgpu::clear_error();
    if (!flops) return pdfgpu::fail(PDF_E_ARG, "null output");
    if (shape < 0 || shape > 3) return pdfgpu::fail(PDF_E_ARG, "shape must be 0..3");
    int dev = 0, sms = 0;
    PDF_CUDA(cudaGetDevice(&dev));
    PDF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int block = 256, per_sm = 4;
    const int blocks = sms * per_sm;
    double *buf = nullptr;
    int rc = pdfgpu::dev_malloc((void **)&buf, (size_t)blocks * block * sizeof(double), "probe buffer");
    if (rc) return rc;
    switch (shape) {
    case 0: rc = time_dmma<0>(buf, blocks, block, flops); break;
    case 1: rc = time_dmma<1>(buf, blocks, block, flops); break;
    case 2: rc = time_dmma<2>(buf, blocks, block, flops); break;
    default: rc = time_dmma<3>(buf, blocks, block, flops); break;
    }
    cudaFree(buf);
    return rc;
}

// ------------------------------------------------- DFMA and DMMA in one warp
//
// Does the FP64 tensor instruction run beside the FMA pipe or on it?  Each
// iteration issues, per warp, 64 DFMA per thread (8 rounds over 8 chains:
// 4096 flops per warp) and 8 m8n8k4 DMMA (4096 flops per warp).  MODE 0
// issues only the DFMA half, 1 only the DMMA half, 2 both, interleaved.  If
// the two share one pipe the mixed kernel takes about the sum of the two
// times; if they ran side by side it would take about the longer one.

namespace {

template <int MODE>
__global__ void k_fp64_mixed(double *out, int iters, double b, double c)
{
    double f[kChains], acc[kChains][2];
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        f[k] = threadIdx.x * 1e-3 + k;
        acc[k][0] = k;
        acc[k][1] = k + 0.5;
    }
    const double a = 1e-3 * threadIdx.x;
    for (int it = 0; it < iters; ++it) {
        if (MODE != 1) {
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int k = 0; k < kChains; ++k) f[k] = fma(f[k], b, c);
        }
        if (MODE != 0) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) mma_f64<0>(acc[k], &a, &b);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += f[k] + acc[k][0] + acc[k][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int MODE>
int time_mixed(double *buf, int blocks, int block, float *ms_out)
{
    const int iters = 1024;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fp64_mixed<MODE><<<blocks, block>>>(buf, 16, 0.999, 1e-3);
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0);
        k_fp64_mixed<MODE><<<blocks, block>>>(buf, iters, 0.999, 1e-3);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return pdfgpu::cuda_fail(err, "mixed probe kernel");
    *ms_out = best;
    return PDF_OK;
}

}  // namespace

extern "C" int pdf_probe_fp64_mixed(double *dfma_flops, double *dmma_flops, double *mixed_flops)
{
    PDF_TRACE("pdf_probe_fp64_mixed");
    pdfgpu::clear_error();
    if (!dfma_flops || !dmma_flops || !mixed_flops) return pdfgpu::fail(PDF_E_ARG, "null output");
    int dev = 0, sms = 0;
    PDF_CUDA(cudaGetDevice(&dev));
    PDF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int block = 256, per_sm = 4, iters = 1024;
    const int blocks = sms * per_sm;
    double *buf = nullptr;
    int rc = pdfgpu::dev_malloc((void **)&buf, (size_t)blocks * block * sizeof(double), "probe buffer");
    if (rc) return rc;
    float ms[3] = {0, 0, 0};
    rc = time_mixed<0>(buf, blocks, block, &ms[0]);
    if (!rc) rc = time_mixed<1>(buf, blocks, block, &ms[1]);
    if (!rc) rc = time_mixed<2>(buf, blocks, block, &ms[2]);
    cudaFree(buf);
    if (rc) return rc;
    const double half = 4096.0 * iters * ((double)blocks * (block / 32));   // flops of one half
    *dfma_flops = half / (ms[0] * 1e-3);
    *dmma_flops = half / (ms[1] * 1e-3);
    *mixed_flops = 2.0 * half / (ms[2] * 1e-3);
    return PDF_OK;
}
