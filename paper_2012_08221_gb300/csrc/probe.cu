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
