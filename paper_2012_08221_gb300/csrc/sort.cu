// Counting-sort helpers shared by the adjoints that group work by grid cell
// (the luminosity adjoint and the pointwise grid gradient): the exclusive
// scan of a bin histogram into bin offsets.
#include "pdf_internal.h"

namespace {

constexpr int kScanBlock = 1024;

// One block scans hist[0..nbins) in chunks of 1024: each warp scans its 32
// values with shuffles, warp 0 scans the 32 warp totals, and a running carry
// links the chunks.  offs[k] = cursor[k] = sum of hist[0..k); offs[nbins] =
// the total.
__global__ void __launch_bounds__(kScanBlock) k_scan(const int *__restrict__ hist, int nbins,
                                                     int *__restrict__ offs, int *__restrict__ cursor)
{
    __shared__ int wsum[kScanBlock / 32];
    __shared__ int carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nbins; base += kScanBlock) {
        const int k = base + threadIdx.x;
        const int v = k < nbins ? hist[k] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int w = wsum[lane], wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            wsum[lane] = wi - w;               // exclusive prefix of the warp totals
        }
        __syncthreads();
        const int excl = carry + wsum[wid] + incl - v;
        if (k < nbins) {
            offs[k] = excl;
            cursor[k] = excl;
        }
        __syncthreads();
        if (threadIdx.x == kScanBlock - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) offs[nbins] = carry;
}

}  // namespace

namespace pdfgpu {

int exclusive_scan(const int *hist, int nbins, int *offs, int *cursor, cudaStream_t s)
{
    k_scan<<<1, kScanBlock, 0, s>>>(hist, nbins, offs, cursor);
    PDF_CUDA(cudaGetLastError());
    return PDF_OK;
}

}  // namespace pdfgpu
