// Counting-sort helpers shared by the adjoints that group work by grid cell
// (the luminosity adjoint and the grid gradients): the exclusive scan of a
// bin histogram into bin offsets.
#include "pdf_internal.h"

namespace {

constexpr int kScanBlock = 1024;
constexpr int kScanPer = 8;               // consecutive bins per thread and pass
constexpr int kScanPass = kScanBlock * kScanPer;

// One block scans hist[0..nbins) in passes of kScanPass bins.  A pass loads
// its bins into shared memory with coalesced loads; each thread sums its
// kScanPer consecutive bins, the threads' totals are scanned (shuffles in
// each warp, then warp 0 over the warp totals), each thread writes its bins'
// exclusive prefixes back to shared memory, and the pass leaves with
// coalesced stores; a running carry links the passes.  offs[k] = cursor[k] =
// sum of hist[0..k); offs[nbins] = the total.
__global__ void __launch_bounds__(kScanBlock) k_scan(const int *__restrict__ hist, int nbins,
                                                     int *__restrict__ offs, int *__restrict__ cursor)
{
    __shared__ int buf[kScanPass];
    __shared__ int wsum[kScanBlock / 32];
    __shared__ int carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    for (int base = 0; base < nbins; base += kScanPass) {
#pragma unroll
        for (int e = 0; e < kScanPer; ++e) {
            const int k = base + e * kScanBlock + threadIdx.x;
            buf[e * kScanBlock + threadIdx.x] = k < nbins ? hist[k] : 0;
        }
        __syncthreads();
        int v[kScanPer];
        int tot = 0;
#pragma unroll
        for (int e = 0; e < kScanPer; ++e) {
            v[e] = buf[threadIdx.x * kScanPer + e];
            tot += v[e];
        }
        int incl = tot;
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
        int run = carry + wsum[wid] + incl - tot;
#pragma unroll
        for (int e = 0; e < kScanPer; ++e) {
            buf[threadIdx.x * kScanPer + e] = run;
            run += v[e];
        }
        __syncthreads();
        if (threadIdx.x == kScanBlock - 1) carry = run;
#pragma unroll
        for (int e = 0; e < kScanPer; ++e) {
            const int k = base + e * kScanBlock + threadIdx.x;
            if (k < nbins) {
                const int o = buf[e * kScanBlock + threadIdx.x];
                offs[k] = o;
                cursor[k] = o;
            }
        }
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
