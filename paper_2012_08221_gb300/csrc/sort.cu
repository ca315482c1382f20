// Counting-sort helpers shared by the adjoints that group work by grid cell
// (the luminosity adjoint and the grid gradients): the exclusive scan of a
// bin histogram into bin offsets.
#include "pdf_internal.h"

#include <algorithm>

namespace {

constexpr int kScanBlock = 1024;
constexpr int kScanPer = 8;               // consecutive bins per thread and pass
constexpr int kScanPass = kScanBlock * kScanPer;
constexpr int kScanMaxBlocks = 64;        // one block per pass up to this many passes

// One pass over hist[base, base + kScanPass) by the whole block, given the
// sum of hist[0, base) in `carry`: the pass's bins are loaded into shared
// memory with coalesced loads; each thread sums its kScanPer consecutive
// bins, the threads' totals are scanned (shuffles in each warp, then warp 0
// over the warp totals), each thread writes its bins' exclusive prefixes
// back to shared memory, and the pass leaves with coalesced stores of
// offs[k] = cursor[k] = carry + sum of hist[base, k).  Returns the sum of
// hist[0, base + kScanPass) (to every thread).
__device__ int scan_pass(const int *__restrict__ hist, int nbins, int base, int carry, int *__restrict__ offs,
                         int *__restrict__ cursor, int *buf, int *wsum, int *shared_carry)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
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
    if (threadIdx.x == kScanBlock - 1) *shared_carry = run;
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
    return *shared_carry;
}

// One block scans hist[0..nbins) in passes of kScanPass bins, a running
// carry linking the passes.  offs[k] = cursor[k] = sum of hist[0..k);
// offs[nbins] = the total.
__global__ void __launch_bounds__(kScanBlock) k_scan(const int *__restrict__ hist, int nbins,
                                                     int *__restrict__ offs, int *__restrict__ cursor)
{
    __shared__ int buf[kScanPass];
    __shared__ int wsum[kScanBlock / 32];
    __shared__ int carry;
    int c = 0;
    for (int base = 0; base < nbins; base += kScanPass)
        c = scan_pass(hist, nbins, base, c, offs, cursor, buf, wsum, &carry);
    if (threadIdx.x == 0) offs[nbins] = c;
}

// The same result with one block per pass (at most kScanMaxBlocks passes):
// block b first sums hist[0, b kScanPass) itself (the histogram is small and
// L2-resident, so re-reading the passes before it costs less than waiting
// for them), then scans its own pass from that carry; the last block writes
// the total.  No block waits for another.
__global__ void __launch_bounds__(kScanBlock) k_scan_blocks(const int *__restrict__ hist, int nbins,
                                                            int *__restrict__ offs, int *__restrict__ cursor)
{
    __shared__ int buf[kScanPass];
    __shared__ int wsum[kScanBlock / 32];
    __shared__ int carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int base = blockIdx.x * kScanPass;
    int part = 0;
    for (int k = threadIdx.x; k < base; k += 4 * kScanBlock) {
        int a0 = hist[k];
        int a1 = k + kScanBlock < base ? hist[k + kScanBlock] : 0;
        int a2 = k + 2 * kScanBlock < base ? hist[k + 2 * kScanBlock] : 0;
        int a3 = k + 3 * kScanBlock < base ? hist[k + 3 * kScanBlock] : 0;
        part += (a0 + a1) + (a2 + a3);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) wsum[wid] = part;
    __syncthreads();
    if (wid == 0) {
        int w = wsum[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (lane == 0) carry = w;
    }
    __syncthreads();
    const int c0 = carry;
    __syncthreads();
    const int c = scan_pass(hist, nbins, base, c0, offs, cursor, buf, wsum, &carry);
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) offs[nbins] = c;
}

constexpr int kHistBlock = 1024;
constexpr int kHistSmemBins = 50 * 1024;   // 200 KB of counters, one block per SM

// Histogram of the keys, four loads in flight per thread; counters in
// shared memory (flushed once per block) when they fit.
__global__ void __launch_bounds__(kHistBlock) k_key_hist(const int *__restrict__ keys, int64_t n,
                                                         int *__restrict__ hist, int nbins, unsigned *status)
{
    extern __shared__ int shist[];
    const bool sh = nbins <= kHistSmemBins;
    if (sh) {
        for (int k = threadIdx.x; k < nbins; k += blockDim.x) shist[k] = 0;
        __syncthreads();
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r0 < n; r0 += 4 * stride) {
        int k[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) k[u] = r0 + u * stride < n ? __ldg(keys + r0 + u * stride) : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (k[u] < 0) continue;
            const int b = pdfgpu::checked_index(status, k[u], nbins);
            if (sh) atomicAdd(&shist[b], 1);
            else atomicAdd(&hist[b], 1);
        }
    }
    if (sh) {
        __syncthreads();
        for (int k = threadIdx.x; k < nbins; k += blockDim.x)
            if (shist[k]) atomicAdd(&hist[k], shist[k]);
    }
}

}  // namespace

namespace pdfgpu {

int key_histogram(const int *keys, int64_t n, int *hist, int nbins, unsigned *status, int sm_count,
                  cudaStream_t s)
{
    if (n <= 0) return PDF_OK;
    const size_t smem = nbins <= kHistSmemBins ? (size_t)nbins * sizeof(int) : 0;
    int rc = allow_dynamic_smem((const void *)k_key_hist, smem);
    if (rc) return rc;
    const int64_t want = (n + 4 * kHistBlock - 1) / (4 * kHistBlock);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(sm_count, want));
    k_key_hist<<<grid, kHistBlock, smem, s>>>(keys, n, hist, nbins, status);
    PDF_CUDA(cudaGetLastError());
    return PDF_OK;
}

int exclusive_scan(const int *hist, int nbins, int *offs, int *cursor, cudaStream_t s)
{
    const int passes = (nbins + kScanPass - 1) / kScanPass;
    if (passes >= 2 && passes <= kScanMaxBlocks)
        k_scan_blocks<<<passes, kScanBlock, 0, s>>>(hist, nbins, offs, cursor);
    else
        k_scan<<<1, kScanBlock, 0, s>>>(hist, nbins, offs, cursor);
    PDF_CUDA(cudaGetLastError());
    return PDF_OK;
}

}  // namespace pdfgpu
