// Host-side internals shared by the pdfgpu translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "pdf_common.cuh"

struct pdfgpu_grid {
    int device = 0;
    int sm_count = 0;
    pdfgpu::GridDev d{};            // device view (pointers into `blocks`)
    std::vector<void *> blocks;     // device allocations owned by the grid
    bool bound = false;             // coefficients built
    bool has_alphas = false;
    std::vector<int32_t> pids;      // host copy
    std::vector<int32_t> n_q;
    std::vector<double> U, W;       // knot logs (host)
    // scratch for the luminosity reduction (block partial sums)
    double *partials = nullptr;
    int partials_cap = 0;
    // scratch of the luminosity adjoint (event records, cell-sorted order)
    void *lumi_scratch = nullptr;
    size_t lumi_scratch_bytes = 0;
    // scratch of the sorted pointwise grid gradient (keys, records, bins)
    void *bwd_scratch = nullptr;
    size_t bwd_scratch_bytes = 0;
    // staging for the host-buffer entry point
    std::mutex host_mu;
    cudaStream_t hs[3] = {nullptr, nullptr, nullptr};
    double *stage[3][3] = {{nullptr}};  // [slot][x, q2, out]
    int64_t stage_pts = 0;
    int stage_pid = 0;
};

namespace pdfgpu {

// One NVTX range per ABI call, named after the entry point, so that a
// profiler's timeline shows which call launched which kernels (a no-op when
// no tool is attached).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
#define PDF_TRACE(name) pdfgpu::TraceRange pdf_trace_range__(name)

// Thread-local error message and return-code helpers.
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
void clear_error();

// cudaMalloc that leaves no error behind: on failure *p is NULL, the CUDA
// runtime's last-error state is cleared (so that a later launch check on this
// thread does not report it again) and PDF_E_NOMEM is returned with `what` in
// the thread's message.
int dev_malloc(void **p, size_t bytes, const char *what);

#define PDF_CUDA(call)                                      \
    do {                                                    \
        cudaError_t e__ = (call);                           \
        if (e__ != cudaSuccess) return pdfgpu::cuda_fail(e__, #call); \
    } while (0)

// Resident CTAs per SM for a kernel at a block size and dynamic smem.
int occupancy(const void *kernel, int block, size_t smem);

// Let `kernel` launch with `bytes` of dynamic shared memory on the current
// device.  Raise-only and serialised: the limit of a kernel is never lowered
// below what an earlier caller (a prepared batch, another thread) relies on.
int allow_dynamic_smem(const void *kernel, size_t bytes);

// Grid of a grid-stride launch: enough CTAs for n items, at most one wave.
int wave_grid(const pdfgpu_grid *g, const void *kernel, int block, size_t smem, int64_t items);

// Coefficient build (grid.cu) used by load and bind.
int build_coefficients(pdfgpu_grid *g, const double *dev_values, cudaStream_t s);

// Column list of a matrix-form call (resolved from the pid list on the host).
struct Cols {
    signed char c[PDF_MAX_PIDS];
};
int resolve_cols(const pdfgpu_grid *g, const int32_t *pids, int32_t n_pid, Cols *cols);

// Exclusive scan of a bin histogram (on `s`): offs[k] = cursor[k] =
// sum of hist[0..k), offs[nbins] = the total.  offs and cursor hold nbins + 1
// and nbins ints.
int exclusive_scan(const int *hist, int nbins, int *offs, int *cursor, cudaStream_t s);

// Histogram of n bin keys (a negative key adds nothing) into hist[0..nbins),
// which the caller has zeroed: in shared memory, one block of 1024 threads
// per SM (sm_count blocks at most), when the bins fit in 50 * 1024 counters,
// else with global atomics.  A key >= nbins sets PDF_S_BOUNDS in the checked
// build.
int key_histogram(const int *keys, int64_t n, int *hist, int nbins, unsigned *status, int sm_count,
                  cudaStream_t s);

// Shared argument checks.
int check_grid(const pdfgpu_grid *g, bool need_values);

}  // namespace pdfgpu
