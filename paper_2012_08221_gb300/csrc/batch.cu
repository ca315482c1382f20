// Batched evaluation: many requests (grids of different knot counts,
// members, flavour subsets and sizes) in ONE persistent launch, captured in a
// CUDA graph and replayed (the counterpart of PDFFlow's compiled, traced
// graph, Sec. 2.1, for a whole batch of queries).
//
// Work is cut into tiles of block*qpt points.  A CTA takes the next tile from
// a global ticket counter (one atomicAdd per tile; no CTA ever waits for
// another), finds its request by binary search over the tiles' prefix sums,
// and evaluates it with the same patch arithmetic as the single-grid kernel.
// The launch shape (block size, points per thread, shared-memory staging of
// the knot and log tables) is chosen by a small autotuner whose results are
// cached per workload signature in a JSON file ($PDFGPU_TUNE_CACHE).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <stddef.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pdf_internal.h"

using namespace pdfgpu;

namespace {

constexpr int kMaxReqPids = 16;
constexpr int kStageX = 256;      // x cells that fit the staged tables
constexpr int kStageQ = 64;       // Q cells that fit the staged tables

struct BatchReq {
    int grid;
    int member;
    int npid;
    signed char cols[kMaxReqPids];
    const double *x;
    const double *q2;
    double *out;
    int64_t n;
    int64_t tile0;
};

__device__ __forceinline__ double qnan() { return __longlong_as_double(0x7FF8000000000000ll); }

struct StageTables {
    LogEntry logtab[kLogTab];
    uint64_t xbits[kStageX];
    double2 xcell[kStageX];
    uint64_t qbits[kStageQ];
    double2 qcell[kStageQ];
};

template <int QPT, bool STAGE, bool CONT>
__global__ void k_batch(const GridDev *__restrict__ grids, const BatchReq *__restrict__ reqs, int nreq,
                        int64_t ntiles, unsigned long long *ticket, int out_stride)
{
    extern __shared__ __align__(16) unsigned char smem[];
    double *sout = reinterpret_cast<double *>(smem);
    StageTables *st = reinterpret_cast<StageTables *>(smem + (size_t)blockDim.x * out_stride * sizeof(double));
    __shared__ GridDev sg;
    __shared__ BatchReq sr;
    __shared__ long long s_tile;
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            long long t = (long long)atomicAdd(ticket, 1ull);
            int r = 0;
            if (t < ntiles) {
                int lo = 0, hi = nreq - 1;
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (reqs[mid].tile0 <= t) lo = mid;
                    else hi = mid - 1;
                }
                r = lo;
                sr = reqs[r];
            }
            s_tile = t;
        }
        __syncthreads();
        const long long t = s_tile;
        if (t >= ntiles) break;
        if (sr.grid != cur) {
            cur = sr.grid;
            if (threadIdx.x == 0) sg = grids[cur];
            __syncthreads();
            if (STAGE && sg.nxc <= kStageX && sg.nqc <= kStageQ) {
                for (int k = threadIdx.x; k < kLogTab; k += blockDim.x) st->logtab[k] = sg.logtab[k];
                for (int k = threadIdx.x; k < sg.nxc; k += blockDim.x) {
                    st->xbits[k] = sg.xbits[k];
                    st->xcell[k] = sg.xcell[k];
                }
                for (int k = threadIdx.x; k < sg.nqc; k += blockDim.x) {
                    st->qbits[k] = sg.qbits[k];
                    st->qcell[k] = sg.qcell[k];
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    sg.logtab = st->logtab;
                    sg.xbits = st->xbits;
                    sg.xcell = st->xcell;
                    sg.qbits = st->qbits;
                    sg.qcell = st->qcell;
                }
            }
            __syncthreads();
        }
        const GridDev &g = sg;
        const int npid = sr.npid;
        const int64_t n = sr.n;
        const size_t cell_stride = (size_t)g.nflav * 16;
        const double *cm = g.coef + (size_t)sr.member * g.nqc * g.nxc * cell_stride;
        const int64_t p0 = (int64_t)(t - sr.tile0) * ((int64_t)blockDim.x * QPT);
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        double *wbuf = sout + (size_t)wid * 32 * out_stride;
#pragma unroll 1
        for (int qq = 0; qq < QPT; ++qq) {
            // this warp's 32 consecutive points of the tile
            const int64_t base = p0 + (int64_t)qq * blockDim.x + 32 * wid;
            if (base >= n) break;
            const int64_t i = base + lane;
            const bool live = i < n;
            double xi = live ? sr.x[i] : 0.5;
            double qi = live ? sr.q2[i] : 10.0;
            bool bad = live && !(x_ok(dbits(xi)) && q2_ok(dbits(qi)));
            flag_status(g, bad);
            if (bad) {
                xi = 0.5;
                qi = 10.0;
            }
            double u, w;
            Axis X = axis_x(g, xi, &u);
            Axis Q = axis_q2(g, qi, &w);
            const bool oor = live && out_of_range(g, X, Q);
            flag_status(g, oor, PDF_S_RANGE);
            bad |= oor;
            const double *cell = cm + ((size_t)Q.cell * g.nxc + X.cell) * cell_stride;
            double *srow = wbuf + lane * npid;
            for (int a = 0; a < npid; ++a) {
                int col = sr.cols[a];
                if (col >= 0) col = checked_index(g.status, col, g.nflav);
                double v = col >= 0 ? patch_any<CONT>(g, cell + col * 16, X, Q) : 0.0;
                srow[a] = bad ? qnan() : v;
            }
            __syncwarp();
            const int rows = (int)min((int64_t)32, n - base);
            const int cnt = rows * npid;
            double *dst = sr.out + base * npid;
            for (int k = lane; k < cnt; k += 32) dst[k] = wbuf[k];
            __syncwarp();
        }
        __syncthreads();   // everyone is done with sr/s_tile before thread 0 refills them
    }
}

struct Shape {
    int block, qpt, stage;
};

using KernelFn = void (*)(const GridDev *, const BatchReq *, int, int64_t, unsigned long long *, int);

template <bool CONT>
KernelFn kernel_for_t(const Shape &s)
{
    if (s.stage) {
        if (s.qpt == 1) return k_batch<1, true, CONT>;
        if (s.qpt == 2) return k_batch<2, true, CONT>;
        return k_batch<4, true, CONT>;
    }
    if (s.qpt == 1) return k_batch<1, false, CONT>;
    if (s.qpt == 2) return k_batch<2, false, CONT>;
    return k_batch<4, false, CONT>;
}

// `cont`: some grid of the launch uses the continuation extrapolation.
KernelFn kernel_for(const Shape &s, bool cont) { return cont ? kernel_for_t<true>(s) : kernel_for_t<false>(s); }

// ---------------------------------------------------------- tune cache (JSON)
// One entry per line: "signature": {"block": B, "qpt": Q, "stage": S, "ms": T}

std::map<std::string, std::pair<Shape, float>> read_cache(const char *path)
{
    std::map<std::string, std::pair<Shape, float>> m;
    FILE *f = path ? fopen(path, "r") : nullptr;
    if (!f) return m;
    char line[1024];
    while (fgets(line, sizeof line, f)) {
        char *q0 = strchr(line, '"');
        if (!q0) continue;
        char *q1 = strchr(q0 + 1, '"');
        if (!q1) continue;
        std::string key(q0 + 1, q1);
        Shape s{};
        float ms = 0;
        if (sscanf(q1 + 1, ": {\"block\": %d, \"qpt\": %d, \"stage\": %d, \"ms\": %f", &s.block, &s.qpt,
                   &s.stage, &ms) == 4)
            m[key] = {s, ms};
    }
    fclose(f);
    return m;
}

void write_cache(const char *path, const std::map<std::string, std::pair<Shape, float>> &m)
{
    if (!path) return;
    std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{\n");
    size_t k = 0;
    for (auto &e : m) {
        fprintf(f, " \"%s\": {\"block\": %d, \"qpt\": %d, \"stage\": %d, \"ms\": %.6f}%s\n", e.first.c_str(),
                e.second.first.block, e.second.first.qpt, e.second.first.stage, e.second.second,
                ++k < m.size() ? "," : "");
    }
    fprintf(f, "}\n");
    fclose(f);
    rename(tmp.c_str(), path);
}

}  // namespace

struct pdfgpu_batch {
    int device = 0;
    int sm_count = 0;
    std::vector<pdfgpu_grid_t> grid_handles;
    std::vector<BatchReq> host_reqs;   // tile0 filled per shape
    GridDev *d_grids = nullptr;
    BatchReq *d_reqs = nullptr;
    unsigned long long *d_ticket = nullptr;
    int nreq = 0;
    int out_stride = 1;
    int64_t ntiles = 0;
    Shape shape{256, 2, 1};
    bool cont = false;                  // some grid uses the continuation extrapolation
    int ctas = 0;
    size_t smem = 0;
    float tuned_ms = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static size_t shape_smem(const pdfgpu_batch *b, const Shape &s)
{
    size_t out = (size_t)s.block * b->out_stride * sizeof(double);
    return out + (s.stage ? sizeof(StageTables) : 0);
}

// Fill tile offsets for a shape and upload the request table.
static int configure(pdfgpu_batch *b, const Shape &s, cudaStream_t st)
{
    int64_t tile = (int64_t)s.block * s.qpt, acc = 0;
    for (auto &r : b->host_reqs) {
        r.tile0 = acc;
        acc += (r.n + tile - 1) / tile;
    }
    b->ntiles = acc;
    PDF_CUDA(cudaMemcpyAsync(b->d_reqs, b->host_reqs.data(), b->host_reqs.size() * sizeof(BatchReq),
                             cudaMemcpyHostToDevice, st));
    KernelFn k = kernel_for(s, b->cont);
    size_t smem = shape_smem(b, s);
    int rc = allow_dynamic_smem((const void *)k, smem);
    if (rc) return rc;
    b->ctas = b->sm_count * occupancy((const void *)k, s.block, smem);
    b->smem = smem;
    b->shape = s;
    return PDF_OK;
}

static int enqueue(pdfgpu_batch *b, cudaStream_t st)
{
    PDF_CUDA(cudaMemsetAsync(b->d_ticket, 0, sizeof(unsigned long long), st));
    KernelFn k = kernel_for(b->shape, b->cont);
    k<<<b->ctas, b->shape.block, b->smem, st>>>(b->d_grids, b->d_reqs, b->nreq, b->ntiles, b->d_ticket,
                                                 b->out_stride);
    PDF_CUDA(cudaGetLastError());
    return PDF_OK;
}

// Frees everything a batch owns, leaving the thread's error message alone
// (a failing pdf_batch_prepare keeps the message of the step that failed).
static void release_batch(pdfgpu_batch *b)
{
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->d_grids) cudaFree(b->d_grids);
    if (b->d_reqs) cudaFree(b->d_reqs);
    if (b->d_ticket) cudaFree(b->d_ticket);
    delete b;
}

extern "C" int pdf_batch_free(pdfgpu_batch_t b)
{
    PDF_TRACE("pdf_batch_free");
    clear_error();
    if (!b) return fail(PDF_E_ARG, "null batch");
    release_batch(b);
    return PDF_OK;
}

#define BTRY(x)                  \
    do {                         \
        int rc__ = (x);          \
        if (rc__ != PDF_OK) {    \
            release_batch(b);    \
            return rc__;         \
        }                        \
    } while (0)

extern "C" int pdf_batch_prepare(const pdfgpu_batch_desc *descs, int32_t n_desc, int32_t autotune,
                                 pdfgpu_stream_t stream, pdfgpu_batch_t *out)
{
    PDF_TRACE("pdf_batch_prepare");
    clear_error();
    if (!descs || !out || n_desc < 1) return fail(PDF_E_ARG, "need at least one request");
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    pdfgpu_batch *b = new pdfgpu_batch();
    cudaGetDevice(&b->device);
    cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
    std::vector<GridDev> gd;
    int64_t pts = 0, evals = 0;
    for (int i = 0; i < n_desc; ++i) {
        const pdfgpu_batch_desc &D = descs[i];
        int rc = check_grid(D.grid, true);
        if (rc) {
            release_batch(b);
            return rc;
        }
        if (D.member < 0 || D.member >= D.grid->d.nmem || D.n_pid < 1 || D.n_pid > kMaxReqPids || D.n < 0 ||
            (D.n > 0 && (!D.x || !D.q2 || !D.out))) {
            release_batch(b);
            return fail(PDF_E_ARG, "bad request " + std::to_string(i));
        }
        if (D.grid->device != b->device) {
            release_batch(b);
            return fail(PDF_E_ARG, "request " + std::to_string(i) + ": grid lives on another device");
        }
        int gi = -1;
        for (size_t k = 0; k < b->grid_handles.size(); ++k)
            if (b->grid_handles[k] == D.grid) gi = (int)k;
        if (gi < 0) {
            gi = (int)b->grid_handles.size();
            b->grid_handles.push_back(D.grid);
            gd.push_back(D.grid->d);
            if (D.grid->d.extrap == PDF_EXTRAP_CONTINUATION) b->cont = true;
        }
        Cols cols;
        int rc2 = resolve_cols(D.grid, D.pids, D.n_pid, &cols);
        if (rc2) {
            release_batch(b);
            return rc2;
        }
        BatchReq r{};
        r.grid = gi;
        r.member = D.member;
        r.npid = D.n_pid;
        for (int a = 0; a < kMaxReqPids; ++a) r.cols[a] = a < D.n_pid ? cols.c[a] : -1;
        r.x = D.x;
        r.q2 = D.q2;
        r.out = D.out;
        r.n = D.n;
        b->host_reqs.push_back(r);
        b->out_stride = std::max(b->out_stride, (int)D.n_pid);
        pts += D.n;
        evals += D.n * D.n_pid;
    }
    b->nreq = n_desc;
    // Tiles are handed out in table order: grouping the requests by (grid,
    // member) makes the CTAs that run at one time read one member's
    // coefficient table, which then stays in L2, instead of every member of
    // every set at once (the outputs go to each request's own array, so the
    // order changes no result).
    std::stable_sort(b->host_reqs.begin(), b->host_reqs.end(), [](const BatchReq &a, const BatchReq &c) {
        return a.grid != c.grid ? a.grid < c.grid : a.member < c.member;
    });
    BTRY(dev_malloc((void **)&b->d_grids, gd.size() * sizeof(GridDev), "batch grid table"));
    BTRY(dev_malloc((void **)&b->d_reqs, b->host_reqs.size() * sizeof(BatchReq), "batch request table"));
    BTRY(dev_malloc((void **)&b->d_ticket, sizeof(unsigned long long), "batch ticket"));
    if (cudaMemcpy(b->d_grids, gd.data(), gd.size() * sizeof(GridDev), cudaMemcpyHostToDevice) != cudaSuccess) {
        release_batch(b);
        return fail(PDF_E_CUDA, "upload of grid table failed");
    }

    // workload signature for the tune cache
    char sig[512];
    snprintf(sig, sizeof sig, "batch/sm%d/req%d/pts%lld/evals%lld/grids%zu/np%d", b->sm_count, n_desc,
             (long long)pts, (long long)evals, gd.size(), b->out_stride);
    for (auto &g : gd) {
        char t[64];
        snprintf(t, sizeof t, "/%dx%dx%d", g.nxc, g.nqc, g.nflav);
        strncat(sig, t, sizeof(sig) - strlen(sig) - 1);
    }
    const char *cache_path = getenv("PDFGPU_TUNE_CACHE");
    auto cache = read_cache(cache_path);
    Shape best{256, 2, 1};
    float best_ms = 0.0f;
    auto hit = cache.find(sig);
    if (hit != cache.end()) {
        best = hit->second.first;
        best_ms = hit->second.second;
    } else if (autotune) {
        const int blocks[3] = {128, 256, 512};
        const int qpts[3] = {1, 2, 4};
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        best_ms = 1e30f;
        for (int bi = 0; bi < 3; ++bi)
            for (int qi = 0; qi < 3; ++qi)
                for (int s = 0; s < 2; ++s) {
                    Shape sh{blocks[bi], qpts[qi], s};
                    BTRY(configure(b, sh, st));
                    BTRY(enqueue(b, st));     // warm-up
                    float ms_min = 1e30f;
                    for (int rep = 0; rep < 2; ++rep) {
                        cudaEventRecord(e0, st);
                        BTRY(enqueue(b, st));
                        cudaEventRecord(e1, st);
                        if (cudaEventSynchronize(e1) != cudaSuccess) {
                            release_batch(b);
                            return fail(PDF_E_CUDA, "tuning launch failed");
                        }
                        float ms = 0;
                        cudaEventElapsedTime(&ms, e0, e1);
                        ms_min = std::min(ms_min, ms);
                    }
                    if (ms_min < best_ms) {
                        best_ms = ms_min;
                        best = sh;
                    }
                }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cache[sig] = {best, best_ms};
        write_cache(cache_path, cache);
    }
    b->tuned_ms = best_ms;
    BTRY(configure(b, best, st));
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        release_batch(b);
        return fail(PDF_E_CUDA, "prepare");
    }
    // capture the launch (ticket reset + persistent kernel) into a graph
    cudaStream_t cap;
    BTRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess ? PDF_OK
                                                                               : fail(PDF_E_CUDA, "stream"));
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        int rc = enqueue(b, cap);
        cudaError_t e2 = cudaStreamEndCapture(cap, &b->graph);
        if (rc != PDF_OK || e2 != cudaSuccess) e = cudaErrorUnknown;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        release_batch(b);
        return cuda_fail(e, "graph capture of the batched launch");
    }
    *out = b;
    return PDF_OK;
}

extern "C" int pdf_batch_run(pdfgpu_batch_t b, pdfgpu_stream_t stream)
{
    PDF_TRACE("pdf_batch_run");
    clear_error();
    if (!b || !b->exec) return fail(PDF_E_ARG, "batch not prepared");
    int dev = 0;
    PDF_CUDA(cudaGetDevice(&dev));
    if (dev != b->device) PDF_CUDA(cudaSetDevice(b->device));
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (dev != b->device) cudaSetDevice(dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch of the batched launch");
    return PDF_OK;
}

extern "C" int pdf_batch_info(pdfgpu_batch_t b, int32_t *block, int32_t *qpt, int32_t *stage, int32_t *ctas,
                              float *ms)
{
    PDF_TRACE("pdf_batch_info");
    clear_error();
    if (!b) return fail(PDF_E_ARG, "null batch");
    if (block) *block = b->shape.block;
    if (qpt) *qpt = b->shape.qpt;
    if (stage) *stage = b->shape.stage;
    if (ctas) *ctas = b->ctas;
    if (ms) *ms = b->tuned_ms;
    return PDF_OK;
}

// ------------------------------------------------ allocation-free variant
//
// The same persistent kernel, launched once per call with a fixed shape
// (256 threads, 2 points per thread), whose scratch -- the tile ticket and
// the request and grid tables -- lives in one file-scope device array instead
// of memory allocated per batch.  Nothing here calls cudaMalloc or cudaFree.
// The tables reach the array by value, as the parameters of small copy
// kernels launched on the caller's stream ahead of the evaluation, so no
// host buffer of the library holds a call's tables once the call returns.

namespace {

constexpr int kNoAllocMaxRequests = 1024;
constexpr int kNoAllocMaxGrids = 32;

struct NoAllocScratch {
    unsigned long long ticket;
    unsigned long long pad[31];              // keeps the tables 256-byte aligned
    GridDev grids[kNoAllocMaxGrids];
    BatchReq reqs[kNoAllocMaxRequests];
};

// Kernel parameters of the copy kernels (each well inside the 32 KB that a
// launch may carry).
constexpr int kFillReqs = 384;
struct NoAllocHead {
    int ngrids;
    GridDev grids[kNoAllocMaxGrids];
};
struct NoAllocReqs {
    int first, count;
    BatchReq reqs[kFillReqs];
};
static_assert(sizeof(NoAllocHead) <= 30000 && sizeof(NoAllocReqs) <= 30000, "kernel parameters too large");
static_assert(sizeof(GridDev) % 8 == 0 && sizeof(BatchReq) % 8 == 0, "tables copied as 8-byte words");

// Resets the ticket and writes the grid table.
__global__ void k_noalloc_head(const __grid_constant__ NoAllocHead h, NoAllocScratch *S)
{
    if (threadIdx.x == 0) S->ticket = 0ull;
    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(h.grids);
    unsigned long long *dst = reinterpret_cast<unsigned long long *>(S->grids);
    const int words = h.ngrids * (int)(sizeof(GridDev) / 8);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
}

// Writes requests [first, first + count) of the request table.
__global__ void k_noalloc_reqs(const __grid_constant__ NoAllocReqs c, NoAllocScratch *S)
{
    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(c.reqs);
    unsigned long long *dst = reinterpret_cast<unsigned long long *>(S->reqs + c.first);
    const int words = c.count * (int)(sizeof(BatchReq) / 8);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
}

constexpr int kNoAllocDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_dev_addr[kNoAllocDevices];   // device address of the array, per device
// Host-side parameter blocks, static (no heap use, no large stack frame);
// a launch copies its parameters when it is issued, so they are refilled
// freely by the next launch.
NoAllocHead g_noalloc_head;
NoAllocReqs g_noalloc_reqs;

}  // namespace

// About 85 KB per device that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

extern "C" int pdf_batch_run_noalloc(const pdfgpu_batch_desc *descs, int32_t n_desc,
                                     pdfgpu_stream_t stream)
{
    PDF_TRACE("pdf_batch_run_noalloc");
    clear_error();
    if (!descs) return fail(PDF_E_ARG, "null request list");
    if (n_desc < 1 || n_desc > kNoAllocMaxRequests)
        return fail(PDF_E_RANGE, "pdf_batch_run_noalloc takes 1 to 1024 requests; got " +
                                     std::to_string(n_desc));
    int dev = 0;
    PDF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocDevices) return fail(PDF_E_RANGE, "device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocHead &H = g_noalloc_head;
    int ngrids = 0;
    bool cont = false;                  // some grid uses the continuation extrapolation
    pdfgpu_grid_t handles[kNoAllocMaxGrids];
    int out_stride = 1;
    const int block = 256, qpt = 2;
    const int64_t tile = (int64_t)block * qpt;
    // first pass: validate every request and build the grid table
    for (int i = 0; i < n_desc; ++i) {
        const pdfgpu_batch_desc &D = descs[i];
        int rc = check_grid(D.grid, true);
        if (rc) return rc;
        if (D.grid->device != dev) return fail(PDF_E_ARG, "request grid lives on another device");
        if (D.member < 0 || D.member >= D.grid->d.nmem || D.n_pid < 1 || D.n_pid > kMaxReqPids ||
            D.n < 0 || (D.n > 0 && (!D.x || !D.q2 || !D.out)))
            return fail(PDF_E_ARG, "bad request " + std::to_string(i));
        int gi = -1;
        for (int k = 0; k < ngrids; ++k)
            if (handles[k] == D.grid) gi = k;
        if (gi < 0) {
            if (ngrids == kNoAllocMaxGrids)
                return fail(PDF_E_RANGE, "pdf_batch_run_noalloc takes at most 32 distinct grids");
            gi = ngrids++;
            handles[gi] = D.grid;
            if (D.grid->d.extrap == PDF_EXTRAP_CONTINUATION) cont = true;
            H.grids[gi] = D.grid->d;
        }
        Cols cols;
        rc = resolve_cols(D.grid, D.pids, D.n_pid, &cols);
        if (rc) return rc;
        out_stride = std::max(out_stride, (int)D.n_pid);
    }
    H.ngrids = ngrids;
    if (!g_noalloc_dev_addr[dev]) {
        // once per device, with that device current
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the batch scratch");
        g_noalloc_dev_addr[dev] = p;
    }
    NoAllocScratch *S = reinterpret_cast<NoAllocScratch *>(g_noalloc_dev_addr[dev]);
    cudaStream_t st = (cudaStream_t)stream;
    k_noalloc_head<<<1, 256, 0, st>>>(H, S);
    PDF_CUDA(cudaGetLastError());
    // second pass: the request table, in chunks that fit a launch's parameters
    int64_t ntiles = 0;
    for (int c0 = 0; c0 < n_desc; c0 += kFillReqs) {
        NoAllocReqs &R = g_noalloc_reqs;
        R.first = c0;
        R.count = std::min(kFillReqs, n_desc - c0);
        for (int j = 0; j < R.count; ++j) {
            const pdfgpu_batch_desc &D = descs[c0 + j];
            int gi = 0;
            for (int k = 0; k < ngrids; ++k)
                if (handles[k] == D.grid) gi = k;
            Cols cols;
            int rc = resolve_cols(D.grid, D.pids, D.n_pid, &cols);
            if (rc) return rc;
            BatchReq &r = R.reqs[j];
            r = BatchReq{};
            r.grid = gi;
            r.member = D.member;
            r.npid = D.n_pid;
            for (int a = 0; a < kMaxReqPids; ++a) r.cols[a] = a < D.n_pid ? cols.c[a] : -1;
            r.x = D.x;
            r.q2 = D.q2;
            r.out = D.out;
            r.n = D.n;
            r.tile0 = ntiles;
            ntiles += (D.n + tile - 1) / tile;
        }
        k_noalloc_reqs<<<1, 256, 0, st>>>(R, S);
        PDF_CUDA(cudaGetLastError());
    }
    if (ntiles == 0) return PDF_OK;
    KernelFn k = kernel_for(Shape{block, qpt, 0}, cont);
    size_t smem = (size_t)block * out_stride * sizeof(double);
    int rc = allow_dynamic_smem((const void *)k, smem);
    if (rc) return rc;
    int sms = 0;
    PDF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int ctas = sms * occupancy((const void *)k, block, smem);
    k<<<ctas, block, smem, st>>>(S->grids, S->reqs, n_desc, ntiles, &S->ticket, out_stride);
    PDF_CUDA(cudaGetLastError());
    return PDF_OK;
}
