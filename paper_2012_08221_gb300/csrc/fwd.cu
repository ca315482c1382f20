// Forward kernels: x*f for a shared pid list (matrix form), for one pid per
// point (pointwise form), alpha_s, and the host-buffer pipeline.
//
// PDFFlow Sec. 2.1: the query is a flavour set plus equal-length arrays of x
// and Q; the answer is one interpolated value per point and flavour.
#include <math.h>
#include <stdlib.h>

#include <algorithm>

#include "pdf_internal.h"
#include "sort_acc.cuh"

using namespace pdfgpu;

namespace {

constexpr int kBlock = 256;
__device__ __forceinline__ double qnan() { return __longlong_as_double(0x7FF8000000000000ll); }

// One point per thread; each warp takes 32 consecutive points at a time
// (grid-stride over warps).  A warp's results are staged in its own slice of
// shared memory and leave as one contiguous run of 32 * npid doubles (the
// output is [n][npid] row-major): one bulk copy issued by lane 0 when the run
// is 16-byte aligned and a multiple of 16 bytes long, else coalesced stores
// by the whole warp.  Only warp-level synchronisation, no block barriers in
// the loop.  With TAPE each point's adjoint tape record is written as well;
// with AS alpha_s at the point's Q^2 goes to as_out[i], from the same Q
// search and logarithm as the PDFs (a point whose x alone is out of the
// domain still gets its alpha_s, as alphasQ2 would give it).
template <bool Q_IS_Q, bool CONT, bool TAPE, bool AS = false>
__global__ void __launch_bounds__(kBlock) k_xfxq2(GridDev g, Cols cols, int npid, int member,
                                                  const double *__restrict__ x,
                                                  const double *__restrict__ q,
                                                  int64_t n, double *__restrict__ out,
                                                  double *__restrict__ tape, double *__restrict__ as_out = nullptr)
{
    extern __shared__ __align__(16) double sout[];
    __shared__ signed char scol[PDF_MAX_PIDS];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < PDF_MAX_PIDS; ++k) scol[k] = cols.c[k];
    }
    __syncthreads();
    const size_t cell_stride = (size_t)g.nflav * 16;
    const double *cm = g.coef + (size_t)member * g.nqc * g.nxc * cell_stride;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double *wbuf = sout + (size_t)wid * 32 * npid;
    const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5) * 32;
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + wid) * 32; base < n; base += wstride) {
        int64_t i = base + lane;
        bool live = i < n;
        double xi = live ? x[i] : 0.5;
        double qi = live ? q[i] : 10.0;
        if (Q_IS_Q) qi = qi * qi;
        const bool qbad = !q2_ok(dbits(qi));
        bool bad = live && !(x_ok(dbits(xi)) && !qbad);
        flag_status(g, bad);
        if (bad) {
            xi = 0.5;
            if (!AS || qbad) qi = 10.0;
        }
        double u, w;
        Axis X = axis_x(g, xi, &u);
        Axis Q = axis_q2(g, qi, &w);
        const bool oor = live && out_of_range(g, X, Q);
        flag_status(g, oor, PDF_S_RANGE);
        bad |= oor;
        if (TAPE && live) tape_put(tape, i, X, Q, bad);
        if (AS && live) {
            const double a = alphas_any(g, ld4(g.acoef + (size_t)Q.cell * 4), Q);
            as_out[i] = (qbad || (g.extrap == PDF_EXTRAP_ERROR && !Q.in)) ? qnan() : a;
        }
        const double *cell = cm + ((size_t)Q.cell * g.nxc + X.cell) * cell_stride;
        double *srow = wbuf + lane * npid;
        warp_run_reuse(lane);                 // the previous run has left the slice
        for (int a = 0; a < npid; ++a) {
            int col = scol[a];
            if (col >= 0) col = checked_index(g.status, col, g.nflav);
            double v = col >= 0 ? patch_any<CONT>(g, cell + col * 16, X, Q) : 0.0;
            srow[a] = bad ? qnan() : v;
        }
        const int rows = (int)min((int64_t)32, n - base);
        warp_run_store(out + base * npid, wbuf, rows * npid, lane);
    }
    if (lane == 0) bulk_wait_all();
}

// Small queries (at most kPairMax point-flavour pairs): one thread per pair,
// so that a few thousand points still spread over every SM and each thread's
// dependent chain is one flavour long; the coordinates are recomputed for
// every flavour of a point.  Outputs are written in pair order, which is the
// row-major [n][npid] layout.
constexpr int64_t kPairMax = 1 << 18;

template <bool Q_IS_Q, bool CONT, bool TAPE>
__global__ void __launch_bounds__(kBlock) k_xfxq2_pairs(GridDev g, Cols cols, int npid, int member,
                                                        const double *__restrict__ x,
                                                        const double *__restrict__ q,
                                                        int64_t n, double *__restrict__ out,
                                                        double *__restrict__ tape)
{
    __shared__ signed char scol[PDF_MAX_PIDS];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < PDF_MAX_PIDS; ++k) scol[k] = cols.c[k];
    }
    __syncthreads();
    const size_t cell_stride = (size_t)g.nflav * 16;
    const double *cm = g.coef + (size_t)member * g.nqc * g.nxc * cell_stride;
    const int64_t total = n * npid;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = p / npid;
        const int a = (int)(p - i * npid);
        double xi = x[i], qi = q[i];
        if (Q_IS_Q) qi = qi * qi;
        bool bad = !(x_ok(dbits(xi)) && q2_ok(dbits(qi)));
        flag_status(g, bad);
        if (bad) {
            xi = 0.5;
            qi = 10.0;
        }
        double u, w;
        Axis X = axis_x(g, xi, &u);
        Axis Q = axis_q2(g, qi, &w);
        const bool oor = out_of_range(g, X, Q);
        flag_status(g, oor, PDF_S_RANGE);
        bad |= oor;
        if (TAPE && a == 0) tape_put(tape, i, X, Q, bad);
        int col = scol[a];
        double v = 0.0;
        if (col >= 0) {
            col = checked_index(g.status, col, g.nflav);
            v = patch_any<CONT>(g, cm + ((size_t)Q.cell * g.nxc + X.cell) * cell_stride + col * 16, X, Q);
        }
        out[p] = bad ? qnan() : v;
    }
}

// DT (with TAPE): also keep each point's patch derivatives in t_x and t_q,
// computed with the value (patch_vd: the value's bits are unchanged), in
// dtape[i] = (dP/dtx, dP/dtq) (zeros for an absent pid), and the point's bin
// in the pointwise sorted adjoint in dbins[i] (-1 for none).
template <bool CONT, bool TAPE, bool DT = false>
__global__ void __launch_bounds__(kBlock) k_xfxq2_pw(GridDev g, int member,
                                                     const int *__restrict__ pid,
                                                     const double *__restrict__ x,
                                                     const double *__restrict__ q2,
                                                     int64_t n, double *__restrict__ out,
                                                     double *__restrict__ tape, double *__restrict__ dtape,
                                                     int *__restrict__ dbins, int nbins)
{
    const size_t cell_stride = (size_t)g.nflav * 16;
    const double *cm = g.coef + (size_t)member * g.nqc * g.nxc * cell_stride;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double xi = x[i], qi = q2[i];
        int col = pid_col(g, pid[i]);
        bool bad = !(x_ok(dbits(xi)) && q2_ok(dbits(qi)));
        flag_status(g, bad);
        if (bad) {
            xi = 0.5;
            qi = 10.0;
        }
        double u, w;
        Axis X = axis_x(g, xi, &u);
        Axis Q = axis_q2(g, qi, &w);
        const bool oor = out_of_range(g, X, Q);
        flag_status(g, oor, PDF_S_RANGE);
        bad |= oor;
        if (TAPE) tape_put(tape, i, X, Q, bad);
        double v = 0.0;
        if (DT) {
            double dtx = 0.0, dtq = 0.0;
            if (col >= 0) v = patch_vd(cm + ((size_t)Q.cell * g.nxc + X.cell) * cell_stride + col * 16, X, Q, &dtx, &dtq);
            reinterpret_cast<double2 *>(dtape)[i] = make_double2(dtx, dtq);
            dbins[i] = sorted_bin(g, X, Q, bad, col, half_pair(X, Q), nbins);
        } else if (col >= 0) {
            v = patch_any<CONT>(g, cm + ((size_t)Q.cell * g.nxc + X.cell) * cell_stride + col * 16, X, Q);
        }
        out[i] = bad ? qnan() : v;
    }
}

template <bool Q_IS_Q>
__global__ void __launch_bounds__(kBlock) k_alphas(GridDev g, const double *__restrict__ q,
                                                   int64_t n, double *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double qi = q[i];
        if (Q_IS_Q) qi = qi * qi;
        bool bad = !q2_ok(dbits(qi));
        flag_status(g, bad);
        if (bad) qi = 10.0;
        double w;
        Axis Q = axis_q2(g, qi, &w);
        const bool oor = g.extrap == PDF_EXTRAP_ERROR && !Q.in;
        flag_status(g, oor, PDF_S_RANGE);
        bad |= oor;
        double v = alphas_any(g, ld4(g.acoef + (size_t)Q.cell * 4), Q);
        out[i] = bad ? qnan() : v;
    }
}

// alpha_s and d alpha_s / d Q^2 = (da/dtq) / dW / Q^2 (zero across a frozen edge).
__global__ void __launch_bounds__(kBlock) k_alphas_grad(GridDev g, const double *__restrict__ q2, int64_t n,
                                                        double *__restrict__ out, double *__restrict__ dq2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double qi = q2[i];
        bool bad = !q2_ok(dbits(qi));
        flag_status(g, bad);
        if (bad) qi = 10.0;
        double w;
        Axis Q = axis_q2(g, qi, &w);
        const bool oor = g.extrap == PDF_EXTRAP_ERROR && !Q.in;
        flag_status(g, oor, PDF_S_RANGE);
        bad |= oor;
        const D4 a = ld4(g.acoef + (size_t)Q.cell * 4);
        double v = alphas_any(g, a, Q);
        double d2 = Q.in ? 2.0 * Q.t : 1.0, d3 = Q.in ? 3.0 * Q.t * Q.t : 1.0;
        double dt = fma(d3, a.w, fma(d2, a.z, a.y));
        if (!Q.in && g.extrap == PDF_EXTRAP_FREEZE) dt = 0.0;
        if (!Q.in && g.extrap == PDF_EXTRAP_CONTINUATION) {
            // d/dt of the continuation from the edge values y0 = a(0), y1 = a(1)
            const double y0 = a.x, y1 = a.x + a.y + a.z + a.w;
            dt = (y0 > kContMin && y1 > kContMin) ? v * log(y1 / y0) : y1 - y0;
        }
        if (out) out[i] = bad ? qnan() : v;
        dq2[i] = bad ? qnan() : dt * g.qcell[Q.cell].y * __drcp_rn(qi);
    }
}

// The cells the kernels' knot searches give (x, Q^2 given as bit patterns;
// the guide table when the grid has one): a test hook.
__global__ void k_cells(GridDev g, const double *__restrict__ x, const double *__restrict__ q2, int64_t n,
                        int *__restrict__ xc, int *__restrict__ qc)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double u, w;
        xc[i] = axis_x(g, x[i], &u).cell;
        qc[i] = axis_q2(g, q2[i], &w).cell;
    }
}

__global__ void k_log(GridDev g, const double *__restrict__ in, int64_t n, double *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = dlog(g, in[i]);
}

// A tape is only written for the adjoint's grids (not under the power-law
// continuation, which has no adjoint) and must allow 32-byte loads.
int check_tape(const pdfgpu_grid *g, const double *tape)
{
    if (!tape) return PDF_OK;
    if (g->d.extrap == PDF_EXTRAP_CONTINUATION)
        return fail(PDF_E_ARG, "no adjoint tape under the power-law continuation (the adjoint needs linear, "
                               "freeze or error extrapolation)");
    if ((uintptr_t)tape % 32) return fail(PDF_E_ARG, "tape must be 32-byte aligned");
    return PDF_OK;
}

int launch_matrix(pdfgpu_grid *g, int32_t member, const int32_t *pids, int32_t n_pid,
                  const double *x, const double *q, int64_t n, double *out, double *tape, cudaStream_t s,
                  bool q_is_q)
{
    clear_error();
    int rc = check_grid(g, true);
    if (rc) return rc;
    if (n < 0) return fail(PDF_E_ARG, "negative n");
    if (member < 0 || member >= g->d.nmem) return fail(PDF_E_ARG, "member out of range");
    Cols cols;
    rc = resolve_cols(g, pids, n_pid, &cols);
    if (rc) return rc;
    rc = check_tape(g, tape);
    if (rc) return rc;
    if (n == 0) return PDF_OK;
    if (!x || !q || !out) return fail(PDF_E_ARG, "null array");
    using PairKern = void (*)(GridDev, Cols, int, int, const double *, const double *, int64_t, double *, double *);
    using Kern = void (*)(GridDev, Cols, int, int, const double *, const double *, int64_t, double *, double *,
                          double *);
    const bool cont = g->d.extrap == PDF_EXTRAP_CONTINUATION;
    if (n * n_pid <= kPairMax) {
        PairKern k = tape ? k_xfxq2_pairs<false, false, true>
                 : q_is_q ? (cont ? k_xfxq2_pairs<true, true, false> : k_xfxq2_pairs<true, false, false>)
                          : (cont ? k_xfxq2_pairs<false, true, false> : k_xfxq2_pairs<false, false, false>);
        int grid = wave_grid(g, (const void *)k, kBlock, 0, n * n_pid);
        k<<<grid, kBlock, 0, s>>>(g->d, cols, n_pid, member, x, q, n, out, tape);
        PDF_CUDA(cudaGetLastError());
        return PDF_OK;
    }
    size_t smem = (size_t)kBlock * n_pid * sizeof(double);
    Kern k = tape ? k_xfxq2<false, false, true>
             : q_is_q ? (cont ? k_xfxq2<true, true, false> : k_xfxq2<true, false, false>)
                      : (cont ? k_xfxq2<false, true, false> : k_xfxq2<false, false, false>);
    rc = allow_dynamic_smem((const void *)k, smem);
    if (rc) return rc;
    // A query shorter than one wave runs in the smallest CTAs (32, 64 or 128
    // threads) whose grid still fits in one wave, so that the CTAs spread
    // evenly over the SMs: in 256-thread CTAs a short query leaves some SMs
    // a whole CTA (8 warps of points) more than others.
    int block = kBlock;
    for (int b : {32, 64, 128}) {
        const size_t sb = (size_t)b * n_pid * sizeof(double);
        if ((n + b - 1) / b <= (int64_t)g->sm_count * occupancy((const void *)k, b, sb)) {
            block = b;
            smem = sb;
            break;
        }
    }
    int grid = wave_grid(g, (const void *)k, block, smem, n);
    k<<<grid, block, smem, s>>>(g->d, cols, n_pid, member, x, q, n, out, tape, nullptr);
    PDF_CUDA(cudaGetLastError());
    return PDF_OK;
}

// x*f and alpha_s at the same points in one launch of the per-point kernel.
int launch_xf_alphas(pdfgpu_grid *g, int32_t member, const int32_t *pids, int32_t n_pid, const double *x,
                     const double *q2, int64_t n, double *out, double *alphas, cudaStream_t s)
{
    clear_error();
    int rc = check_grid(g, true);
    if (rc) return rc;
    if (!g->has_alphas) return fail(PDF_E_DESC, "grid has no alpha_s values");
    if (n < 0) return fail(PDF_E_ARG, "negative n");
    if (member < 0 || member >= g->d.nmem) return fail(PDF_E_ARG, "member out of range");
    Cols cols;
    rc = resolve_cols(g, pids, n_pid, &cols);
    if (rc) return rc;
    if (n == 0) return PDF_OK;
    if (!x || !q2 || !out || !alphas) return fail(PDF_E_ARG, "null array");
    const bool cont = g->d.extrap == PDF_EXTRAP_CONTINUATION;
    auto k = cont ? k_xfxq2<false, true, false, true> : k_xfxq2<false, false, false, true>;
    size_t smem = (size_t)kBlock * n_pid * sizeof(double);
    rc = allow_dynamic_smem((const void *)k, smem);
    if (rc) return rc;
    int block = kBlock;
    for (int b : {32, 64, 128}) {
        const size_t sb = (size_t)b * n_pid * sizeof(double);
        if ((n + b - 1) / b <= (int64_t)g->sm_count * occupancy((const void *)k, b, sb)) {
            block = b;
            smem = sb;
            break;
        }
    }
    int grid = wave_grid(g, (const void *)k, block, smem, n);
    k<<<grid, block, smem, s>>>(g->d, cols, n_pid, member, x, q2, n, out, nullptr, alphas);
    PDF_CUDA(cudaGetLastError());
    return PDF_OK;
}

int launch_alphas(pdfgpu_grid *g, const double *q, int64_t n, double *out, cudaStream_t s, bool q_is_q)
{
    clear_error();
    int rc = check_grid(g, false);
    if (rc) return rc;
    if (!g->has_alphas) return fail(PDF_E_DESC, "grid has no alpha_s values");
    if (n < 0) return fail(PDF_E_ARG, "negative n");
    if (n == 0) return PDF_OK;
    if (!q || !out) return fail(PDF_E_ARG, "null array");
    const void *kern = q_is_q ? (const void *)k_alphas<true> : (const void *)k_alphas<false>;
    int grid = wave_grid(g, kern, kBlock, 0, n);
    if (q_is_q)
        k_alphas<true><<<grid, kBlock, 0, s>>>(g->d, q, n, out);
    else
        k_alphas<false><<<grid, kBlock, 0, s>>>(g->d, q, n, out);
    PDF_CUDA(cudaGetLastError());
    return PDF_OK;
}

int launch_pw(pdfgpu_grid *g, int32_t member, const int32_t *pid, const double *x, const double *q2, int64_t n,
              double *out, double *tape, double *dtape, cudaStream_t s)
{
    clear_error();
    int rc = check_grid(g, true);
    if (rc) return rc;
    if (n < 0) return fail(PDF_E_ARG, "negative n");
    if (member < 0 || member >= g->d.nmem) return fail(PDF_E_ARG, "member out of range");
    rc = check_tape(g, tape);
    if (rc) return rc;
    if (dtape && !tape) return fail(PDF_E_ARG, "a derivative tape goes with a tape");
    if (dtape && (uintptr_t)dtape % 16) return fail(PDF_E_ARG, "derivative tape must be 16-byte aligned");
    const int64_t nbins64 = (int64_t)g->d.nqc * g->d.nxc * g->d.nflav * 4;   // the pointwise adjoint's bins
    if (dtape && nbins64 >= (int64_t)1 << 30) return fail(PDF_E_RANGE, "grid too large for the derivative tape");
    if (n == 0) return PDF_OK;
    if (!pid || !x || !q2 || !out) return fail(PDF_E_ARG, "null array");
    auto k = dtape  ? k_xfxq2_pw<false, true, true>
             : tape ? k_xfxq2_pw<false, true>
             : g->d.extrap == PDF_EXTRAP_CONTINUATION ? k_xfxq2_pw<true, false> : k_xfxq2_pw<false, false>;
    int grid = wave_grid(g, (const void *)k, kBlock, 0, n);
    int *dbins = dtape ? reinterpret_cast<int *>(dtape + 2 * n) : nullptr;
    k<<<grid, kBlock, 0, s>>>(g->d, member, pid, x, q2, n, out, tape, dtape, dbins,
                              (int)std::min<int64_t>(nbins64, (int64_t)1 << 30));
    PDF_CUDA(cudaGetLastError());
    return PDF_OK;
}

}  // namespace

extern "C" int xfxQ2_alphasQ2(pdfgpu_grid_t g, int32_t member, const int32_t *pids, int32_t n_pid,
                              const double *x, const double *q2, int64_t n, double *out, double *alphas,
                              pdfgpu_stream_t stream)
{
    PDF_TRACE("xfxQ2_alphasQ2");
    return launch_xf_alphas(g, member, pids, n_pid, x, q2, n, out, alphas, (cudaStream_t)stream);
}

extern "C" int xfxQ2(pdfgpu_grid_t g, int32_t member, const int32_t *pids, int32_t n_pid,
                     const double *x, const double *q2, int64_t n, double *out, pdfgpu_stream_t stream)
{
    PDF_TRACE("xfxQ2");
    return launch_matrix(g, member, pids, n_pid, x, q2, n, out, nullptr, (cudaStream_t)stream, false);
}

extern "C" int xfxQ(pdfgpu_grid_t g, int32_t member, const int32_t *pids, int32_t n_pid,
                    const double *x, const double *q, int64_t n, double *out, pdfgpu_stream_t stream)
{
    PDF_TRACE("xfxQ");
    return launch_matrix(g, member, pids, n_pid, x, q, n, out, nullptr, (cudaStream_t)stream, true);
}

extern "C" int xfxQ2_pw(pdfgpu_grid_t g, int32_t member, const int32_t *pid, const double *x,
                        const double *q2, int64_t n, double *out, pdfgpu_stream_t stream)
{
    PDF_TRACE("xfxQ2_pw");
    return launch_pw(g, member, pid, x, q2, n, out, nullptr, nullptr, (cudaStream_t)stream);
}

extern "C" int xfxQ2_tape(pdfgpu_grid_t g, int32_t member, const int32_t *pids, int32_t n_pid,
                          const double *x, const double *q2, int64_t n, double *out, double *tape,
                          pdfgpu_stream_t stream)
{
    PDF_TRACE("xfxQ2_tape");
    if (!tape && n != 0) {
        clear_error();
        return fail(PDF_E_ARG, "null tape");
    }
    return launch_matrix(g, member, pids, n_pid, x, q2, n, out, tape, (cudaStream_t)stream, false);
}

extern "C" int xfxQ2_pw_tape(pdfgpu_grid_t g, int32_t member, const int32_t *pid, const double *x,
                             const double *q2, int64_t n, double *out, double *tape, double *dtape,
                             pdfgpu_stream_t stream)
{
    PDF_TRACE("xfxQ2_pw_tape");
    if (!tape && n != 0) {
        clear_error();
        return fail(PDF_E_ARG, "null tape");
    }
    return launch_pw(g, member, pid, x, q2, n, out, tape, dtape, (cudaStream_t)stream);
}

extern "C" int alphasQ2(pdfgpu_grid_t g, const double *q2, int64_t n, double *out, pdfgpu_stream_t stream)
{
    PDF_TRACE("alphasQ2");
    return launch_alphas(g, q2, n, out, (cudaStream_t)stream, false);
}

extern "C" int alphasQ(pdfgpu_grid_t g, const double *q, int64_t n, double *out, pdfgpu_stream_t stream)
{
    PDF_TRACE("alphasQ");
    return launch_alphas(g, q, n, out, (cudaStream_t)stream, true);
}

extern "C" int alphasQ2_grad(pdfgpu_grid_t g, const double *q2, int64_t n, double *out, double *dq2,
                             pdfgpu_stream_t stream)
{
    PDF_TRACE("alphasQ2_grad");
    clear_error();
    int rc = check_grid(g, false);
    if (rc) return rc;
    if (!g->has_alphas) return fail(PDF_E_DESC, "grid has no alpha_s values");
    if (n < 0) return fail(PDF_E_ARG, "negative n");
    if (n == 0) return PDF_OK;
    if (!q2 || !dq2) return fail(PDF_E_ARG, "null array");
    int grid = wave_grid(g, (const void *)k_alphas_grad, kBlock, 0, n);
    k_alphas_grad<<<grid, kBlock, 0, (cudaStream_t)stream>>>(g->d, q2, n, out, dq2);
    PDF_CUDA(cudaGetLastError());
    return PDF_OK;
}

extern "C" int pdf_debug_log(pdfgpu_grid_t g, const double *in, int64_t n, double *out,
                             pdfgpu_stream_t stream)
{
    PDF_TRACE("pdf_debug_log");
    clear_error();
    int rc = check_grid(g, false);
    if (rc) return rc;
    if (n < 0) return fail(PDF_E_ARG, "negative n");
    if (n == 0) return PDF_OK;
    if (!in || !out) return fail(PDF_E_ARG, "null array");
    int grid = wave_grid(g, (const void *)k_log, kBlock, 0, n);
    k_log<<<grid, kBlock, 0, (cudaStream_t)stream>>>(g->d, in, n, out);
    PDF_CUDA(cudaGetLastError());
    return PDF_OK;
}

extern "C" int pdf_debug_cells(pdfgpu_grid_t g, const double *x, const double *q2, int64_t n, int32_t *x_cell,
                               int32_t *q_cell, int32_t *guided, pdfgpu_stream_t stream)
{
    PDF_TRACE("pdf_debug_cells");
    clear_error();
    int rc = check_grid(g, false);
    if (rc) return rc;
    if (n < 0) return fail(PDF_E_ARG, "negative n");
    if (guided) {
        guided[0] = g->d.nxg > 0;
        guided[1] = g->d.nqg > 0;
    }
    if (n == 0) return PDF_OK;
    if (!x || !q2 || !x_cell || !q_cell) return fail(PDF_E_ARG, "null array");
    int grid = wave_grid(g, (const void *)k_cells, kBlock, 0, n);
    k_cells<<<grid, kBlock, 0, (cudaStream_t)stream>>>(g->d, x, q2, n, x_cell, q_cell);
    PDF_CUDA(cudaGetLastError());
    return PDF_OK;
}

// Host buffers: chunks of points flow through three device staging slots on
// three internal streams, so the copy-in of one chunk, the kernel of the
// next and the copy-out of a third overlap.
extern "C" int xfxQ2_host(pdfgpu_grid_t g, int32_t member, const int32_t *pids, int32_t n_pid,
                          const double *x, const double *q2, int64_t n, double *out)
{
    PDF_TRACE("xfxQ2_host");
    clear_error();
    int rc = check_grid(g, true);
    if (rc) return rc;
    if (n < 0) return fail(PDF_E_ARG, "negative n");
    if (n_pid < 1 || n_pid > PDF_MAX_PIDS) return fail(PDF_E_RANGE, "bad pid count");
    if (n == 0) return PDF_OK;
    if (!x || !q2 || !out) return fail(PDF_E_ARG, "null array");
    std::lock_guard<std::mutex> lock(g->host_mu);
    // points per chunk: small enough that the pipeline fills quickly (the
    // device-to-host copy of the outputs is the bound), large enough to fill
    // the GPU; $PDFGPU_HOST_CHUNK overrides it
    static const int64_t chunk_pts = [] {
        const char *e = getenv("PDFGPU_HOST_CHUNK");
        long long v = e ? atoll(e) : 0;
        return (int64_t)(v >= 4096 ? v : (1 << 18));
    }();
    const int64_t chunk = std::min<int64_t>(n, chunk_pts);
    if (g->stage_pts < chunk || g->stage_pid < n_pid) {
        for (int s = 0; s < 3; ++s)
            for (int k = 0; k < 3; ++k) {
                if (g->stage[s][k]) cudaFree(g->stage[s][k]);
                g->stage[s][k] = nullptr;
            }
        int64_t pts = std::max<int64_t>(chunk, g->stage_pts);
        int np = std::max(n_pid, g->stage_pid);
        for (int s = 0; s < 3; ++s) {
            if (dev_malloc((void **)&g->stage[s][0], pts * sizeof(double), "host-path staging") ||
                dev_malloc((void **)&g->stage[s][1], pts * sizeof(double), "host-path staging") ||
                dev_malloc((void **)&g->stage[s][2], pts * np * sizeof(double), "host-path staging"))
                return PDF_E_NOMEM;
        }
        g->stage_pts = pts;
        g->stage_pid = np;
    }
    for (int s = 0; s < 3; ++s)
        if (!g->hs[s]) PDF_CUDA(cudaStreamCreateWithFlags(&g->hs[s], cudaStreamNonBlocking));
    // on any failure, copies already queued are drained before returning, so
    // that none of them touches the caller's buffers after the call
    auto drain = [&](int code) {
        for (int s = 0; s < 3; ++s) cudaStreamSynchronize(g->hs[s]);
        return code;
    };
    int64_t nchunks = (n + chunk - 1) / chunk;
    for (int64_t c = 0; c < nchunks; ++c) {
        int s = (int)(c % 3);
        cudaStream_t st = g->hs[s];
        int64_t off = c * chunk, m = std::min(chunk, n - off);
        cudaError_t e = cudaMemcpyAsync(g->stage[s][0], x + off, m * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g->stage[s][1], q2 + off, m * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return drain(cuda_fail(e, "host-to-device copy"));
        rc = launch_matrix(g, member, pids, n_pid, g->stage[s][0], g->stage[s][1], m, g->stage[s][2], nullptr, st, false);
        if (rc) return drain(rc);
        e = cudaMemcpyAsync(out + off * n_pid, g->stage[s][2], m * n_pid * sizeof(double), cudaMemcpyDeviceToHost,
                            st);
        if (e != cudaSuccess) return drain(cuda_fail(e, "device-to-host copy"));
    }
    for (int s = 0; s < 3; ++s) PDF_CUDA(cudaStreamSynchronize(g->hs[s]));
    return PDF_OK;
}
