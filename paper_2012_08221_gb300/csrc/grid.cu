// Grid loading: validation, knot tables, bicubic patch coefficients.
//
// A grid follows the LHAPDF layout the paper keeps (PDFFlow Sec. 1 and 4):
// x*f values on x knots times Q knots, the Q knots split into subgrids at
// flavour thresholds with the threshold knot stored in both neighbours.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "pdf_internal.h"

using namespace pdfgpu;

namespace pdfgpu {

static thread_local std::string t_err;

int fail(int code, const std::string &msg)
{
    t_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    t_err = std::string(what) + ": " + cudaGetErrorString(e);
    (void)cudaGetLastError();   // a non-sticky error must not resurface in a later check
    return PDF_E_CUDA;
}

int dev_malloc(void **p, size_t bytes, const char *what)
{
    if (cudaMalloc(p, bytes) == cudaSuccess) return PDF_OK;
    *p = nullptr;
    (void)cudaGetLastError();
    return fail(PDF_E_NOMEM, std::string(what) + ": out of device memory");
}

void clear_error() { t_err.clear(); }

int occupancy(const void *kernel, int block, size_t smem)
{
    // cached per (device, kernel, block, shared memory): launches ask often
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, int, size_t>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, kernel, block, smem);
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, smem) != cudaSuccess) {
        (void)cudaGetLastError();
        n = 1;
    }
    n = n < 1 ? 1 : n;
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = n;
    return n;
}

int allow_dynamic_smem(const void *kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return PDF_OK;    // the default limit, never lowered here
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> granted;
    int dev = 0;
    PDF_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    size_t &have = granted[{dev, kernel}];
    if (bytes > have) {
        PDF_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        have = bytes;
    }
    return PDF_OK;
}

int wave_grid(const pdfgpu_grid *g, const void *kernel, int block, size_t smem, int64_t items)
{
    int64_t need = (items + block - 1) / block;
    int64_t wave = (int64_t)g->sm_count * occupancy(kernel, block, smem);
    return (int)std::max<int64_t>(1, std::min(need, wave));
}

int check_grid(const pdfgpu_grid *g, bool need_values)
{
    if (!g) return fail(PDF_E_ARG, "null grid handle");
    if (need_values && !g->bound) return fail(PDF_E_UNBOUND, "grid has no values bound");
    if (cudaSetDevice(g->device) != cudaSuccess) return fail(PDF_E_CUDA, "cudaSetDevice failed");
    return PDF_OK;
}

int resolve_cols(const pdfgpu_grid *g, const int32_t *pids, int32_t n_pid, Cols *cols)
{
    if (!pids || n_pid < 1) return fail(PDF_E_ARG, "empty pid list");
    if (n_pid > PDF_MAX_PIDS) return fail(PDF_E_RANGE, "more than PDF_MAX_PIDS pids");
    for (int a = 0; a < n_pid; ++a) {
        int p = pids[a] == 21 ? 0 : pids[a];
        int c = -1;
        for (size_t k = 0; k < g->pids.size(); ++k)
            if (g->pids[k] == p) c = (int)k;
        cols->c[a] = (signed char)c;
    }
    return PDF_OK;
}

}  // namespace pdfgpu

// ------------------------------------------------------------- host tables

// Tables of the log routine: (1/c_j, -ln(1/c_j) as high + low parts) with
// c_j = 1 + (j + 1/2)/1024 (c_0 = 1, c_1023 = 2), and e ln 2 as high + low
// parts for every biased exponent; long double for the logs.
static void make_log_tables(std::vector<LogEntry> &tab, std::vector<double2> &etab)
{
    tab.resize(kLogTab);
    for (int j = 0; j < kLogTab; ++j) {
        double c = 1.0 + (j + 0.5) / (double)kLogTab;     // exact
        if (j == 0) c = 1.0;
        if (j == kLogTab - 1) c = 2.0;
        double inv = 1.0 / c;                              // correctly rounded
        long double L = -logl((long double)inv);
        double hi = (double)L;
        double lo = (double)(L - (long double)hi);
        tab[j] = LogEntry{inv, hi, lo, 0.0};
    }
    etab.resize(2048);
    const long double ln2 = 0.693147180559945309417232121458176568L;
    for (int e = 0; e < 2048; ++e) {
        long double v = (long double)(e - 1023) * ln2;
        double hi = (double)v;
        etab[e] = make_double2(hi, (double)(v - (long double)hi));
    }
}

// Finite-difference coefficients of cell k on knots z[0..n-1]:
//   dz_k D_k     = p0 g_{k-1} + p1 g_k + p2 g_{k+1}
//   dz_k D_{k+1} = q0 g_k     + q1 g_{k+1} + q2 g_{k+2}
// (one-sided secant at the first/last knot, mean of the secants inside),
// assembled into M[m][i]: monomial coefficient m of the interval cubic in
// t = (z - z_k)/dz_k from stencil value i (i <-> knot k-1+i).  With `linear`
// the interval polynomial is the straight line between its two knots.
//
// In Hermite form the weights are W(t) = e_k h00(t) + P h10(t) + e_k+1 h01(t)
// + Q h11(t), with P = (p0, p1, p2, 0), Q = (0, q0, q1, q2) and e_k, e_k+1
// the unit rows of the cell's two knots.  Ms is the same cubic as a
// polynomial in s = 1 - t (the distance to the upper knot): with
// h00(t) = h01(s), h01(t) = h00(s), h10(t) = -h11(s), h11(t) = -h10(s),
//   W = e_k+1 h00(s) + e_k h01(s) - P h11(s) - Q h10(s),
// so that its constant and linear rows are exact (e_k+1 and -Q): near the
// upper knot the weights that vanish there come out of small powers of s,
// not of a cancellation between the rows of M.
static void cell_matrix(const double *z, int n, int k, double M[16], bool linear, double Ms[16])
{
    if (linear) {
        // straight line between the interval's two knots: c0 = g_k, c1 = g_{k+1} - g_k
        const double m[16] = {0.0, 1.0, 0.0, 0.0, 0.0, -1.0, 1.0, 0.0,
                              0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        // in s: g_{k+1} + s (g_k - g_{k+1})
        const double ms[16] = {0.0, 0.0, 1.0, 0.0, 0.0, 1.0, -1.0, 0.0,
                               0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        memcpy(M, m, sizeof(m));
        memcpy(Ms, ms, sizeof(ms));
        return;
    }
    double dz = z[k + 1] - z[k];
    double p0, p1, p2, q0, q1, q2;
    if (k == 0) {
        p0 = 0.0; p1 = -1.0; p2 = 1.0;
    } else {
        double rho = dz / (z[k] - z[k - 1]);
        p0 = -0.5 * rho; p1 = 0.5 * rho - 0.5; p2 = 0.5;
    }
    if (k + 1 == n - 1) {
        q0 = -1.0; q1 = 1.0; q2 = 0.0;
    } else {
        double sig = dz / (z[k + 2] - z[k + 1]);
        q0 = -0.5; q1 = 0.5 - 0.5 * sig; q2 = 0.5 * sig;
    }
    const double m[16] = {
        0.0, 1.0, 0.0, 0.0,
        p0, p1, p2, 0.0,
        -2.0 * p0, -3.0 - 2.0 * p1 - q0, 3.0 - 2.0 * p2 - q1, -q2,
        p0, 2.0 + p1 + q0, -2.0 + p2 + q1, q2};
    memcpy(M, m, sizeof(m));
    // h00(s) = 1 - 3s^2 + 2s^3, h01(s) = 3s^2 - 2s^3, h10(s) = s - 2s^2 + s^3,
    // h11(s) = -s^2 + s^3
    const double ms[16] = {
        0.0, 0.0, 1.0, 0.0,
        0.0, -q0, -q1, -q2,
        p0, 3.0 + p1 + 2.0 * q0, -3.0 + p2 + 2.0 * q1, 2.0 * q2,
        -p0, -2.0 - p1 - q0, 2.0 - p2 - q1, -q2};
    memcpy(Ms, ms, sizeof(ms));
}

// Guide table of a cell search over ascending lower keys (see
// find_cell_guided): the widest bucket width 2^shift, at most kGuideMax
// buckets from the first key to key_hi, for which no bucket holds more than
// kGuideRun further lower keys (the last bucket counts every cell above it,
// since keys beyond key_hi fall into it).  Left empty when no width
// qualifies (knots clustered far more densely in one place than another);
// the kernels then search by bisection.
static constexpr uint64_t kGuideMax = 4096;

static void build_guide(const std::vector<uint64_t> &keys, uint64_t key_hi, std::vector<int> &guide, int *shift)
{
    guide.clear();
    *shift = 0;
    const int ncell = (int)keys.size();
    const uint64_t key0 = keys[0];
    auto cell_of = [&](uint64_t key) {   // largest c with keys[c] <= key (key >= key0)
        return (int)(std::upper_bound(keys.begin(), keys.end(), key) - keys.begin()) - 1;
    };
    std::vector<int> gd;
    for (int s = 63; s >= 0; --s) {
        const uint64_t nb = ((key_hi - key0) >> s) + 1;
        if (nb > kGuideMax) return;
        gd.assign(nb, 0);
        bool ok = true;
        for (uint64_t b = 0; b < nb && ok; ++b) {
            const uint64_t first = key0 + (b << s);
            gd[b] = cell_of(first);
            const int last = b + 1 < nb ? cell_of(first + ((((uint64_t)1) << s) - 1)) : ncell - 1;
            ok = last - gd[b] <= kGuideRun;
        }
        if (ok) {
            guide.swap(gd);
            *shift = s;
            return;
        }
    }
}

static int largest_pow2_below(int n)
{
    int s = 0;
    if (n >= 2) {
        s = 1;
        while (s * 2 <= n - 1) s *= 2;
    }
    return s;
}

// ------------------------------------------------- coefficient build kernel

// One thread per (member, Q cell, x cell, flavour): expand the bicubic patch
// C[n][m] = sum_r Mq[n][r] sum_i Mx[m][i] v[row r][knot i] over the 4x4
// stencil (rows outside the cell's subgrid and knots outside the x axis have
// zero weight and are not read).
__global__ void k_build_coef(GridDev g, const double *__restrict__ values, double *__restrict__ coef)
{
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t total = (int64_t)g.nmem * g.nqc * g.nxc * g.nflav;
    if (tid >= total) return;
    int a = (int)(tid % g.nflav);
    int64_t r = tid / g.nflav;
    int ix = (int)(r % g.nxc);
    r /= g.nxc;
    int c = (int)(r % g.nqc);
    int mem = (int)(r / g.nqc);
    const double *Mx = g.mx + (size_t)ix * 16;
    const double *Mq = g.mq + (size_t)c * 16;
    int qmask = g.qmask[c];
    int row0 = g.qrow[c] - 1;
    const double *vm = values + (size_t)mem * g.nrows * g.nx * g.nflav;
    double cx[4][4];
    for (int rr = 0; rr < 4; ++rr) {
        double gi[4];
        for (int i = 0; i < 4; ++i) {
            int k = ix - 1 + i;
            bool ok = ((qmask >> rr) & 1) && k >= 0 && k < g.nx;
            gi[i] = ok ? vm[((size_t)(row0 + rr) * g.nx + k) * g.nflav + a] : 0.0;
        }
        for (int m = 0; m < 4; ++m) {
            double s = 0.0;
            for (int i = 0; i < 4; ++i) s = fma(Mx[m * 4 + i], gi[i], s);
            cx[rr][m] = s;
        }
    }
    double *out = coef + (size_t)tid * 16;
    for (int n = 0; n < 4; ++n)
        for (int m = 0; m < 4; ++m) {
            double s = 0.0;
            for (int rr = 0; rr < 4; ++rr) s = fma(Mq[n * 4 + rr], cx[rr][m], s);
            out[n * 4 + m] = s;
        }
}

namespace pdfgpu {

int build_coefficients(pdfgpu_grid *g, const double *dev_values, cudaStream_t s)
{
    int64_t total = (int64_t)g->d.nmem * g->d.nqc * g->d.nxc * g->d.nflav;
    int block = 128;
    int64_t blocks = (total + block - 1) / block;
    k_build_coef<<<(unsigned)blocks, block, 0, s>>>(g->d, dev_values, const_cast<double *>(g->d.coef));
    PDF_CUDA(cudaGetLastError());
    g->bound = true;
    return PDF_OK;
}

}  // namespace pdfgpu

// --------------------------------------------------------------- the ABI

// Frees everything a grid handle owns.  Leaves the thread's error message
// alone, so that a failing pdf_load_grid keeps the message of the step that
// failed.
static void release_grid(pdfgpu_grid *g)
{
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    for (void *p : g->blocks) cudaFree(p);
    if (g->partials) cudaFree(g->partials);
    if (g->lumi_scratch) cudaFree(g->lumi_scratch);
    if (g->bwd_scratch) cudaFree(g->bwd_scratch);
    for (int s = 0; s < 3; ++s) {
        for (int k = 0; k < 3; ++k)
            if (g->stage[s][k]) cudaFree(g->stage[s][k]);
        if (g->hs[s]) cudaStreamDestroy(g->hs[s]);
    }
    delete g;
}

template <typename T>
static int dev_upload(pdfgpu_grid *g, const T *host, size_t count, const T **dst)
{
    void *p = nullptr;
    size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    int rc = dev_malloc(&p, bytes, "grid table");
    if (rc) return rc;
    g->blocks.push_back(p);
    if (count) PDF_CUDA(cudaMemcpy(p, host, count * sizeof(T), cudaMemcpyHostToDevice));
    *dst = (const T *)p;
    return PDF_OK;
}

#define TRY(x)                          \
    do {                                \
        int rc__ = (x);                 \
        if (rc__ != PDF_OK) {           \
            release_grid(g);            \
            return rc__;                \
        }                               \
    } while (0)

extern "C" int pdf_load_grid(const pdfgpu_grid_desc *desc, pdfgpu_grid_t *out)
{
    PDF_TRACE("pdf_load_grid");
    clear_error();
    if (!desc || !out) return fail(PDF_E_ARG, "null argument");
    *out = nullptr;
    const pdfgpu_grid_desc &D = *desc;
    if (D.n_x < 2 || !D.x_knots) return fail(PDF_E_DESC, "need at least 2 x knots");
    if (D.n_sub < 1 || !D.n_q || !D.q_knots) return fail(PDF_E_DESC, "need at least 1 Q subgrid");
    if (D.n_flav < 1 || D.n_flav > PDF_MAX_FLAV || !D.pids) return fail(PDF_E_DESC, "bad flavour count");
    if (D.n_members < 1) return fail(PDF_E_DESC, "need at least 1 member");
    if (D.interp < PDF_INTERP_LOGBICUBIC || D.interp > PDF_INTERP_LOGBICUBIC_SMALL_LINEAR)
        return fail(PDF_E_DESC, "unknown interpolation kind");
    if (D.extrap < PDF_EXTRAP_LINEAR || D.extrap > PDF_EXTRAP_CONTINUATION)
        return fail(PDF_E_DESC, "unknown extrapolation mode");
    for (int k = 0; k < D.n_x; ++k) {
        double x = D.x_knots[k];
        if (!(x > 0.0 && x <= 1.0)) return fail(PDF_E_DESC, "x knot outside (0, 1]");
        if (k && !(x > D.x_knots[k - 1])) return fail(PDF_E_DESC, "x knots not strictly ascending");
    }
    int rows = 0;
    for (int s = 0; s < D.n_sub; ++s) {
        if (D.n_q[s] < 2) return fail(PDF_E_DESC, "a Q subgrid has fewer than 2 knots");
        rows += D.n_q[s];
    }
    {
        int r = 0;
        for (int s = 0; s < D.n_sub; ++s) {
            for (int j = 0; j < D.n_q[s]; ++j) {
                double q = D.q_knots[r + j];
                if (!(q > 0.0 && q * q < INFINITY)) return fail(PDF_E_DESC, "Q knot not positive finite");
                if (j && !(q * q > D.q_knots[r + j - 1] * D.q_knots[r + j - 1]))
                    return fail(PDF_E_DESC, "Q knots not strictly ascending inside a subgrid");
            }
            if (s + 1 < D.n_sub && D.q_knots[r + D.n_q[s] - 1] != D.q_knots[r + D.n_q[s]])
                return fail(PDF_E_DESC, "threshold knot not duplicated between subgrids");
            r += D.n_q[s];
        }
    }
    bool gluon = false;
    for (int a = 0; a < D.n_flav; ++a) {
        int p = D.pids[a];
        if (p < -64 || p > 64) return fail(PDF_E_DESC, "pid outside [-64, 64]");
        if (p == 0 || p == 21) {
            if (gluon) return fail(PDF_E_DESC, "gluon listed twice");
            gluon = true;
        }
        for (int b = 0; b < a; ++b)
            if (D.pids[b] == p) return fail(PDF_E_DESC, "duplicate pid");
    }

    pdfgpu_grid *g = new pdfgpu_grid();
    if (cudaGetDevice(&g->device) != cudaSuccess) {
        delete g;
        return fail(PDF_E_CUDA, "no CUDA device");
    }
    cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device);
    g->n_q.assign(D.n_q, D.n_q + D.n_sub);
    for (int a = 0; a < D.n_flav; ++a) g->pids.push_back(D.pids[a] == 21 ? 0 : D.pids[a]);

    std::vector<LogEntry> ltab;
    std::vector<double2> etab;
    make_log_tables(ltab, etab);
    const int nx = D.n_x, nxc = nx - 1;
    g->U.resize(nx);
    for (int k = 0; k < nx; ++k) g->U[k] = tlog(D.x_knots[k], ltab.data(), etab.data());
    std::vector<double> Q2(rows);
    g->W.resize(rows);
    for (int r = 0; r < rows; ++r) {
        Q2[r] = D.q_knots[r] * D.q_knots[r];
        g->W[r] = tlog(Q2[r], ltab.data(), etab.data());
    }
    for (int k = 1; k < nx; ++k)
        if (!(g->U[k] > g->U[k - 1])) {
            delete g;
            return fail(PDF_E_DESC, "x knots too close (ln x not ascending)");
        }

    // x cells
    const bool x_linear = D.interp == PDF_INTERP_LOGBILINEAR ||
                          (D.interp == PDF_INTERP_LOGBICUBIC_SMALL_LINEAR && nx < 4);
    std::vector<uint64_t> xbits(nxc);
    std::vector<int64_t> ukey(nxc);
    std::vector<double2> xcell(nxc);
    std::vector<double> mx((size_t)nxc * 16), mxs((size_t)nxc * 16);
    for (int k = 0; k < nxc; ++k) {
        xbits[k] = dbits(D.x_knots[k]);
        ukey[k] = dkey(g->U[k]);
        xcell[k] = make_double2(g->U[k], 1.0 / (g->U[k + 1] - g->U[k]));
        cell_matrix(g->U.data(), nx, k, &mx[(size_t)k * 16], x_linear, &mxs[(size_t)k * 16]);
    }
    // Q cells, subgrid by subgrid
    std::vector<uint64_t> qbits;
    std::vector<int64_t> wkey;
    std::vector<double2> qcell;
    std::vector<double> mq, mqs;
    std::vector<int> qrow, qmask;
    {
        int r0 = 0;
        for (int s = 0; s < D.n_sub; ++s) {
            int n = D.n_q[s];
            const double *Ws = g->W.data() + r0;
            for (int j = 0; j + 1 < n; ++j) {
                if (!(Ws[j + 1] > Ws[j])) {
                    delete g;
                    return fail(PDF_E_DESC, "Q knots too close (ln Q^2 not ascending)");
                }
                qbits.push_back(dbits(Q2[r0 + j]));
                wkey.push_back(dkey(Ws[j]));
                qcell.push_back(make_double2(Ws[j], 1.0 / (Ws[j + 1] - Ws[j])));
                double M[16], Ms[16];
                const bool q_linear = D.interp == PDF_INTERP_LOGBILINEAR ||
                                      (D.interp == PDF_INTERP_LOGBICUBIC_SMALL_LINEAR && n < 4);
                cell_matrix(Ws, n, j, M, q_linear, Ms);
                mq.insert(mq.end(), M, M + 16);
                mqs.insert(mqs.end(), Ms, Ms + 16);
                qrow.push_back(r0 + j);
                int mask = 0x6 | (j > 0 ? 0x1 : 0) | (j + 2 <= n - 1 ? 0x8 : 0);
                qmask.push_back(mask);
            }
            r0 += n;
        }
    }
    const int nqc = (int)qbits.size();
    for (int c = 1; c < nqc; ++c)
        if (!(qbits[c] > qbits[c - 1])) {
            delete g;
            return fail(PDF_E_DESC, "Q cells overlap across subgrids");
        }

    std::vector<signed char> pidmap(129, -1);
    for (int a = 0; a < D.n_flav; ++a) {
        int p = g->pids[a];
        pidmap[p + 64] = (signed char)a;
        if (p == 0) pidmap[21 + 64] = (signed char)a;
    }

    GridDev &d = g->d;
    d.nx = nx;
    d.nxc = nxc;
    d.nqc = nqc;
    d.nrows = rows;
    d.nsub = D.n_sub;
    d.nflav = D.n_flav;
    d.nmem = D.n_members;
    d.xstep = largest_pow2_below(nxc);
    d.qstep = largest_pow2_below(nqc);
    std::vector<int> xguide, qguide;
    build_guide(xbits, dbits(D.x_knots[nx - 1]), xguide, &d.xgshift);
    build_guide(qbits, dbits(Q2[rows - 1]), qguide, &d.qgshift);
    d.nxg = (int)xguide.size();
    d.nqg = (int)qguide.size();
    d.xlo = dbits(D.x_knots[0]);
    d.xhi = dbits(D.x_knots[nx - 1]);
    d.qlo = dbits(Q2[0]);
    d.qhi = dbits(Q2[rows - 1]);
    d.ulo = dkey(g->U[0]);
    d.uhi = dkey(g->U[nx - 1]);
    d.wlo = dkey(g->W[0]);
    d.whi = dkey(g->W[rows - 1]);
    d.extrap = D.extrap;

    TRY(dev_upload(g, xbits.data(), xbits.size(), &d.xbits));
    TRY(dev_upload(g, ukey.data(), ukey.size(), &d.ukey));
    TRY(dev_upload(g, xcell.data(), xcell.size(), &d.xcell));
    TRY(dev_upload(g, qbits.data(), qbits.size(), &d.qbits));
    if (d.nxg) TRY(dev_upload(g, xguide.data(), xguide.size(), &d.xguide));
    if (d.nqg) TRY(dev_upload(g, qguide.data(), qguide.size(), &d.qguide));
    TRY(dev_upload(g, wkey.data(), wkey.size(), &d.wkey));
    TRY(dev_upload(g, qcell.data(), qcell.size(), &d.qcell));
    TRY(dev_upload(g, ltab.data(), ltab.size(), &d.logtab));
    TRY(dev_upload(g, etab.data(), etab.size(), &d.etab));
    TRY(dev_upload(g, mx.data(), mx.size(), &d.mx));
    TRY(dev_upload(g, mq.data(), mq.size(), &d.mq));
    TRY(dev_upload(g, mxs.data(), mxs.size(), &d.mxs));
    TRY(dev_upload(g, mqs.data(), mqs.size(), &d.mqs));
    TRY(dev_upload(g, qrow.data(), qrow.size(), &d.qrow));
    TRY(dev_upload(g, qmask.data(), qmask.size(), &d.qmask));
    TRY(dev_upload(g, pidmap.data(), pidmap.size(), &d.pidmap));
    {
        const uint32_t zero = 0;
        const uint32_t *st;
        TRY(dev_upload(g, &zero, 1, &st));
        d.status = const_cast<uint32_t *>(st);
    }
    if (D.alphas) {
        std::vector<double> ac((size_t)nqc * 4);
        for (int c = 0; c < nqc; ++c) {
            const double *M = &mq[(size_t)c * 16];
            for (int nn = 0; nn < 4; ++nn) {
                double s = 0.0;
                for (int rr = 0; rr < 4; ++rr) {
                    if (!((qmask[c] >> rr) & 1)) continue;
                    s = fma(M[nn * 4 + rr], D.alphas[qrow[c] - 1 + rr], s);
                }
                ac[(size_t)c * 4 + nn] = s;
            }
        }
        TRY(dev_upload(g, ac.data(), ac.size(), &d.acoef));
        g->has_alphas = true;
    }
    // coefficient storage
    size_t ncoef = (size_t)D.n_members * nqc * nxc * D.n_flav * 16;
    {
        void *p = nullptr;
        if (dev_malloc(&p, ncoef * sizeof(double), "coefficient table") != PDF_OK) {
            release_grid(g);
            return PDF_E_NOMEM;
        }
        g->blocks.push_back(p);
        d.coef = (const double *)p;
    }
    if (D.values) {
        size_t nval = (size_t)D.n_members * rows * nx * D.n_flav;
        void *p = nullptr;
        if (dev_malloc(&p, nval * sizeof(double), "value upload") != PDF_OK) {
            release_grid(g);
            return PDF_E_NOMEM;
        }
        cudaError_t e = cudaMemcpy(p, D.values, nval * sizeof(double), cudaMemcpyHostToDevice);
        int rc = e == cudaSuccess ? build_coefficients(g, (const double *)p, 0) : cuda_fail(e, "upload");
        if (rc == PDF_OK) {
            e = cudaDeviceSynchronize();
            if (e != cudaSuccess) rc = cuda_fail(e, "coefficient build");
        }
        cudaFree(p);
        if (rc != PDF_OK) {
            release_grid(g);
            return rc;
        }
    }
    *out = g;
    return PDF_OK;
}

extern "C" int pdf_bind_values(pdfgpu_grid_t g, const double *dev_values, pdfgpu_stream_t stream)
{
    PDF_TRACE("pdf_bind_values");
    clear_error();
    int rc = check_grid(g, false);
    if (rc) return rc;
    if (!dev_values) return fail(PDF_E_ARG, "null values");
    return build_coefficients(g, dev_values, (cudaStream_t)stream);
}

extern "C" int pdf_free_grid(pdfgpu_grid_t g)
{
    PDF_TRACE("pdf_free_grid");
    clear_error();
    if (!g) return fail(PDF_E_ARG, "null grid handle");
    release_grid(g);
    return PDF_OK;
}

extern "C" int pdf_grid_info(pdfgpu_grid_t g, int32_t *n_x, int32_t *n_rows, int32_t *n_flav,
                             int32_t *n_members, int32_t *has_alphas)
{
    PDF_TRACE("pdf_grid_info");
    clear_error();
    if (!g) return fail(PDF_E_ARG, "null grid handle");
    if (n_x) *n_x = g->d.nx;
    if (n_rows) *n_rows = g->d.nrows;
    if (n_flav) *n_flav = g->d.nflav;
    if (n_members) *n_members = g->d.nmem;
    if (has_alphas) *has_alphas = g->has_alphas ? 1 : 0;
    return PDF_OK;
}

extern "C" int pdf_get_status(pdfgpu_grid_t g, pdfgpu_stream_t stream, uint32_t *bits)
{
    PDF_TRACE("pdf_get_status");
    clear_error();
    int rc = check_grid(g, false);
    if (rc) return rc;
    if (!bits) return fail(PDF_E_ARG, "null output");
    cudaStream_t s = (cudaStream_t)stream;
    PDF_CUDA(cudaStreamSynchronize(s));
    uint32_t v = 0;
    PDF_CUDA(cudaMemcpy(&v, g->d.status, sizeof(v), cudaMemcpyDeviceToHost));
    PDF_CUDA(cudaMemset(g->d.status, 0, sizeof(uint32_t)));
    *bits = v;
    return PDF_OK;
}

extern "C" const char *pdf_last_error(void) { return pdfgpu::t_err.c_str(); }
