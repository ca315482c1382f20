// Shared device-side building blocks of the pdfgpu kernels.
//
// The interpolant (PDFFlow Sec. 2.1 and Sec. 4: LHAPDF-style log-bicubic with
// Q subgrids; formulas in include/pdfgpu.h) is stored per grid cell as the 16
// monomial coefficients C[n][m] of the bicubic patch in the local coordinates
// tx = (ln x - U_k)/dU_k and tq = (ln Q^2 - W_c)/dW_c.  These are the Hermite
// cubics with finite-difference knot derivatives, expanded once at load time,
// so a query costs two table lookups, two knot searches and 15 FP64 FMAs per
// flavour:   P = sum_n bq_n sum_m bx_m C[n][m],  b = (1, t, t^2, t^3).
// Outside the grid the basis becomes (1, t, t, t): that turns the edge patch
// into the linear continuation from its two edge knots (P(0) + t (P(1)-P(0))).
//
// The knot searches compare IEEE bit patterns as integers (the FP64 pipe of
// this GPU is ~60x slower than its integer pipes), and ln is a table-driven
// routine (Tang's method, ACM TOMS 16 (1990) 378) that costs 8 FP64
// operations instead of the ~36-slot library log.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "pdfgpu.h"

#if defined(__CUDACC__)
#define PDF_HD __host__ __device__ __forceinline__
#else
#define PDF_HD inline
#endif

namespace pdfgpu {

constexpr int kLogBits = 10;              // table index: top 10 mantissa bits
constexpr int kLogTab = 1 << kLogBits;
constexpr int kMaxStencilRows = 4;

PDF_HD uint64_t dbits(double x)
{
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
#endif
}

PDF_HD double dfrom(uint64_t b)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double x;
    memcpy(&x, &b, 8);
    return x;
#endif
}

// Signed-integer key with the same order as the double (both signs).
PDF_HD int64_t dkey(double x)
{
    int64_t b = (int64_t)dbits(x);
    return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFll);
}

// ln x for a positive, finite, normal double.
//   x = 2^e m, m in [1,2); j = top 10 bits of m; c_j = 1 + (j + 1/2)/1024,
//   except c_0 = 1 and c_1023 = 2 (so that ln is exact at 1 and accurate to
//   relative rounding on both sides of 1); tab[j] = (1/c_j rounded, and the
//   high and low parts of -ln of that reciprocal); r = m/c_j - 1 by one FMA
//   (|r| <= 2^-10); ln(1+r) = r - r^2/2 + r^3/3 - r^4/4 + r^5/5 (next term
//   < 2e-19); etab[biased e] = e ln 2 as high and low parts.  The result is
//   (E_hi + L_hi) + (p + (E_lo + L_lo)): the high parts cancel exactly where
//   they nearly cancel, and the error stays within about one unit in the
//   last place.  Both sides of the library (host tables, device kernels)
//   call this same routine, so knot logs and query logs agree bit for bit.
struct LogEntry {
    double inv_c, lhi, llo, pad;
};

PDF_HD double tlog(double x, const LogEntry *tab, const double2 *etab)
{
    uint64_t b = dbits(x);
    uint32_t eb = (uint32_t)(b >> 52);
    uint32_t j = (uint32_t)(b >> (52 - kLogBits)) & (kLogTab - 1);
    double m = dfrom((b & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull);
    const LogEntry &L = tab[j];
    const double2 E = etab[eb];
    double r = fma(m, L.inv_c, -1.0);
    double a = fma(r, 0.2, -0.25);
    a = fma(r, a, 1.0 / 3.0);
    a = fma(r, a, -0.5);
    double r2 = r * r;
    double p = fma(r2, a, r);
    double hi = E.x + L.lhi;
    double lo = p + (E.y + L.llo);
    return hi + lo;
}

// Device view of one loaded grid (passed by value to kernels).
struct GridDev {
    int nx, nxc;          // x knots, x cells (nx - 1)
    int nqc;              // Q cells over all subgrids
    int nrows, nsub, nflav, nmem;
    int xstep, qstep;     // search start steps (largest power of two < cells)
    int nxg, nqg;         // guide-table buckets per axis (0: no guide, binary search)
    int xgshift, qgshift; // log2 of the guide buckets' width in key units
    uint64_t xlo, xhi;    // bit patterns of the first / last x knot
    uint64_t qlo, qhi;    // bit patterns of the first / last Q^2 knot
    int64_t ulo, uhi;     // order keys of ln(first / last x knot)
    int64_t wlo, whi;     // order keys of ln(first / last Q^2 knot)
    const uint64_t *xbits;   // [nxc] bits of each x cell's lower knot
    const int64_t *ukey;     // [nxc] order keys of each x cell's lower ln x
    const double2 *xcell;    // [nxc] (U_k, 1/dU_k)
    const uint64_t *qbits;   // [nqc] bits of each Q cell's lower Q^2 knot
    const int *xguide;       // [nxg] first cell of each x guide bucket
    const int *qguide;       // [nqg] the same for Q^2
    const int64_t *wkey;     // [nqc] order keys of each Q cell's lower ln Q^2
    const double2 *qcell;    // [nqc] (W_c, 1/dW_c)
    const LogEntry *logtab;  // [kLogTab]
    const double2 *etab;     // [2048] (hi, lo) of e ln 2
    const double *coef;      // [nmem][nqc][nxc][nflav][16]
    const double *acoef;     // [nqc][4] alpha_s cubic in tq, or null
    const double *mx;        // [nxc][16] stencil -> monomial matrix M[m][i]
    const double *mq;        // [nqc][16]
    const double *mxs;       // [nxc][16] the same in powers of s = 1 - t
    const double *mqs;       // [nqc][16]
    const int *qrow;         // [nqc] grid row of each Q cell's lower knot
    const int *qmask;        // [nqc] bit i (0..3): stencil row i-1 exists
    const signed char *pidmap;  // [129] column of pid in [-64, 64], -1 absent
    uint32_t *status;
    int extrap;              // PDF_EXTRAP_*
};

// Largest cell c in [0, ncell) whose lower key is <= key (0 below the grid).
// Tables are read with generic loads: they may sit in global or shared memory.
template <typename K>
__device__ __forceinline__ int find_cell(const K *keys, int ncell, int step, K key)
{
    int lo = 0;
    for (int s = step; s > 0; s >>= 1) {
        int c = lo + s;
        if (c < ncell && keys[c] <= key) lo = c;
    }
    return lo;
}

// The same search through a guide table: bucket b covers the keys
// key0 + [b 2^shift, (b + 1) 2^shift) (the last bucket also everything
// above) and holds the largest cell whose lower key is <= the bucket's first
// key; the host builds the table so that no bucket holds more than
// kGuideRun further lower keys.  The cell of a key is then the bucket's cell
// plus the number of the next kGuideRun lower keys that are <= it (the keys
// ascend): one table load and kGuideRun independent key loads, instead of a
// chain of log2(cells) dependent ones.  Without a table (nguide == 0) the
// binary search.
constexpr int kGuideRun = 3;

__device__ __forceinline__ int find_cell_guided(const uint64_t *keys, int ncell, int step, const int *guide,
                                                int nguide, int shift, uint64_t key0, uint64_t key)
{
    if (nguide == 0) return find_cell<uint64_t>(keys, ncell, step, key);
    if (key < key0) return 0;
    const uint64_t off = (key - key0) >> shift;
    const int c = __ldg(guide + (off < (uint64_t)nguide ? (int)off : nguide - 1));
    int add = 0;
#pragma unroll
    for (int r = 1; r <= kGuideRun; ++r) add += (c + r < ncell && keys[c + r] <= key) ? 1 : 0;
    return c + add;
}

// Checked builds (-DPDFGPU_CHECKED, the library built with PDFGPU_CHECKED=1):
// table indices computed on the device are tested before use; one out of
// range sets PDF_S_BOUNDS in the grid's status word and is replaced by 0, so
// that no access leaves its array (the result is then wrong, and the status
// says so).  Release builds compile the tests away.
#ifdef PDFGPU_CHECKED
__device__ __forceinline__ int checked_index(unsigned *status, int i, int n)
{
    if (i >= 0 && i < n) return i;
    atomicOr(status, (unsigned)PDF_S_BOUNDS);
    return 0;
}
#else
__device__ __forceinline__ int checked_index(unsigned *, int i, int) { return i; }
#endif

// Per-axis local coordinate and basis of one query.
struct Axis {
    int cell;
    double t, b2, b3;     // basis (1, t, b2, b3)
    double h;             // Horner factor: t inside, 1 outside
    bool in;              // inside the knot range
    bool below;           // below the first knot
};

// Basis of the patch polynomial along one axis.  Inside the knot range
// (1, t, t^2, t^3).  Outside: linear continuation (1, t, t, t), i.e.
// P(0) + t (P(1) - P(0)); frozen at the edge, t becomes 0 (below) or 1
// (above), the edge knot of the edge cell.  The error mode is handled by the
// caller (the point is flagged, the basis does not matter).
__device__ __forceinline__ void make_basis(Axis &A, double t, int extrap)
{
    if (!A.in && extrap == PDF_EXTRAP_FREEZE) t = A.below ? 0.0 : 1.0;
    A.t = t;
    double t2 = t * t;
    double t3 = t2 * t;
    A.b2 = A.in ? t2 : t;
    A.b3 = A.in ? t3 : t;
    A.h = A.in ? t : 1.0;
}

// c0 + c1 t + c2 b2 + c3 b3 by Horner's rule, c0 + t (c1 + h (c2 + h c3)):
// 3 FMAs and no powers of t (outside, h = 1 gives c0 + t (c1 + c2 + c3)).
__device__ __forceinline__ double horner(const Axis &A, double c0, double c1, double c2, double c3)
{
    return fma(A.t, fma(A.h, fma(A.h, c3, c2), c1), c0);
}

// Domain checks on bit patterns: x in (0, 1], Q^2 in (0, max finite].
__device__ __forceinline__ bool x_ok(uint64_t b) { return b - 1ull < 0x3FF0000000000000ull; }
__device__ __forceinline__ bool q2_ok(uint64_t b) { return b - 1ull < 0x7FEFFFFFFFFFFFFFull; }

// ln for any positive finite double (subnormals rescaled; rare path).
__device__ __forceinline__ double dlog(const GridDev &g, double v)
{
    if (dbits(v) < 0x0010000000000000ull) {
        return tlog(v * 18014398509481984.0 /* 2^54 */, g.logtab, g.etab) -
               37.4299477502370467085305 /* 54 ln 2 */;
    }
    return tlog(v, g.logtab, g.etab);
}

// x axis from x (bit search on x), returns u = ln x in *u.
__device__ __forceinline__ Axis axis_x(const GridDev &g, double x, double *u)
{
    uint64_t b = dbits(x);
    Axis A;
    A.cell = checked_index(g.status, find_cell_guided(g.xbits, g.nxc, g.xstep, g.xguide, g.nxg, g.xgshift, g.xlo, b),
                           g.nxc);
    A.in = (b >= g.xlo) & (b <= g.xhi);
    A.below = b < g.xlo;
    double uu = dlog(g, x);
    double2 c = g.xcell[A.cell];
    make_basis(A, (uu - c.x) * c.y, g.extrap);
    *u = uu;
    return A;
}

// x axis from u = ln x directly (order-key search on u).
__device__ __forceinline__ Axis axis_u(const GridDev &g, double u)
{
    int64_t k = dkey(u);
    Axis A;
    A.cell = checked_index(g.status, find_cell<int64_t>(g.ukey, g.nxc, g.xstep, k), g.nxc);
    A.in = (k >= g.ulo) & (k <= g.uhi);
    A.below = k < g.ulo;
    double2 c = g.xcell[A.cell];
    make_basis(A, (u - c.x) * c.y, g.extrap);
    return A;
}

__device__ __forceinline__ Axis axis_q2(const GridDev &g, double q2, double *w)
{
    uint64_t b = dbits(q2);
    Axis A;
    A.cell = checked_index(g.status, find_cell_guided(g.qbits, g.nqc, g.qstep, g.qguide, g.nqg, g.qgshift, g.qlo, b),
                           g.nqc);
    A.in = (b >= g.qlo) & (b <= g.qhi);
    A.below = b < g.qlo;
    double ww = dlog(g, q2);
    double2 c = g.qcell[A.cell];
    make_basis(A, (ww - c.x) * c.y, g.extrap);
    *w = ww;
    return A;
}

__device__ __forceinline__ Axis axis_w(const GridDev &g, double w)
{
    int64_t k = dkey(w);
    Axis A;
    A.cell = checked_index(g.status, find_cell<int64_t>(g.wkey, g.nqc, g.qstep, k), g.nqc);
    A.in = (k >= g.wlo) & (k <= g.whi);
    A.below = k < g.wlo;
    double2 c = g.qcell[A.cell];
    make_basis(A, (w - c.x) * c.y, g.extrap);
    return A;
}

// Four consecutive doubles in one 32-byte read-only load (sm_100 and later).
// The address must be 32-byte aligned: every coefficient block and cell
// matrix is 128 B long and starts at a multiple of 128 B from a cudaMalloc
// base.
struct D4 {
    double x, y, z, w;
};
__device__ __forceinline__ D4 ld4(const double *p)
{
    D4 v;
    asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(v.x), "=d"(v.y), "=d"(v.z), "=d"(v.w) : "l"(p));
    return v;
}

// 16-coefficient patch contraction: 15 FP64 FMAs (Horner along x in each
// row, then along Q).  C[4n + m] multiplies tx^m tq^n: row n of the block is
// one 32-byte load.
__device__ __forceinline__ double patch(const double *__restrict__ C, const Axis &X, const Axis &Q)
{
    D4 r0 = ld4(C), r1 = ld4(C + 4), r2 = ld4(C + 8), r3 = ld4(C + 12);
    double i0 = horner(X, r0.x, r0.y, r0.z, r0.w);
    double i1 = horner(X, r1.x, r1.y, r1.z, r1.w);
    double i2 = horner(X, r2.x, r2.y, r2.z, r2.w);
    double i3 = horner(X, r3.x, r3.y, r3.z, r3.w);
    return horner(Q, i0, i1, i2, i3);
}

// LHAPDF-style continuation from the values y0, y1 at the lower and upper
// knot of an edge interval to the position t in it (t < 0 or t > 1): the
// power law y0^(1-t) y1^t when both values exceed kContMin, else the straight
// line (no logarithm of a value that is not clearly positive).
constexpr double kContMin = 1e-3;
__device__ __forceinline__ double cont(double y0, double y1, double t)
{
    if (y0 > kContMin && y1 > kContMin) return y0 * exp(t * log(y1 / y0));
    return fma(t, y1 - y0, y0);
}

// A patch outside the knot range under PDF_EXTRAP_CONTINUATION.  The patch
// of the edge cell restricted to tq = 0 / 1 (or tx = 0 / 1) is the
// interpolant along the lower / upper knot of that cell, so the edge values
// come from the same 16 coefficients: Q is continued first (per edge x
// column in a corner), then x.
__device__ inline double patch_cont(const double *__restrict__ C, const Axis &X, const Axis &Q)
{
    D4 r0 = ld4(C), r1 = ld4(C + 4), r2 = ld4(C + 8), r3 = ld4(C + 12);
    if (X.in) {   // Q out of range: rows tq = 0 and tq = 1 at tx
        double i0 = horner(X, r0.x, r0.y, r0.z, r0.w);
        double i1 = horner(X, r1.x, r1.y, r1.z, r1.w);
        double i2 = horner(X, r2.x, r2.y, r2.z, r2.w);
        double i3 = horner(X, r3.x, r3.y, r3.z, r3.w);
        return cont(i0, i0 + i1 + i2 + i3, Q.t);
    }
    // the column sums give the tx = 1 edge; column 0 the tx = 0 edge
    const double s0 = r0.x + r0.y + r0.z + r0.w, s1 = r1.x + r1.y + r1.z + r1.w;
    const double s2 = r2.x + r2.y + r2.z + r2.w, s3 = r3.x + r3.y + r3.z + r3.w;
    double a0, a1;
    if (Q.in) {
        a0 = horner(Q, r0.x, r1.x, r2.x, r3.x);
        a1 = horner(Q, s0, s1, s2, s3);
    } else {
        a0 = cont(r0.x, r0.x + r1.x + r2.x + r3.x, Q.t);
        a1 = cont(s0, s0 + s1 + s2 + s3, Q.t);
    }
    return cont(a0, a1, X.t);
}

// Value of a patch under the grid's extrapolation option.  Kernels are
// instantiated with CONT = false for launches on grids without the
// continuation option, so that the common path carries none of its code.
template <bool CONT>
__device__ __forceinline__ double patch_any(const GridDev &g, const double *__restrict__ C, const Axis &X,
                                            const Axis &Q)
{
    if (CONT && g.extrap == PDF_EXTRAP_CONTINUATION && !(X.in && Q.in)) return patch_cont(C, X, Q);
    return patch(C, X, Q);
}

// alpha_s from the 4 cubic coefficients of its Q cell, under the grid's
// extrapolation option.
__device__ __forceinline__ double alphas_any(const GridDev &g, const D4 &a, const Axis &Q)
{
    if (g.extrap == PDF_EXTRAP_CONTINUATION && !Q.in) return cont(a.x, a.x + a.y + a.z + a.w, Q.t);
    return horner(Q, a.x, a.y, a.z, a.w);
}

// Value and derivative in t of one cubic by Horner's rule: the value
// c0 + t B1 with B1 = c1 + h B2, B2 = c2 + h c3 (the operations of horner(),
// so the same bits), and the derivative B1 + g (B2 + g c3): with g = h = t
// inside the knot range that is c1 + 2 c2 t + 3 c3 t^2; outside, g = 0 and
// the derivative of the linear basis (1, t, t, t) is B1 = c1 + c2 + c3.
// Two FMAs beyond the value.
struct VD {
    double v, d;
};
__device__ __forceinline__ VD horner_vd(const Axis &A, double c0, double c1, double c2, double c3)
{
    const double b2 = fma(A.h, c3, c2);
    const double b1 = fma(A.h, b2, c1);
    const double gt = A.in ? A.t : 0.0;
    return {fma(A.t, b1, c0), fma(gt, fma(gt, c3, b2), b1)};
}

// A patch and its derivatives in t_x and t_q in one pass over its four
// coefficient rows: each row's value i_n and t_x-derivative j_n, then the
// value and the t_q-derivative from the i_n and the t_x-derivative by
// Horner's rule over the j_n.  The value is patch()'s, bit for bit; the
// two derivatives cost 13 FMAs beyond it (28 in all).  Every adjoint takes
// its patch derivatives from here, so that derivatives kept by a forward
// pass and derivatives recomputed later are the same bits.
__device__ __forceinline__ double patch_vd_rows(const D4 r[4], const Axis &X, const Axis &Q, double *dtx,
                                                double *dtq)
{
    VD row[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) row[n] = horner_vd(X, r[n].x, r[n].y, r[n].z, r[n].w);
    const VD q = horner_vd(Q, row[0].v, row[1].v, row[2].v, row[3].v);
    *dtx = horner(Q, row[0].d, row[1].d, row[2].d, row[3].d);
    *dtq = q.d;
    return q.v;
}

__device__ __forceinline__ double patch_vd(const double *__restrict__ C, const Axis &X, const Axis &Q, double *dtx,
                                           double *dtq)
{
    const D4 r[4] = {ld4(C), ld4(C + 4), ld4(C + 8), ld4(C + 12)};
    return patch_vd_rows(r, X, Q, dtx, dtq);
}

// Stencil weights of one axis (i <-> knot cell-1+i): W_i = sum_m M[m][i] t^m
// in the lower half of the cell, sum_m Ms[m][i] s^m with s = 1 - t in the
// upper half (Ms: the cell's matrix in powers of s), so that a weight that
// vanishes at the near knot comes out of small powers, not of cancelling
// ones.  Outside the knot range the exact weights of the linear
// continuation, (1 - t, t) on the cell's two knots.
__device__ __forceinline__ void stencil_weights(const double *__restrict__ M, const double *__restrict__ Ms,
                                                const Axis &A, double W[4])
{
    if (!A.in) {
        W[0] = 0.0;
        W[1] = 1.0 - A.t;
        W[2] = A.t;
        W[3] = 0.0;
        return;
    }
    const bool up = dbits(A.t) > 0x3FE0000000000000ull;   // t > 1/2 (t >= 0 inside)
    const double *P = up ? Ms : M;
    const double z = up ? 1.0 - A.t : A.t, z2 = z * z, z3 = z2 * z;
    D4 r0 = ld4(P), r1 = ld4(P + 4), r2 = ld4(P + 8), r3 = ld4(P + 12);
    W[0] = fma(z3, r3.x, fma(z2, r2.x, fma(z, r1.x, r0.x)));
    W[1] = fma(z3, r3.y, fma(z2, r2.y, fma(z, r1.y, r0.y)));
    W[2] = fma(z3, r3.z, fma(z2, r2.z, fma(z, r1.z, r0.z)));
    W[3] = fma(z3, r3.w, fma(z2, r2.w, fma(z, r1.w, r0.w)));
}

// Bulk copy (TMA engine) of `bytes` from shared to global memory: both
// addresses 16-byte aligned, bytes a multiple of 16.  The shared source may be
// rewritten once bulk_wait_read() has returned in the issuing thread.
__device__ __forceinline__ void bulk_store(double *dst, const double *src, unsigned bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n\t"
                 "cp.async.bulk.commit_group;" ::"l"(dst),
                 "r"((unsigned)__cvta_generic_to_shared(src)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Orders this thread's shared-memory writes before later bulk copies.
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// A warp's staged run of `cnt` doubles at `wbuf` (shared) goes to `dst`:
// one bulk copy issued by lane 0 when both ends allow it, else coalesced
// stores by the whole warp.  The caller has written wbuf (each lane its own
// rows) and, before rewriting it, calls warp_run_reuse().
__device__ __forceinline__ void warp_run_store(double *dst, const double *wbuf, int cnt, int lane)
{
    if (((reinterpret_cast<uintptr_t>(dst) | (uintptr_t)(cnt * 8)) & 15) == 0) {
        fence_smem_to_async();
        __syncwarp();
        if (lane == 0) bulk_store(dst, wbuf, (unsigned)cnt * 8u);
    } else {
        __syncwarp();
        for (int k = lane; k < cnt; k += 32) dst[k] = wbuf[k];
        __syncwarp();
    }
}
// The warp's staging slice may be rewritten after this returns.
__device__ __forceinline__ void warp_run_reuse(int lane)
{
    if (lane == 0) bulk_wait_read();
    __syncwarp();
}

__device__ __forceinline__ void flag_status(const GridDev &g, bool bad, unsigned bit = PDF_S_DOMAIN)
{
    unsigned m = __ballot_sync(__activemask(), bad);
    if (m && (threadIdx.x & 31) == (unsigned)(__ffs(m) - 1)) atomicOr(g.status, bit);
}

// Outside the knot range of a grid that asks for NaN there.
__device__ __forceinline__ bool out_of_range(const GridDev &g, const Axis &X, const Axis &Q)
{
    return g.extrap == PDF_EXTRAP_ERROR && !(X.in && Q.in);
}

// Adjoint tape: 32 bytes per point that a forward pass keeps for the adjoint
// of the same points, so that the adjoint skips the domain checks, both knot
// searches and both logarithms.  Layout (four doubles, 32-byte aligned):
//   [0] t of the x axis, [1] t of the Q axis (after make_basis),
//   [2] bits: x cell (low 32) and Q cell (high 32),
//   [3] bits: 1 x inside, 2 x below, 4 Q inside, 8 Q below, 16 bad point
//       (domain error, or outside the grid under the error option), 32 t of
//       the x axis above 1/2, 64 t of the Q axis above 1/2.
// It depends on the points, the knots and the extrapolation option only (not
// on the member or the values), so it stays valid across pdf_bind_values.
constexpr unsigned kTapeBad = 16u;

// t > 1/2 for a t in [0, 1] (inside the knot range), as an integer compare of
// its bit pattern (which keeps the FP64 pipe free).
__device__ __forceinline__ bool upper_half(double t) { return dbits(t) > 0x3FE0000000000000ull; }

__device__ __forceinline__ void tape_put(double *__restrict__ tape, int64_t i, const Axis &X, const Axis &Q,
                                         bool bad)
{
    const unsigned f = (X.in ? 1u : 0u) | (X.below ? 2u : 0u) | (Q.in ? 4u : 0u) | (Q.below ? 8u : 0u) |
                       (bad ? kTapeBad : 0u) | (upper_half(X.t) ? 32u : 0u) | (upper_half(Q.t) ? 64u : 0u);
    double2 *d = reinterpret_cast<double2 *>(tape + 4 * i);
    d[0] = make_double2(X.t, Q.t);
    d[1] = make_double2(dfrom((uint64_t)(uint32_t)X.cell | ((uint64_t)(uint32_t)Q.cell << 32)),
                        dfrom((uint64_t)f));
}

// A cell read back from a tape: range-checked (and flagged) in checked
// builds, clamped into the table otherwise, so that a tape from another grid
// gives wrong numbers but no access outside the tables.
__device__ __forceinline__ int tape_cell(unsigned *status, uint32_t v, int n)
{
#ifdef PDFGPU_CHECKED
    return checked_index(status, (int)v, n);
#else
    (void)status;
    return (int)min(v, (uint32_t)(n - 1));
#endif
}

// Cells and range flags of a tape record from its second half (cells, flag
// bits); returns whether the point is bad.
__device__ __forceinline__ bool tape_decode(const GridDev &g, double cells_bits, double flag_bits, Axis &X,
                                            Axis &Q, unsigned *halves = nullptr)
{
    const uint64_t cells = dbits(cells_bits);
    const unsigned f = (unsigned)dbits(flag_bits);
    X.cell = tape_cell(g.status, (uint32_t)cells, g.nxc);
    Q.cell = tape_cell(g.status, (uint32_t)(cells >> 32), g.nqc);
    X.in = f & 1u;
    X.below = f & 2u;
    Q.in = f & 4u;
    Q.below = f & 8u;
    if (halves) *halves = (f >> 5) & 3u;
    return f & kTapeBad;
}

// The half of point i's tape record that holds the cells and the flags (for
// tape_decode), from one 16-byte load.
__device__ __forceinline__ double2 tape_cells_raw(const double *__restrict__ tape, int64_t i)
{
    return __ldg(reinterpret_cast<const double2 *>(tape + 4 * i + 2));
}

// Rebuilds the two axes of point i from its tape record; returns whether the
// point is bad.
__device__ __forceinline__ bool tape_get(const GridDev &g, const double *__restrict__ tape, int64_t i, Axis &X,
                                         Axis &Q)
{
    const D4 r = ld4(tape + 4 * i);
    const bool bad = tape_decode(g, r.z, r.w, X, Q);
    make_basis(X, r.x, g.extrap);
    make_basis(Q, r.y, g.extrap);
    return bad;
}

__device__ __forceinline__ int pid_col(const GridDev &g, int pid)
{
    int col = (pid >= -64 && pid <= 64) ? (int)__ldg(g.pidmap + pid + 64) : -1;
    return col < 0 ? col : checked_index(g.status, col, g.nflav);
}

}  // namespace pdfgpu
