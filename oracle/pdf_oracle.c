/*
 * Plain FP64 CPU oracle for batched PDF and alpha_s interpolation.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled and called by the test
 * suite, by the smoke check and by the benchmark's CPU-baseline arm.  The
 * library under test never links, imports or calls it, and it shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it computes (PDFFlow, Sec. 2.1: a flavour set {a} plus equal-length
 * arrays x_i, Q_i in, interpolated values out; alpha_s(Q) interpolated the same
 * way; Sec. 4: the LHAPDF data layout and interpolation algorithms):
 *
 *   x*f_a(x, Q^2) by log-bicubic interpolation on a grid of knot values, in
 *   the coordinates u = ln x and w = ln Q^2, with Q knots split into subgrids
 *   at flavour thresholds.  The paper names the method but does not print its
 *   formulas; this oracle fixes them as follows, in the order it evaluates:
 *
 *   1. Domain: x <= 0, x > 1, Q^2 <= 0, Q^2 infinite or NaN -> NaN.  Then the
 *      flavour: pid 21 means the gluon, pid 0, in a query and in the grid's
 *      flavour list; a pid absent from the grid -> 0.
 *   2. Knot derivative of data g on knots z_0..z_{n-1}: one-sided secant at the
 *      first and last knot, mean of the two adjacent secants inside.
 *   3. Cubic Hermite on [z_k, z_{k+1}] with t = (z - z_k)/dz:
 *      H = (2t^3-3t^2+1) g_k + (t^3-2t^2+t) dz D_k + (-2t^3+3t^2) g_{k+1}
 *          + (t^3-t^2) dz D_{k+1}.
 *   4. In range: every Q row r of the subgrid near w is interpolated in u
 *      (steps 2-3 along x); the row results R_r are then interpolated in w by
 *      steps 2-3 applied to the sequence R over the subgrid's own knots.  No
 *      row of another subgrid is ever used.
 *   5. Subgrid: the one whose knots enclose w; w equal to an internal
 *      threshold belongs to the upper subgrid.  Interval: the largest k with
 *      z_k <= z, clamped to n-2.
 *   6. Out of range, linear continuation in the log coordinates from the two
 *      edge knots: in u from the first (last) two x columns, each first
 *      interpolated in w; in w from the first (last) two rows of the lowest
 *      (highest) subgrid, each first interpolated (or continued) in u.
 *   7. alpha_s: step 5 then steps 2-3 in w on the alpha_s knot values, and
 *      step 6 at both ends (or the grid's extrapolation option below).
 *   8. Derivatives: d/du and d/dw of the same piecewise polynomial; the
 *      derivative with respect to one grid value is the interpolation of the
 *      indicator grid of that value (the result is linear in the values).
 *   Variants (grid options): log-bilinear interpolation (straight lines
 *   between the two interval knots on both axes), or log-bicubic with
 *   straight lines on any axis or subgrid of fewer than 4 knots; outside the
 *   grid, the value frozen at the nearest edge (u and w clamped into the
 *   knot range, zero derivative across the edge), NaN, or an LHAPDF-style
 *   continuation: from the same two values as step 6, y0 and y1 at the lower
 *   and upper knot of the edge interval, with t the position in that interval
 *   (t < 0 below the grid, t > 1 above), the power law y0^(1-t) y1^t in the
 *   log coordinate when both values exceed 1e-3, else step 6's straight line
 *   (sign-safe: no logarithm of a value that is not clearly positive).  The w
 *   direction is continued first (per edge column when u is out of range
 *   too), then u.
 *
 * Pins: every step above is checked by the test suite against closed forms,
 * invariants, an exact-rational brute force and central differences.  The
 * one thing no pin can fix is the *choice* of the rules outside the grid
 * (step 6 and its options): the paper is silent there, so that choice is
 * parity unpinned; its implementation is pinned (linear and power-law data
 * reproduced exactly, continuity at the edge).
 *
 * Built with -O2 -ffp-contract=off (no fused multiply-add contraction, no
 * fast-math), parallelised over points with OpenMP in the batch drivers only.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

typedef struct {
    int n_x;                 /* x knots, ascending, 0 < x <= 1            */
    const double *x_knots;
    int n_sub;               /* number of Q subgrids                      */
    const int *n_q;          /* knots per subgrid (>= 2)                  */
    const double *q_knots;   /* Q (GeV), subgrid after subgrid            */
    int n_flav;
    const int *pids;
    int n_members;
    const double *values;    /* [n_members][rows][n_x][n_flav] of x*f     */
    const double *alphas;    /* [rows] or NULL                            */
    /* derived by orc_init into caller storage */
    double *U;               /* [n_x]   ln x_k                             */
    double *W;               /* [rows]  ln (Q_r * Q_r)                     */
    int *row0;               /* [n_sub] first row of each subgrid         */
    int rows;
    int interp;              /* 0 log-bicubic, 1 log-bilinear, 2 log-bicubic
                                with linear axes that have fewer than 4 knots */
    int extrap;              /* outside the grid: 0 linear continuation,
                                1 freeze at the edge, 2 NaN, 3 power-law
                                continuation (linear where not positive)   */
} orc_grid;

int orc_init(orc_grid *g)
{
    if (g->n_x < 2 || g->n_sub < 1 || g->n_flav < 1) return -1;
    int r = 0;
    for (int s = 0; s < g->n_sub; ++s) {
        if (g->n_q[s] < 2) return -2;
        g->row0[s] = r;
        r += g->n_q[s];
    }
    g->rows = r;
    for (int k = 0; k < g->n_x; ++k) g->U[k] = log(g->x_knots[k]);
    for (int k = 0; k < r; ++k) g->W[k] = log(g->q_knots[k] * g->q_knots[k]);
    return 0;
}

/* ---- value access: a grid column, or the indicator grid of one cell ---- */

typedef struct {
    const orc_grid *g;
    const double *base;      /* values of one member, or alphas             */
    int stride_row, stride_k;
    int ind_row, ind_k;      /* >= 0: indicator mode                         */
} acc_t;

static double val(const acc_t *a, int row, int k)
{
    if (a->ind_row >= 0) return (row == a->ind_row && k == a->ind_k) ? 1.0 : 0.0;
    return a->base[(size_t)row * a->stride_row + (size_t)k * a->stride_k];
}

/* Step 2: knot derivative at local knot k of n, from neighbour values. */
static double fd_deriv(int k, int n, const double *z, double gm, double g0, double gp)
{
    if (k == 0) return (gp - g0) / (z[1] - z[0]);
    if (k == n - 1) return (g0 - gm) / (z[n - 1] - z[n - 2]);
    return 0.5 * ((gp - g0) / (z[k + 1] - z[k]) + (g0 - gm) / (z[k] - z[k - 1]));
}

/* Step 3: Hermite value and d/dz on [z0, z0+dz]. */
static double hermite(double t, double dz, double g0, double g1, double d0, double d1,
                      double *ddz)
{
    /* the four basis polynomials in factored form, (2t^3 - 3t^2 + 1) =
     * (1-t)^2 (1+2t) and so on: the same cubics, each accurate to rounding
     * relative to itself near both knots (no cancellation of O(1) terms) */
    double s = 1.0 - t, t2 = t * t, s2 = s * s;
    double h00 = s2 * (1.0 + 2.0 * t);
    double h10 = t * s2;
    double h01 = t2 * (3.0 - 2.0 * t);
    double h11 = -t2 * s;
    if (ddz) {
        double e00 = -6.0 * t * s;
        double e10 = s * (1.0 - 3.0 * t);
        double e01 = 6.0 * t * s;
        double e11 = t * (3.0 * t - 2.0);
        *ddz = (e00 * g0 + e10 * dz * d0 + e01 * g1 + e11 * dz * d1) / dz;
    }
    return h00 * g0 + h10 * dz * d0 + h01 * g1 + h11 * dz * d1;
}

/* Step 5: largest k in [0, n-2] with z_k <= v (clamped). */
static int interval(const double *z, int n, double v)
{
    int k = 0;
    for (int j = 0; j < n; ++j)
        if (z[j] <= v) k = j;
    if (k > n - 2) k = n - 2;
    return k;
}

/* Step 6 with option 3: continuation from y0 and y1, the values at the
 * lower and upper knot of the edge interval of width dz, to the offset off
 * from the lower knot (t = off / dz).  A power law y0^(1-t) y1^t when both
 * values exceed CONT_MIN, else step 6's straight line (the same expression).
 * *doff gets dy/d(off), *d0 and *d1 get dy/dy0 and dy/dy1. */
#define CONT_MIN 1e-3
static double cont(double y0, double y1, double off, double dz, double *doff, double *d0, double *d1)
{
    double t = off / dz;
    if (y0 > CONT_MIN && y1 > CONT_MIN) {
        double lr = log(y1 / y0);
        double y = y0 * exp(t * lr);
        *doff = y * lr / dz;
        *d0 = y * (1.0 - t) / y0;
        *d1 = y * t / y1;
        return y;
    }
    *doff = (y1 - y0) / dz;
    *d0 = 1.0 - t;
    *d1 = t;
    return y0 + off * (y1 - y0) / dz;
}

/* How one Q row is reduced to a number: Hermite in u, or one x column. */
typedef struct {
    int column;    /* >= 0: take this x column as is                 */
    double u;
} xsel_t;

/* Row value and its u-derivative (step 4 along x, step 6 never here). */
static double xrow(const acc_t *a, int row, const xsel_t *xs, double *du)
{
    const orc_grid *g = a->g;
    if (xs->column >= 0) {
        if (du) *du = 0.0;
        return val(a, row, xs->column);
    }
    int n = g->n_x, k = interval(g->U, n, xs->u);
    if (g->interp == 1 || (g->interp == 2 && n < 4)) {
        /* straight line between the interval's two knots */
        double g0 = val(a, row, k), g1 = val(a, row, k + 1);
        double dz = g->U[k + 1] - g->U[k];
        double t = (xs->u - g->U[k]) / dz;
        if (du) *du = (g1 - g0) / dz;
        return (1.0 - t) * g0 + t * g1;
    }
    double gm = k > 0 ? val(a, row, k - 1) : 0.0;
    double g0 = val(a, row, k), g1 = val(a, row, k + 1);
    double gp = k + 2 < n ? val(a, row, k + 2) : 0.0;
    double d0 = fd_deriv(k, n, g->U, gm, g0, g1);
    double d1 = fd_deriv(k + 1, n, g->U, g0, g1, gp);
    double dz = g->U[k + 1] - g->U[k];
    double t = (xs->u - g->U[k]) / dz;
    return hermite(t, dz, g0, g1, d0, d1, du);
}

/* Steps 4-6 along w for a given row reduction.  Returns the value; *dw gets
 * d/dw and *du the u-derivative (carried linearly through the w step). */
static double wdir(const acc_t *a, const xsel_t *xs, double w, double *dw, double *du)
{
    const orc_grid *g = a->g;
    const double *W = g->W;
    int last = g->rows - 1;
    int frozen = 0;
    if ((w < W[0] || w > W[last]) && g->extrap == 1) {
        w = w < W[0] ? W[0] : W[last];
        frozen = 1;
    }
    if (w < W[0] || w > W[last]) {
        /* step 6 in w: the two edge rows of the lowest or highest subgrid */
        int r0 = w < W[0] ? 0 : last - 1;
        double du0, du1;
        double B0 = xrow(a, r0, xs, &du0), B1 = xrow(a, r0 + 1, xs, &du1);
        double dz = W[r0 + 1] - W[r0];
        double t = (w - W[r0]) / dz;
        if (g->extrap == 3) {
            double doff, d0, d1;
            double y = cont(B0, B1, w - W[r0], dz, &doff, &d0, &d1);
            if (dw) *dw = doff;
            if (du) *du = d0 * du0 + d1 * du1;
            return y;
        }
        if (dw) *dw = (B1 - B0) / dz;
        if (du) *du = du0 + t * (du1 - du0);
        return B0 + (w - W[r0]) * (B1 - B0) / dz;
    }
    int s = 0;
    for (int j = 0; j < g->n_sub; ++j)
        if (W[g->row0[j]] <= w) s = j;
    int n = g->n_q[s], r0 = g->row0[s];
    const double *Ws = W + r0;
    int k = interval(Ws, n, w);
    if (g->interp == 1 || (g->interp == 2 && n < 4)) {
        /* straight line between the interval's two rows */
        double du0, du1;
        double B0 = xrow(a, r0 + k, xs, &du0), B1 = xrow(a, r0 + k + 1, xs, &du1);
        double dz = Ws[k + 1] - Ws[k];
        double t = (w - Ws[k]) / dz;
        if (dw) *dw = frozen ? 0.0 : (B1 - B0) / dz;
        if (du) *du = (1.0 - t) * du0 + t * du1;
        return (1.0 - t) * B0 + t * B1;
    }
    double R[4] = {0, 0, 0, 0}, D[4] = {0, 0, 0, 0};
    for (int j = -1; j <= 2; ++j) {
        int kk = k + j;
        if (kk < 0 || kk >= n) continue;
        R[j + 1] = xrow(a, r0 + kk, xs, &D[j + 1]);
    }
    double d0 = fd_deriv(k, n, Ws, R[0], R[1], R[2]);
    double d1 = fd_deriv(k + 1, n, Ws, R[1], R[2], R[3]);
    double dz = Ws[k + 1] - Ws[k];
    double t = (w - Ws[k]) / dz;
    double value = hermite(t, dz, R[1], R[2], d0, d1, dw);
    if (frozen && dw) *dw = 0.0;
    if (du) {
        /* the same w-Hermite applied to the u-derivatives of the rows */
        double e0 = fd_deriv(k, n, Ws, D[0], D[1], D[2]);
        double e1 = fd_deriv(k + 1, n, Ws, D[1], D[2], D[3]);
        *du = hermite(t, dz, D[1], D[2], e0, e1, NULL);
    }
    return value;
}

/* Full evaluation at (u, w) with the accessor; derivatives optional. */
static double eval_uw(const acc_t *a, double u, double w, double *du, double *dw)
{
    const orc_grid *g = a->g;
    const double *U = g->U;
    int n = g->n_x;
    if ((u < U[0] || u > U[n - 1]) && g->extrap == 1) {
        /* frozen at the edge: clamp u, no derivative across the edge */
        xsel_t xs = {-1, u < U[0] ? U[0] : U[n - 1]};
        double v = wdir(a, &xs, w, dw, du);
        if (du) *du = 0.0;
        return v;
    }
    if (u < U[0] || u > U[n - 1]) {
        /* step 6 in u: A_k = w-interpolation of the two edge columns */
        int k0 = u < U[0] ? 0 : n - 2;
        xsel_t c0 = {k0, 0.0}, c1 = {k0 + 1, 0.0};
        double dw0, dw1;
        double A0 = wdir(a, &c0, w, &dw0, NULL), A1 = wdir(a, &c1, w, &dw1, NULL);
        double dz = U[k0 + 1] - U[k0];
        if (g->extrap == 3) {
            double doff, d0, d1;
            double y = cont(A0, A1, u - U[k0], dz, &doff, &d0, &d1);
            if (du) *du = doff;
            if (dw) *dw = d0 * dw0 + d1 * dw1;
            return y;
        }
        if (du) *du = (A1 - A0) / dz;
        if (dw) *dw = dw0 + (u - U[k0]) / dz * (dw1 - dw0);
        return A0 + (u - U[k0]) * (A1 - A0) / dz;
    }
    xsel_t xs = {-1, u};
    return wdir(a, &xs, w, dw, du);
}

/* ---------------------------------------------------------------- public */

/* The grid's a-th flavour with the gluon as 0: a grid may list its gluon as
 * 21 or as 0, and a query may ask for it either way. */
static int grid_pid(const orc_grid *g, int a) { return g->pids[a] == 21 ? 0 : g->pids[a]; }

static int pid_column(const orc_grid *g, int pid)
{
    if (pid == 21) pid = 0;
    for (int a = 0; a < g->n_flav; ++a)
        if (grid_pid(g, a) == pid) return a;
    return -1;
}

static acc_t member_acc(const orc_grid *g, int member, int col)
{
    acc_t a;
    a.g = g;
    a.base = g->values + (size_t)member * g->rows * g->n_x * g->n_flav + col;
    a.stride_row = g->n_x * g->n_flav;
    a.stride_k = g->n_flav;
    a.ind_row = a.ind_k = -1;
    return a;
}

static int bad_x(double x) { return !(x > 0.0) || !(x <= 1.0); }
static int bad_q2(double q2) { return !(q2 > 0.0) || !(q2 < INFINITY); }

/* x*f for one pid at (u, w) in log coordinates; derivatives d/du, d/dw. */
double orc_xfxq2_uw(const orc_grid *g, int member, int pid, double u, double w,
                    double *du, double *dw)
{
    if (du) *du = 0.0;
    if (dw) *dw = 0.0;
    if (!(u <= 0.0) || !(w > -INFINITY && w < INFINITY)) {
        if (du) *du = NAN;
        if (dw) *dw = NAN;
        return NAN;
    }
    if (g->extrap == 2 && (u < g->U[0] || u > g->U[g->n_x - 1] || w < g->W[0] || w > g->W[g->rows - 1])) {
        if (du) *du = NAN;
        if (dw) *dw = NAN;
        return NAN;
    }
    int col = pid_column(g, pid);
    if (col < 0) return 0.0;
    acc_t a = member_acc(g, member, col);
    return eval_uw(&a, u, w, du, dw);
}

double orc_xfxq2(const orc_grid *g, int member, int pid, double x, double q2)
{
    if (bad_x(x) || bad_q2(q2)) return NAN;
    return orc_xfxq2_uw(g, member, pid, log(x), log(q2), NULL, NULL);
}

/* d(xf)/dx and d(xf)/dQ^2 (chain rule through u = ln x, w = ln Q^2). */
double orc_xfxq2_grad(const orc_grid *g, int member, int pid, double x, double q2,
                      double *dx, double *dq2)
{
    if (bad_x(x) || bad_q2(q2)) {
        *dx = *dq2 = NAN;
        return NAN;
    }
    double du, dw;
    double v = orc_xfxq2_uw(g, member, pid, log(x), log(q2), &du, &dw);
    *dx = du / x;
    *dq2 = dw / q2;
    return v;
}

double orc_alphas_w(const orc_grid *g, double w)
{
    if (!g->alphas || !(w > -INFINITY && w < INFINITY)) return NAN;
    if (g->extrap == 2 && (w < g->W[0] || w > g->W[g->rows - 1])) return NAN;
    acc_t a;
    a.g = g;
    a.base = g->alphas;
    a.stride_row = 1;
    a.stride_k = 0;
    a.ind_row = a.ind_k = -1;
    xsel_t c = {0, 0.0};
    return wdir(&a, &c, w, NULL, NULL);
}

/* alpha_s and d alpha_s / d Q^2 (chain rule through w = ln Q^2). */
double orc_alphas_grad(const orc_grid *g, double q2, double *dq2)
{
    *dq2 = NAN;
    if (bad_q2(q2) || !g->alphas) return NAN;
    double w = log(q2);
    if (g->extrap == 2 && (w < g->W[0] || w > g->W[g->rows - 1])) return NAN;
    acc_t a;
    a.g = g;
    a.base = g->alphas;
    a.stride_row = 1;
    a.stride_k = 0;
    a.ind_row = a.ind_k = -1;
    xsel_t c = {0, 0.0};
    double dw = 0.0;
    double v = wdir(&a, &c, w, &dw, NULL);
    *dq2 = dw / q2;
    return v;
}

double orc_alphas(const orc_grid *g, double q2)
{
    if (bad_q2(q2)) return NAN;
    return orc_alphas_w(g, log(q2));
}

/* Weight of grid value (row, k) in the result at (u, w): the interpolation
 * of the indicator grid of that value (step 8). */
double orc_cell_weight_uw(const orc_grid *g, int row, int k, double u, double w)
{
    acc_t a;
    a.g = g;
    a.base = NULL;
    a.stride_row = a.stride_k = 0;
    a.ind_row = row;
    a.ind_k = k;
    return eval_uw(&a, u, w, NULL, NULL);
}

/* Rows and columns that may carry weight at (u, w): a window around the
 * interval (or the edge interval when out of range).  Used to keep the
 * indicator scan short; cells outside it are exactly zero by construction
 * (checked by a full scan on small grids in the tests). */
static void window(const orc_grid *g, double u, double w, int *c0, int *c1, int *r0, int *r1)
{
    int k = interval(g->U, g->n_x, u);
    *c0 = k - 2 < 0 ? 0 : k - 2;
    *c1 = k + 3 > g->n_x - 1 ? g->n_x - 1 : k + 3;
    int s = 0;
    if (w > g->W[g->rows - 1]) s = g->n_sub - 1;
    else
        for (int j = 0; j < g->n_sub; ++j)
            if (g->W[g->row0[j]] <= w) s = j;
    int n = g->n_q[s], b = g->row0[s];
    int q = interval(g->W + b, n, w);
    *r0 = b + (q - 2 < 0 ? 0 : q - 2);
    *r1 = b + (q + 3 > n - 1 ? n - 1 : q + 3);
}

/* ------------------------------------------------------- batch drivers */

void orc_xfxq2_batch(const orc_grid *g, int member, const int *pids, int n_pid,
                     const double *x, const double *q2, int64_t n, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int p = 0; p < n_pid; ++p)
            out[i * n_pid + p] = orc_xfxq2(g, member, pids[p], x[i], q2[i]);
}

void orc_xfxq2_pw_batch(const orc_grid *g, int member, const int *pid,
                        const double *x, const double *q2, int64_t n, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = orc_xfxq2(g, member, pid[i], x[i], q2[i]);
}

void orc_alphas_batch(const orc_grid *g, const double *q2, int64_t n, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = orc_alphas(g, q2[i]);
}

/* d/dx and d/dQ^2 for pointwise pids (pid per point). */
void orc_grad_pw_batch(const orc_grid *g, int member, const int *pid, const double *x,
                       const double *q2, int64_t n, double *dx, double *dq2)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) orc_xfxq2_grad(g, member, pid[i], x[i], q2[i], &dx[i], &dq2[i]);
}

/* kappa = sum over cells |weight * value| for each (point, pid): the size of
 * the terms the interpolation adds up, used to scale rounding tolerances. */
void orc_kappa_batch(const orc_grid *g, int member, const int *pids, int n_pid, int pointwise,
                     const double *x, const double *q2, int64_t n, double *kappa)
{
    int stride = g->n_x * g->n_flav;
    const double *vm = g->values + (size_t)member * g->rows * stride;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int np = pointwise ? 1 : n_pid;
        for (int p = 0; p < np; ++p) kappa[i * np + p] = 0.0;
        if (bad_x(x[i]) || bad_q2(q2[i])) {
            for (int p = 0; p < np; ++p) kappa[i * np + p] = NAN;
            continue;
        }
        double u = log(x[i]), w = log(q2[i]);
        int c0, c1, r0, r1;
        window(g, u, w, &c0, &c1, &r0, &r1);
        for (int r = r0; r <= r1; ++r)
            for (int k = c0; k <= c1; ++k) {
                double wt = orc_cell_weight_uw(g, r, k, u, w);
                if (wt == 0.0) continue;
                for (int p = 0; p < np; ++p) {
                    int col = pid_column(g, pointwise ? pids[i] : pids[p]);
                    if (col < 0) continue;
                    kappa[i * np + p] += fabs(wt * vm[(size_t)r * stride + (size_t)k * g->n_flav + col]);
                }
            }
    }
}

/* kappa of alpha_s at each Q^2: the sum over the alpha_s knots r of
 * |W_r(w) alpha_r|, W_r the interpolation of the indicator of knot r (step
 * 8, as for the PDF values; outside the grid under option 3 the indicator
 * falls back to the straight line, whose weights are used as the scale).
 * NaN where alpha_s is NaN. */
void orc_alphas_kappa_batch(const orc_grid *g, const double *q2, int64_t n, double *kappa)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double v = orc_alphas(g, q2[i]);
        if (v != v) {
            kappa[i] = NAN;
            continue;
        }
        double w = log(q2[i]);
        int c0, c1, r0, r1;
        window(g, g->U[0], w, &c0, &c1, &r0, &r1);
        double sum = 0.0;
        for (int r = r0; r <= r1; ++r) {
            acc_t a;
            a.g = g;
            a.base = NULL;
            a.stride_row = a.stride_k = 0;
            a.ind_row = r;
            a.ind_k = 0;
            xsel_t c = {0, 0.0};
            sum += fabs(wdir(&a, &c, w, NULL, NULL) * g->alphas[r]);
        }
        kappa[i] = sum;
    }
}

/* dL/dvalues for L = sum_i gw_i * xf_{pid_i}(x_i, Q^2_i), accumulated into
 * grad[rows][n_x][n_flav] (member's slice).  Serial: the sum order is fixed.
 * absval != 0 accumulates |gw_i * weight| instead: the magnitude of the terms
 * of each sum, used to scale rounding tolerances. */
void orc_dgrid_pw(const orc_grid *g, const int *pid, const double *x, const double *q2,
                  const double *gw, int64_t n, double *grad, int absval)
{
    for (int64_t i = 0; i < n; ++i) {
        int col = pid_column(g, pid[i]);
        if (col < 0 || bad_x(x[i]) || bad_q2(q2[i])) continue;
        double u = log(x[i]), w = log(q2[i]);
        int c0, c1, r0, r1;
        window(g, u, w, &c0, &c1, &r0, &r1);
        for (int r = r0; r <= r1; ++r)
            for (int k = c0; k <= c1; ++k) {
                double wt = orc_cell_weight_uw(g, r, k, u, w);
                double t = gw[i] * wt;
                grad[((size_t)r * g->n_x + k) * g->n_flav + col] += absval ? fabs(t) : t;
            }
    }
}

/* Matrix form: gradient of L = sum_i sum_p gout[i][p] * xf_{pids[p]}(x_i, Q^2_i). */
void orc_dgrid_batch(const orc_grid *g, const int *pids, int n_pid, const double *x,
                     const double *q2, const double *gout, int64_t n, double *grad, int absval)
{
    for (int64_t i = 0; i < n; ++i) {
        if (bad_x(x[i]) || bad_q2(q2[i])) continue;
        double u = log(x[i]), w = log(q2[i]);
        int c0, c1, r0, r1;
        window(g, u, w, &c0, &c1, &r0, &r1);
        for (int r = r0; r <= r1; ++r)
            for (int k = c0; k <= c1; ++k) {
                double wt = orc_cell_weight_uw(g, r, k, u, w);
                if (wt == 0.0) continue;
                for (int p = 0; p < n_pid; ++p) {
                    int col = pid_column(g, pids[p]);
                    if (col < 0) continue;
                    double t = gout[i * n_pid + p] * wt;
                    grad[((size_t)r * g->n_x + k) * g->n_flav + col] += absval ? fabs(t) : t;
                }
            }
    }
}

/* ------------------------------------------------- luminosity workload */

/* Kinematics of one event in log variables: ln x1 = ln(tau)/2 + y,
 * ln x2 = ln(tau)/2 - y, ln Q^2 = ln tau + ln s, with the injected tail
 * (flags bit 0: ln Q^2 = ln_mu2, bit 1: ln x1 = ln_x1). */
static void event_uw(double ln_tau, double y, unsigned flags, double ln_mu2, double ln_x1,
                     double ln_s, double *u1, double *u2, double *w)
{
    double h = 0.5 * ln_tau;
    *u1 = h + y;
    *u2 = h - y;
    *w = ln_tau + ln_s;
    if (flags & 1u) *w = ln_mu2;
    if (flags & 2u) *u1 = ln_x1;
}

/* Per event: lum = sum_a xf_a(x1, Q^2) xf_{-a}(x2, Q^2) over the grid's pids
 * (-0 = 0), and alpha_s(Q^2).  Returns (1/N) sum lum (serial sum). */
double orc_lumi_batch(const orc_grid *g, int member, const double *ln_tau, const double *y,
                      const unsigned char *flags, const double *ln_mu2, const double *ln_x1,
                      double ln_s, int64_t n, double *lum, double *as)
{
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n; ++e) {
        double u1, u2, w;
        event_uw(ln_tau[e], y[e], flags[e], ln_mu2[e], ln_x1[e], ln_s, &u1, &u2, &w);
        double s = 0.0;
        for (int a = 0; a < g->n_flav; ++a) {
            int pa = grid_pid(g, a);
            double f1 = orc_xfxq2_uw(g, member, pa, u1, w, NULL, NULL);
            double f2 = orc_xfxq2_uw(g, member, -pa, u2, w, NULL, NULL);
            s += f1 * f2;
        }
        lum[e] = s;
        if (as) as[e] = orc_alphas_w(g, w);
    }
    double tot = 0.0;
    for (int64_t e = 0; e < n; ++e) tot += lum[e];
    return n > 0 ? tot / (double)n : 0.0;
}

/* dL/dvalues (member's slice) for L = (1/N) sum_e lum_e. */
void orc_lumi_dgrid(const orc_grid *g, int member, const double *ln_tau, const double *y,
                    const unsigned char *flags, const double *ln_mu2, const double *ln_x1,
                    double ln_s, int64_t n, double *grad, int absval)
{
    int F = g->n_flav;
    double f1[64], f2[64];
    if (F > 64) return;
    for (int64_t e = 0; e < n; ++e) {
        double uu[2], w;
        event_uw(ln_tau[e], y[e], flags[e], ln_mu2[e], ln_x1[e], ln_s, &uu[0], &uu[1], &w);
        for (int a = 0; a < F; ++a) {
            f1[a] = orc_xfxq2_uw(g, member, grid_pid(g, a), uu[0], w, NULL, NULL);
            f2[a] = orc_xfxq2_uw(g, member, grid_pid(g, a), uu[1], w, NULL, NULL);
        }
        for (int side = 0; side < 2; ++side) {
            const double *other = side == 0 ? f2 : f1;
            int c0, c1, r0, r1;
            window(g, uu[side], w, &c0, &c1, &r0, &r1);
            for (int r = r0; r <= r1; ++r)
                for (int k = c0; k <= c1; ++k) {
                    double wt = orc_cell_weight_uw(g, r, k, uu[side], w);
                    if (wt == 0.0) continue;
                    for (int b = 0; b < F; ++b) {
                        /* d(sum_a f_a(x1) f_{-a}(x2)) / d v[.][b]:
                         * side 0 (a = b): weight at x1 times f_{-b}(x2);
                         * side 1 (-a = b): f_{-b}(x1) times weight at x2. */
                        int cb = pid_column(g, -grid_pid(g, b));
                        if (cb < 0) continue;
                        double t = wt * other[cb] / (double)n;
                        grad[((size_t)r * g->n_x + k) * F + b] += absval ? fabs(t) : t;
                    }
                }
        }
    }
}

/* ------------------------------------------ adaptive Monte Carlo (VEGAS) */
/*
 * The Monte Carlo use of the paper (Sec. 3.1: VegasFlow importance sampling
 * around an integrand that calls the PDFs; matrix element set to 1 here):
 *
 *   I = int_0^1 dr1 dr2 F(r1, r2),
 *   ln tau = (1 - r1) ln tau_min,  y = (2 r2 - 1)(-ln tau / 2),
 *   ln x1,2 = ln tau / 2 +- y,  ln Q^2 = ln tau + ln s,
 *   F = (-ln tau_min)(-ln tau) sum_a xf_a(x1) xf_{-a}(x2)
 *
 * (the Jacobian of (ln tau, y) -> (r1, r2) times the luminosity), sampled
 * through the VEGAS map of Lepage (J. Comput. Phys. 27 (1978) 192): per
 * dimension n_bins bins with edges e_0 = 0 < ... < e_n = 1; a uniform v
 * falls in bin i = floor(v n) at fraction d = v n - i, is mapped to
 * r = e_i + d (e_{i+1} - e_i), with Jacobian n (e_{i+1} - e_i).
 */

/* Sums of one iteration: out[0] = sum w, out[1] = sum (w - shift)^2 (the
 * sample variance about a shift near the mean, normally the previous
 * iteration's estimate: sum (w - c)^2 / n - (mean - c)^2 is the variance of w
 * for any c, and with c near the mean it is a sum of small squares instead of
 * the difference of two nearly equal numbers), then for each of the two
 * dimensions the sum of w^2 over the points in each bin, where w = F(r) J(v)
 * is the weight of the point drawn with uniforms v[i][0..1]. */
void orc_vegas_sums(const orc_grid *g, int member, double ln_tau_min, double ln_s, int n_bins,
                    const double *edges, const double *v, int64_t n, double shift, double *out)
{
    for (int k = 0; k < 2 + 2 * n_bins; ++k) out[k] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double r[2], jac = 1.0;
        int bin[2];
        for (int d = 0; d < 2; ++d) {
            const double *e = edges + (size_t)d * (n_bins + 1);
            double vn = v[2 * i + d] * n_bins;
            int b = (int)vn;
            if (b > n_bins - 1) b = n_bins - 1;
            double frac = vn - b;
            double width = e[b + 1] - e[b];
            r[d] = e[b] + frac * width;
            jac *= n_bins * width;
            bin[d] = b;
        }
        double ln_tau = (1.0 - r[0]) * ln_tau_min;
        double h = 0.5 * ln_tau;
        double y = (2.0 * r[1] - 1.0) * (-h);
        double u1 = h + y, u2 = h - y, w = ln_tau + ln_s;
        double lum = 0.0;
        for (int a = 0; a < g->n_flav; ++a) {
            int pa = grid_pid(g, a);
            lum += orc_xfxq2_uw(g, member, pa, u1, w, NULL, NULL) *
                   orc_xfxq2_uw(g, member, -pa, u2, w, NULL, NULL);
        }
        double f = (-ln_tau_min) * (-ln_tau) * lum;
        double wt = f * jac;
        out[0] += wt;
        out[1] += (wt - shift) * (wt - shift);
        out[2 + bin[0]] += wt * wt;
        out[2 + n_bins + bin[1]] += wt * wt;
    }
}

/* The VEGAS map for an integrand the caller evaluates (any dimension): per
 * point and dimension d, the uniform v lands in bin b = floor(v n) (at most
 * n - 1) at fraction v n - b, and maps to r = e_b + frac (e_{b+1} - e_b); the
 * Jacobian is the product over d of n (e_{b+1} - e_b).  edges [dim][n+1],
 * v and r [n_pts][dim], bins [n_pts][dim]. */
void orc_vegas_map(int dim, int n_bins, const double *edges, const double *v, int64_t n_pts, double *r,
                   double *jac, int *bins)
{
    for (int64_t i = 0; i < n_pts; ++i) {
        double j = 1.0;
        for (int d = 0; d < dim; ++d) {
            const double *e = edges + (size_t)d * (n_bins + 1);
            double vn = v[i * dim + d] * n_bins;
            int b = (int)vn;
            if (b > n_bins - 1) b = n_bins - 1;
            double frac = vn - b;
            double width = e[b + 1] - e[b];
            r[i * dim + d] = e[b] + frac * width;
            j *= n_bins * width;
            bins[i * dim + d] = b;
        }
        jac[i] = j;
    }
}

/* Sums of one iteration from the weights w_i = f(r_i) J_i: out[0] = sum w,
 * out[1] = sum (w - shift)^2, then for each dimension d the per-bin sums of
 * w^2, out[2 + d n + b].  Serial, in point order. */
void orc_vegas_accumulate(int dim, int n_bins, const double *w, const int *bins, int64_t n_pts, double shift,
                          double *out)
{
    for (int k = 0; k < 2 + dim * n_bins; ++k) out[k] = 0.0;
    for (int64_t i = 0; i < n_pts; ++i) {
        double wi = w[i];
        out[0] += wi;
        out[1] += (wi - shift) * (wi - shift);
        for (int d = 0; d < dim; ++d) out[2 + d * n_bins + bins[i * dim + d]] += wi * wi;
    }
}

/* One refinement of one dimension's edges from its per-bin sums of w^2
 * (Lepage's rule): smooth the sums with their neighbours, damp them as
 * r_i = ((1 - d_i) / ln(1 / d_i))^alpha with d_i the normalised smoothed sum,
 * and place the new edges so that every new bin holds an equal share of
 * sum r_i, the old bins' shares spread uniformly over their widths. */
void orc_vegas_refine(const double *bin_w2, int n_bins, double alpha, double *edges)
{
    double d[4096], r[4096], e_old[4097];
    if (n_bins < 2 || n_bins > 4096) return;
    d[0] = 0.5 * (bin_w2[0] + bin_w2[1]);
    for (int i = 1; i < n_bins - 1; ++i) d[i] = (bin_w2[i - 1] + bin_w2[i] + bin_w2[i + 1]) / 3.0;
    d[n_bins - 1] = 0.5 * (bin_w2[n_bins - 2] + bin_w2[n_bins - 1]);
    double dsum = 0.0;
    for (int i = 0; i < n_bins; ++i) dsum += d[i];
    if (!(dsum > 0.0)) return;
    double rsum = 0.0;
    for (int i = 0; i < n_bins; ++i) {
        double di = d[i] / dsum;
        r[i] = (di > 0.0 && di < 1.0) ? pow((1.0 - di) / log(1.0 / di), alpha) : 0.0;
        rsum += r[i];
    }
    if (!(rsum > 0.0)) return;
    for (int i = 0; i <= n_bins; ++i) e_old[i] = edges[i];
    double per_bin = rsum / n_bins, acc = 0.0;
    int k = 0;
    for (int j = 1; j < n_bins; ++j) {
        double target = j * per_bin;
        while (acc + r[k] <= target) {
            acc += r[k];
            ++k;
        }
        /* the new edge lies in old bin k, at the fraction of its share still needed */
        double frac = (target - acc) / r[k];
        edges[j] = e_old[k] + frac * (e_old[k + 1] - e_old[k]);
    }
    edges[0] = 0.0;
    edges[n_bins] = 1.0;
}
