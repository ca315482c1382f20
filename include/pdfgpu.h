/*
 * pdfgpu — batched FP64 parton-density (x*f) and alpha_s interpolation on a
 * GB300 GPU (sm_103a), the data-parallel hot path of PDFFlow
 * (Rossi, Carrazza, Cruz-Martinez, arXiv:2012.08221).
 *
 * What is computed (PDFFlow Sec. 2.1: a set of flavours {a} and two arrays of
 * equal length, x_i and Q_i, in; an array of interpolated values out; alpha_s
 * interpolated the same way; Sec. 4: the LHAPDF grid layout and algorithms):
 *
 *   x*f_a(x, Q^2) by log-bicubic interpolation in (ln x, ln Q^2) on a grid of
 *   knot values.  Q knots are split into subgrids at flavour thresholds; the
 *   threshold knot is stored twice (last knot of subgrid s == first knot of
 *   s+1) and interpolation never crosses a subgrid.  Along each axis the
 *   interval cubic is the Hermite cubic whose knot derivatives are finite
 *   differences: a one-sided secant at the first and last knot of an axis
 *   (or subgrid), the mean of the two adjacent secants inside.  The interval
 *   is the largest knot k with z_k <= z, clamped to the last interval; a Q^2
 *   equal to an internal threshold belongs to the upper subgrid.  Outside the
 *   grid the result continues linearly in ln x (from the two edge x columns)
 *   and in ln Q^2 (from the two edge rows of the lowest/highest subgrid).
 *   alpha_s(Q^2) is the same cubic in ln Q^2 on the alpha_s knot values.
 *
 * Conventions for every entry point:
 *   - Return PDF_OK (0) or a negative PDF_E_* code; nothing is thrown across
 *     the boundary.  pdf_last_error() gives a message for the calling thread.
 *   - Arrays documented as DEVICE are device pointers owned by the caller;
 *     the library only reads/writes them inside kernels launched on `stream`
 *     (a cudaStream_t passed as void*; NULL = the legacy default stream).
 *     Calls are asynchronous unless documented otherwise.
 *   - Arrays documented as HOST are read during the call (copied) unless
 *     documented otherwise.
 *   - A grid handle holds state that some calls change while their kernels
 *     run: the interpolation coefficients (pdf_bind_values, which the
 *     differentiable bindings call), the adjoints' and the luminosity
 *     adjoint's scratch (xfxQ2_backward*, pdf_lumi_backward) and the
 *     host-buffer path's staging (xfxQ2_host, which serialises its own
 *     callers).  Such calls on one handle from different streams or host
 *     threads race unless the caller orders them; use one handle per stream
 *     to run them concurrently.  The other calls only read the handle.
 *   - xfxQ2 and alphasQ2 (and their Q forms) may be captured in a CUDA graph
 *     on `stream` once a first call on the grid has run outside the capture
 *     (that call may raise a kernel's shared-memory limit, which a capture
 *     must not do); the graph's replays read the captured device arrays.
 *   - Per-element domain errors do not fail a call: x <= 0, x > 1, Q^2 <= 0,
 *     Q^2 infinite or any NaN input gives NaN for every requested flavour and
 *     sets PDF_S_DOMAIN in the grid's status word (PDF_S_RANGE for points
 *     outside the knot range of a grid loaded with PDF_EXTRAP_ERROR).  A pid absent from the grid
 *     gives 0 (pid 21 and pid 0 both mean the gluon).  n == 0 is a no-op.
 *   - The output is x*f, not f (the paper's luminosity divides by x1*x2).
 */
#ifndef PDFGPU_H
#define PDFGPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pdfgpu_grid *pdfgpu_grid_t;     /* opaque, library-owned */
typedef struct pdfgpu_batch *pdfgpu_batch_t;   /* opaque, library-owned */
typedef void *pdfgpu_stream_t;                 /* a cudaStream_t */

enum {
    PDF_OK = 0,
    PDF_E_ARG = -1,       /* null pointer, negative size, bad member, too many pids */
    PDF_E_DESC = -2,      /* malformed grid description (knots, sizes, thresholds)   */
    PDF_E_CUDA = -3,      /* a CUDA runtime call failed (message has the CUDA error)  */
    PDF_E_UNBOUND = -4,   /* the grid has no values yet (pdf_bind_values not called)  */
    PDF_E_NOMEM = -5,     /* device or host allocation failed                         */
    PDF_E_RANGE = -6      /* a size exceeds a documented limit                        */
};

/* Status bits accumulated by kernels in the grid's device status word. */
enum {
    PDF_S_DOMAIN = 1u,    /* some input x / Q^2 was out of the domain (output NaN)   */
    PDF_S_RANGE = 2u,     /* some input was outside the knot range of a grid loaded
                             with PDF_EXTRAP_ERROR (output NaN)                      */
    PDF_S_BOUNDS = 4u     /* checked builds only (PDFGPU_CHECKED): a table index computed
                             on the device was out of range and was replaced        */
};

/* Interpolation kind of a grid (pdfgpu_grid_desc.interp).  The paper keeps
 * LHAPDF's interpolators without printing them; the default is the
 * log-bicubic one described at the top of this file.
 *   LOGBICUBIC               Hermite cubics with finite-difference slopes
 *   LOGBILINEAR              straight lines between the interval's two knots
 *                            on both axes (ln x, ln Q^2)
 *   LOGBICUBIC_SMALL_LINEAR  log-bicubic, but straight lines along any axis
 *                            or Q subgrid that has fewer than 4 knots       */
enum {
    PDF_INTERP_LOGBICUBIC = 0,
    PDF_INTERP_LOGBILINEAR = 1,
    PDF_INTERP_LOGBICUBIC_SMALL_LINEAR = 2
};

/* Extrapolation outside the knot range (pdfgpu_grid_desc.extrap):
 *   LINEAR        continue linearly in ln x / ln Q^2 from the two edge knots
 *   FREEZE        the value at the nearest edge of the grid (zero derivative
 *                 across the edge)
 *   ERROR         NaN and the PDF_S_RANGE status bit
 *   CONTINUATION  LHAPDF-style power law from the same two edge values y0, y1
 *                 (lower and upper knot of the edge interval, t the position
 *                 in it): y0^(1-t) y1^t when both exceed 1e-3, else the
 *                 LINEAR value (sign-safe); ln Q^2 is continued first (per
 *                 edge x column in the corners), then ln x.  The result is
 *                 not linear in the grid values: the adjoint entry points
 *                 (xfxQ2_backward, pdf_lumi_backward) return PDF_E_ARG for
 *                 such a grid; alphasQ2_grad supports it.                */
enum {
    PDF_EXTRAP_LINEAR = 0,
    PDF_EXTRAP_FREEZE = 1,
    PDF_EXTRAP_ERROR = 2,
    PDF_EXTRAP_CONTINUATION = 3
};

#define PDF_MAX_PIDS 64   /* flavours per matrix-form call                  */
#define PDF_MAX_FLAV 64   /* flavours stored in one grid                    */

/* Grid description: every pointer is HOST memory, read and copied by
 * pdf_load_grid.  Knots are in GeV (Q, not Q^2).
 *   x_knots [n_x]          strictly ascending, 0 < x_k <= 1, n_x >= 2
 *   n_q     [n_sub]        knots per Q subgrid, each >= 2
 *   q_knots [sum n_q]      strictly ascending inside a subgrid; the last knot of
 *                          subgrid s equals the first knot of s+1 (duplicated)
 *   pids    [n_flav]       PDG ids, distinct; 0 or 21 is the gluon
 *   values  [n_members][sum n_q][n_x][n_flav]  x*f at the knots (row-major),
 *                          or NULL: bind later with pdf_bind_values
 *   alphas  [sum n_q]      alpha_s at the Q knots, or NULL (no alpha_s)
 *   interp                 PDF_INTERP_* (0: log-bicubic); alpha_s follows the
 *                          same kind along ln Q^2
 *   extrap                 PDF_EXTRAP_* (0: linear continuation), also for
 *                          alpha_s (which continues by the same rule)        */
typedef struct {
    int32_t n_x;
    const double *x_knots;
    int32_t n_sub;
    const int32_t *n_q;
    const double *q_knots;
    int32_t n_flav;
    const int32_t *pids;
    int32_t n_members;
    const double *values;
    const double *alphas;
    int32_t interp;
    int32_t extrap;
} pdfgpu_grid_desc;

/* Validate a grid description, upload it and build the interpolation tables
 * on the current CUDA device (PDFFlow Sec. 2.1 `mkPDF`; Sec. 4 grid format).
 * Synchronous.  On success *out owns device memory until pdf_free_grid. */
int pdf_load_grid(const pdfgpu_grid_desc *desc, pdfgpu_grid_t *out);

/* (Re)build the per-cell bicubic coefficients of ALL members from a DEVICE
 * array `dev_values` laid out as the description's `values` (beyond the
 * paper: the differentiation form, where the knot values are the
 * parameters a PDF fit moves -- PDFFlow Sec. 1 names the fitting
 * collaborations that produce the grids -- and live in a device tensor).
 * The array is read on `stream` during the call and not kept.  Asynchronous
 * on `stream`.  The coefficients are ONE table per grid handle: a call
 * replaces them for every later call on the handle, on any stream, so two
 * rebinds of one handle with different values from two streams (for example
 * two differentiable evaluations, each of which rebinds) race; use one
 * handle per stream, or order the streams. */
int pdf_bind_values(pdfgpu_grid_t g, const double *dev_values, pdfgpu_stream_t stream);

/* Free every device allocation of the grid (the end of the life of the PDF
 * object of PDFFlow Sec. 2.1 `mkPDF`).  Synchronises the device. */
int pdf_free_grid(pdfgpu_grid_t g);

/* Sizes of a loaded grid, as in the grid description of PDFFlow Sec. 4 (any
 * pointer may be NULL). */
int pdf_grid_info(pdfgpu_grid_t g, int32_t *n_x, int32_t *n_rows, int32_t *n_flav,
                  int32_t *n_members, int32_t *has_alphas);

/* Batched x*f for a shared pid list (PDFFlow Sec. 2.1; `xfxQ2(pids, x, q2)` of
 * the luminosity example, Sec. 3.2).
 *   member            0 <= member < n_members (member 0 = central replica)
 *   pids   HOST  [n_pid], 1 <= n_pid <= PDF_MAX_PIDS
 *   x, q2  DEVICE [n]
 *   out    DEVICE [n][n_pid] row-major                                       */
int xfxQ2(pdfgpu_grid_t g, int32_t member, const int32_t *pids, int32_t n_pid,
          const double *x, const double *q2, int64_t n, double *out, pdfgpu_stream_t stream);

/* Same with Q instead of Q^2 (PDFFlow Sec. 2.1 `py_xfxQ`): Q^2 = q*q. */
int xfxQ(pdfgpu_grid_t g, int32_t member, const int32_t *pids, int32_t n_pid,
         const double *x, const double *q, int64_t n, double *out, pdfgpu_stream_t stream);

/* Pointwise form: one pid per point (beyond the paper's shared flavour set
 * of Sec. 2.1; it serves the differentiation workload, where every point
 * asks for one flavour, and a Monte Carlo integrand that needs one flavour
 * per phase-space point, Sec. 3.1).
 *   pid DEVICE [n], x, q2 DEVICE [n], out DEVICE [n]                         */
int xfxQ2_pw(pdfgpu_grid_t g, int32_t member, const int32_t *pid, const double *x,
             const double *q2, int64_t n, double *out, pdfgpu_stream_t stream);

/* x*f and alpha_s at the same points in one launch (PDFFlow Sec. 2.1 `xfxQ2`
 * and `py_alphasQ`; Sec. 3.1-3.2: an integrand asks for both at the
 * factorisation scale of each phase-space point).  The Q^2 search and
 * logarithm are shared.  Arguments as for xfxQ2, plus alphas DEVICE [n]:
 * alpha_s(q2[i]).  The outputs equal those of xfxQ2 and alphasQ2 on the same
 * arrays bit for bit (alpha_s stays valid where only x is out of the domain).
 * PDF_E_DESC if the grid has no alpha_s values. */
int xfxQ2_alphasQ2(pdfgpu_grid_t g, int32_t member, const int32_t *pids, int32_t n_pid,
                   const double *x, const double *q2, int64_t n, double *out, double *alphas,
                   pdfgpu_stream_t stream);

/* alpha_s(Q^2) (PDFFlow Sec. 2.1, `py_alphasQ`).  q2, out DEVICE [n].
 * PDF_E_DESC if the grid was loaded without alpha_s values. */
int alphasQ2(pdfgpu_grid_t g, const double *q2, int64_t n, double *out, pdfgpu_stream_t stream);
int alphasQ(pdfgpu_grid_t g, const double *q, int64_t n, double *out, pdfgpu_stream_t stream);

/* alpha_s(Q^2) and its derivative d alpha_s / d Q^2 (the derivative of the
 * same piecewise cubic in ln Q^2, divided by Q^2; zero across a frozen edge).
 * Beyond the paper: the differentiation form applied to the alpha_s
 * interpolation of Sec. 2.1.
 * q2, dq2 DEVICE [n]; out DEVICE [n] or NULL. */
int alphasQ2_grad(pdfgpu_grid_t g, const double *q2, int64_t n, double *out, double *dq2,
                  pdfgpu_stream_t stream);

/* End-to-end form of xfxQ2 for HOST buffers (PDFFlow Sec. 2.1: arrays in,
 * an array out, as a host program holds them): x, q2 HOST [n], out HOST
 * [n][n_pid].  The library streams the points through device staging buffers
 * it owns (chunks of 2^18 points, or $PDFGPU_HOST_CHUNK read at the first
 * call, overlapped on three internal streams), and returns when `out` is
 * complete (synchronous).  Pinned host memory gives full copy bandwidth;
 * pageable memory works.  Calls on the same grid are serialised.  Domain
 * errors as for xfxQ2 (NaN rows, status bits).  On a failure the copies
 * already queued are drained before the call returns (nothing writes to
 * `out` afterwards; `out` is then partly written). */
int xfxQ2_host(pdfgpu_grid_t g, int32_t member, const int32_t *pids, int32_t n_pid,
               const double *x, const double *q2, int64_t n, double *out);

/* Adjoint of xfxQ2 / xfxQ2_pw.  Beyond the paper: the differentiation form,
 * d(x*f)/dx, d(x*f)/dQ^2 and d(x*f)/d(knot values) of the interpolant of
 * Sec. 2.1, the last being what a fit of the grid values needs (Sec. 1:
 * PDFs come from fits).
 * For L = sum_i sum_p grad_out[i][p] * xf_{pid_p}(x_i, Q^2_i):
 *   pointwise == 0: pids HOST [n_pid] (shared), grad_out DEVICE [n][n_pid]
 *   pointwise != 0: pids DEVICE [n] (one per point, n_pid ignored), grad_out DEVICE [n]
 *   grad_x  DEVICE [n] or NULL: dL/dx_i      (overwritten)
 *   grad_q2 DEVICE [n] or NULL: dL/dQ^2_i    (overwritten)
 *   grad_values DEVICE [n_rows][n_x][n_flav] of `member`, or NULL: dL/dvalues,
 *     ACCUMULATED (+=) with FP64 atomics (summation order is not fixed).
 * Domain errors give NaN in grad_x / grad_q2 and add nothing to grad_values.
 * PDF_E_ARG for a grid loaded with PDF_EXTRAP_CONTINUATION. */
int xfxQ2_backward(pdfgpu_grid_t g, int32_t member, const int32_t *pids, int32_t n_pid,
                   int32_t pointwise, const double *x, const double *q2, int64_t n,
                   const double *grad_out, double *grad_x, double *grad_q2,
                   double *grad_values, pdfgpu_stream_t stream);

/* Adjoint tape (an addition beyond the paper, for the differentiation above):
 * the forward calls below are xfxQ2 / xfxQ2_pw that also write, per point, a
 * 32-byte record of what the adjoint needs about the point's position in the
 * grid (both cells, both local coordinates, range and domain flags), so that
 * xfxQ2_backward_tape skips the knot searches and logarithms.
 *   tape DEVICE [n][4] doubles, caller-owned, 32-byte aligned (PDF_E_ARG
 *   otherwise); its content is private to the library.  A tape depends on
 *   the points, the grid's knots and its extrapolation option only, not on
 *   the member or the values: it stays valid across pdf_bind_values and for
 *   every member of the grid.  PDF_E_ARG for a grid loaded with
 *   PDF_EXTRAP_CONTINUATION (which has no adjoint) and for a NULL tape
 *   when n > 0 (with n == 0 the calls do nothing, and the tape may be NULL).
 *   dtape (xfxQ2_pw_tape only; may be NULL) DEVICE, 20 bytes per point:
 *   [n][2] doubles then [n] int32, caller-owned, 16-byte aligned (PDF_E_ARG
 *   otherwise, and without a tape; PDF_E_RANGE for a grid of 2^28 or more
 *   cell-flavour pairs): the derivative tape, each point's patch
 *   derivatives in its two local coordinates (zeros for an absent pid),
 *   computed with the value (13 FMAs more per point), and the point's bin
 *   in the sorted grid gradient, so that xfxQ2_backward_tape given it takes
 *   dL/dx and dL/dQ^2 without reloading the point's 16 coefficients and
 *   counts its bins from 4 bytes per point.  Unlike the tape it depends on
 *   the values bound and on the member: it is valid only while the values
 *   of the forward call are bound, for the same member.
 * Outputs of the forward calls are bit for bit those of xfxQ2 / xfxQ2_pw. */
int xfxQ2_tape(pdfgpu_grid_t g, int32_t member, const int32_t *pids, int32_t n_pid,
               const double *x, const double *q2, int64_t n, double *out, double *tape,
               pdfgpu_stream_t stream);
int xfxQ2_pw_tape(pdfgpu_grid_t g, int32_t member, const int32_t *pid, const double *x,
                  const double *q2, int64_t n, double *out, double *tape, double *dtape,
                  pdfgpu_stream_t stream);

/* xfxQ2_backward from the tape a forward call wrote for the same grid and the
 * same points (beyond the paper: the differentiation form, as above) (x and q2 are still read, for the chain rule of grad_x and
 * grad_q2).  Same arguments and results as xfxQ2_backward, bit for bit in
 * grad_x and grad_q2, with or without the derivative tape dtape (NULL, or
 * the one xfxQ2_pw_tape wrote with this tape: pointwise form only, PDF_E_ARG
 * otherwise; the forward's values must still be bound).  A tape of other
 * points or another grid gives wrong numbers; its cells are clamped into the
 * grid's tables, so no access leaves them. */
int xfxQ2_backward_tape(pdfgpu_grid_t g, int32_t member, const int32_t *pids, int32_t n_pid,
                        int32_t pointwise, const double *x, const double *q2, int64_t n,
                        const double *tape, const double *dtape, const double *grad_out,
                        double *grad_x, double *grad_q2, double *grad_values, pdfgpu_stream_t stream);

/* One request of a batched evaluation (several grids, members, flavour
 * subsets and sizes in one launch).  grid/member/pids are read at prepare
 * time; x, q2, out are DEVICE pointers that must stay valid while the batch
 * exists (the launch reads and writes them on every pdf_batch_run). */
typedef struct {
    pdfgpu_grid_t grid;
    int32_t member;
    int32_t n_pid;                  /* 1..16 */
    int32_t pids[16];
    const double *x;
    const double *q2;
    int64_t n;
    double *out;                    /* [n][n_pid] */
} pdfgpu_batch_desc;

/* Prepare a batched evaluation: choose the launch shape with the autotuner
 * (block size, points per thread, shared-memory staging of the knot tables;
 * results cached per workload signature in the JSON file named by
 * $PDFGPU_TUNE_CACHE, if set), upload the request table and capture one
 * persistent launch in a CUDA graph (the counterpart of PDFFlow's `trace()`
 * warm-up, Sec. 2.1).  Tuning runs the kernel on `stream` (outputs are
 * written).  Synchronous. */
int pdf_batch_prepare(const pdfgpu_batch_desc *descs, int32_t n_desc, int32_t autotune,
                      pdfgpu_stream_t stream, pdfgpu_batch_t *out);

/* Replay the captured launch on `stream`: evaluates every request (the
 * traced graph's execution, PDFFlow Sec. 2.1).  Makes the batch's device
 * current for the launch; the caller's current device is restored. */
int pdf_batch_run(pdfgpu_batch_t b, pdfgpu_stream_t stream);

/* Chosen launch shape: threads per block, points per thread, staging flag,
 * persistent CTAs, and the tuned time of one launch (ms); and the release
 * of a prepared batch.  Beyond the paper: the batching form's autotuner and
 * its lifetime (PDFFlow's `trace()` of Sec. 2.1 has no such handle). */
int pdf_batch_info(pdfgpu_batch_t b, int32_t *block, int32_t *qpt, int32_t *stage,
                   int32_t *ctas, float *ms);
int pdf_batch_free(pdfgpu_batch_t b);

/* Batched evaluation that allocates nothing (the paper has no counterpart).
 * For callers that cannot allocate device memory when they evaluate: a host
 * framework that reserved all device memory up front, or an event loop that
 * must not call cudaMalloc (it can fail on a full device and can synchronise
 * the whole device).  Evaluates the requests like pdf_batch_prepare +
 * pdf_batch_run, in one launch of the same persistent kernel with a fixed
 * shape (256 threads, 2 points per thread), but keeps its scratch -- the tile
 * ticket and the request and grid tables -- in one static device array of the
 * library (about 85 KB, held on every GPU that loads the library until the
 * process exits) instead of allocating per batch.  Limits: 1..1024 requests
 * and at most 32 distinct grids per call; beyond them the call fails with
 * PDF_E_RANGE before touching the GPU.  descs is HOST memory read during the
 * call; x, q2, out are DEVICE pointers used by the launch on `stream`.  The
 * first call on a device looks up the array's device address once, with that
 * device current; make that first call before any stream capture.  Every call
 * shares the one array and overwrites it (the ticket is reset on each call):
 * calls that overlap on the GPU (different streams) race; serialise them.
 * Asynchronous on `stream`. */
int pdf_batch_run_noalloc(const pdfgpu_batch_desc *descs, int32_t n_desc, pdfgpu_stream_t stream);

/* Fused parton-luminosity workload (PDFFlow Sec. 3.1-3.2: event kinematics,
 * two xfxQ2 calls, luminosity formed from the products).  Per event e:
 *   ln x1 = ln_tau/2 + y, ln x2 = ln_tau/2 - y, ln Q^2 = ln_tau + ln_s;
 *   flags bit 0: ln Q^2 = ln_mu2[e]; flags bit 1: ln x1 = ln_x1[e];
 *   lum[e] = sum_a xf_a(x1, Q^2) * xf_{-a}(x2, Q^2) over the grid's pids
 *            (the gluon pairs with itself);  alphas[e] = alpha_s(Q^2).
 *   *L = (1/n) sum_e lum[e], summed in a fixed order (deterministic).
 * Inputs DEVICE [n]: ln_tau, y, flags (uint8); ln_mu2, ln_x1 may be NULL when
 * no flag uses them.  Outputs DEVICE: lum [n] or NULL, alphas [n] or NULL
 * (NULL also when the grid has no alpha_s), L one double, and save_p
 * [n][2][n_flav] or NULL: the two partons' x*f values that have a partner
 * flavour, kept for pdf_lumi_backward.  An event with ln x > 0 or a
 * non-finite input gives NaN and sets PDF_S_DOMAIN.  Uses library-owned
 * scratch of the grid handle for the block partial sums: calls on the same
 * grid must not overlap in time.  Luminosity supports at most 16 flavours. */
int pdf_lumi(pdfgpu_grid_t g, int32_t member, const double *ln_tau, const double *y,
             const uint8_t *flags, const double *ln_mu2, const double *ln_x1, double ln_s,
             int64_t n, double *lum, double *alphas, double *L, double *save_p,
             pdfgpu_stream_t stream);

/* dL/dvalues of `member` for L of pdf_lumi, times the HOST scalar dL (beyond
 * the paper: the differentiation form of the Sec. 3.1-3.2 luminosity):
 * grad_values DEVICE [n_rows][n_x][n_flav], ACCUMULATED (+=) with FP64
 * atomics (summation order not fixed).  saved_p: the save_p array of the
 * forward call on the same events and values (DEVICE, read only), or NULL to
 * recompute those values.  Events with a domain error add nothing.  Uses
 * library-owned scratch of the grid handle (allocated on first use, about
 * 0.3 KB per event for up to 8.4e6 events per chunk, or 40 B per event when
 * saved_p is given): calls on the same grid must not overlap in time.
 * PDF_E_ARG for a grid loaded with PDF_EXTRAP_CONTINUATION. */
int pdf_lumi_backward(pdfgpu_grid_t g, int32_t member, const double *ln_tau, const double *y,
                      const uint8_t *flags, const double *ln_mu2, const double *ln_x1,
                      double ln_s, int64_t n, double dL, const double *saved_p,
                      double *grad_values, pdfgpu_stream_t stream);

/* Adaptive Monte Carlo integration of the parton luminosity (PDFFlow Sec.
 * 3.1: VegasFlow importance sampling around an integrand that calls the
 * PDFs; the matrix element is 1 here):
 *   I = int_0^1 dr1 dr2 F(r1, r2),  ln tau = (1 - r1) ln_tau_min,
 *   y = (2 r2 - 1)(-ln tau / 2),  ln x1,2 = ln tau / 2 +- y,
 *   ln Q^2 = ln tau + ln_s,  F = (-ln_tau_min)(-ln tau) sum_a xf_a(x1) xf_-a(x2),
 * sampled through the VEGAS map (Lepage, J. Comput. Phys. 27 (1978) 192):
 * per dimension n_bins bins with edges 0 = e_0 < ... < e_n = 1; a uniform v
 * falls in bin i = floor(v n) and maps to r = e_i + (v n - i)(e_{i+1} - e_i)
 * with Jacobian n (e_{i+1} - e_i).
 * pdf_vegas_lumi_iteration evaluates one iteration:
 *   edges DEVICE [2][n_bins + 1], v DEVICE [n][2] uniforms in [0, 1),
 *   shift HOST scalar c (finite; PDF_E_ARG otherwise),
 *   sums DEVICE [2 + 2 n_bins] (overwritten): sum w, sum (w - c)^2, then per
 *   bin the sum of w^2 for dimension 0 and for dimension 1, w = F(r) x
 *   Jacobian.  With c near the mean (the previous iteration's estimate) the
 *   variance (sum (w - c)^2 / n - (mean - c)^2) / (n - 1) is a sum of small
 *   squares instead of the difference of two nearly equal sums.
 * 2 <= n_bins <= 1024, ln_tau_min < 0.  Uses the grid handle's scratch for
 * block partial sums (calls on one grid must not overlap).  Asynchronous.
 * pdf_vegas_refine moves one dimension's HOST edges [n_bins + 1] from its
 * HOST per-bin sums of w^2: smoothing with the neighbours, damping
 * r_i = ((1 - d_i) / ln(1 / d_i))^alpha (d_i normalised), and new edges that
 * give every bin an equal share of sum r_i.  Host only. */
int pdf_vegas_lumi_iteration(pdfgpu_grid_t g, int32_t member, double ln_tau_min, double ln_s,
                             int32_t n_bins, const double *edges, const double *v, int64_t n,
                             double shift, double *sums, pdfgpu_stream_t stream);
int pdf_vegas_refine(const double *bin_w2, int32_t n_bins, double alpha, double *edges);

/* LHAPDF grid files (PDFFlow Sec. 1 and 4 keep the community "lhagrid1"
 * format and folder layout).  HOST only: no GPU call is made.
 * pdf_lhapdf_open reads members [first_member, first_member + n_members) of
 * the set in folder `set_dir` (files <name>/<name>.info and
 * <name>_<mmmm>.dat, <name> = the folder's last path component).  In a member
 * file, after the header line "---", each Q subgrid block is: a line of x
 * knots, a line of Q knots (GeV), a line of PDG ids, then n_x * n_q lines of
 * x*f values (x knot outer, Q knot inner), closed by "---".  All subgrids must
 * share the x knots and flavours; all members must share the knots.
 * AlphaS_Qs / AlphaS_Vals of the .info file are used when the Q list equals
 * the grid's Q knots.  Errors: PDF_E_ARG (missing file), PDF_E_DESC
 * (malformed), PDF_E_RANGE (members beyond NumMembers).
 * pdf_lhapdf_desc fills a description (interp and extrap 0) whose arrays
 * belong to the handle and stay valid until pdf_lhapdf_close; pass it to
 * pdf_load_grid. */
typedef struct pdfgpu_lhapdf *pdfgpu_lhapdf_t;
int pdf_lhapdf_open(const char *set_dir, int32_t first_member, int32_t n_members,
                    pdfgpu_lhapdf_t *out);
int pdf_lhapdf_desc(pdfgpu_lhapdf_t h, pdfgpu_grid_desc *desc);
int pdf_lhapdf_close(pdfgpu_lhapdf_t h);

/* Read and clear the grid's status word (PDF_S_* bits).  Synchronises
 * `stream` first.  Beyond the paper: failure detection for the batched
 * calls of Sec. 2.1, whose per-element domain errors do not fail a call. */
int pdf_get_status(pdfgpu_grid_t g, pdfgpu_stream_t stream, uint32_t *bits);

/* General VEGAS (Lepage, J. Comput. Phys. 27 (1978) 192) around an
 * integrand the caller evaluates: in the paper's use (Sec. 3.1) the
 * integrand, a matrix element times PDFs, is user code that calls the PDF
 * interface.  One iteration over [0, 1]^dim is
 *   pdf_vegas_map -> r, J, bins;  f(r) by the caller's own kernels (for
 *   example with xfxQ2);  w = f J;  pdf_vegas_accumulate(w, bins) -> sums;
 *   pdf_vegas_refine for each dimension (host).
 * pdf_vegas_map: edges DEVICE [dim][n_bins + 1] (0 = e_0 < ... < e_n = 1 per
 *   dimension), v DEVICE [n][dim] uniforms in [0, 1) (values outside are
 *   clamped into the first / last bin), r DEVICE [n][dim] out: r = e_b +
 *   (v n - b)(e_{b+1} - e_b) with b = floor(v n); jac DEVICE [n] out: the
 *   product over dimensions of n (e_{b+1} - e_b); bins DEVICE [n][dim] int32
 *   out.
 * pdf_vegas_accumulate: w DEVICE [n] weights, bins DEVICE [n][dim] as from
 *   pdf_vegas_map (entries outside [0, n_bins) are left out of the per-bin
 *   sums), shift HOST scalar c (finite), sums DEVICE [2 + dim n_bins]
 *   (overwritten): sum w, sum (w - c)^2, then per dimension the per-bin sums
 *   of w^2.  Summation order is not fixed.
 * 1 <= dim <= 16, 2 <= n_bins <= 1024.  Asynchronous on `stream`; no grid
 * handle and no library-owned scratch, so calls on different streams are
 * independent.  The library has no counterpart of the caller's integrand. */
int pdf_vegas_map(int32_t dim, int32_t n_bins, const double *edges, const double *v, int64_t n, double *r,
                  double *jac, int32_t *bins, pdfgpu_stream_t stream);
int pdf_vegas_accumulate(int32_t dim, int32_t n_bins, const double *w, const int32_t *bins, int64_t n,
                         double shift, double *sums, pdfgpu_stream_t stream);

/* Message of the last failed call on this thread ("" if none).  Beyond the
 * paper: the error channel of this C interface (the paper's interface is
 * Python, Sec. 2.1). */
const char *pdf_last_error(void);

/* Measurement helpers (not part of the interpolation; beyond the paper, the
 * denominators of this GPU's FP64 roofline):
 * FP64 FMA throughput of this GPU in FLOP/s (2 per FMA), from a kernel of
 * independent fused multiply-add chains timed with CUDA events. Synchronous. */
int pdf_probe_fp64_peak(double *flops);

/* Throughput of sm_103a's FP64 tensor instruction, mma.sync with f64
 * operands (the only FP64 matrix path of this GPU; tcgen05 has no f64 kind),
 * in FLOP/s (2 M N K per warp-wide instruction), from a kernel of eight
 * independent accumulator chains per warp timed with CUDA events.
 * shape 0: m8n8k4, 1: m16n8k4, 2: m16n8k8, 3: m16n8k16; PDF_E_ARG otherwise.
 * Beyond the paper: measures whether the interpolation's contraction could
 * leave the DFMA pipe of this GPU.  Synchronous. */
int pdf_probe_fp64_mma_peak(int32_t shape, double *flops);

/* Whether the FP64 tensor instruction runs beside the FMA pipe or on it: a
 * kernel whose warps each issue equal FP64 work (in flops) as DFMA chains and
 * as m8n8k4 mma.sync chains is timed with the DFMA half alone, the DMMA half
 * alone, and both interleaved; the outputs are the three rates in FLOP/s.
 * A mixed rate near the harmonic combination of the two (rather than their
 * sum) says the two share one pipe.  Beyond the paper.  Synchronous. */
int pdf_probe_fp64_mixed(double *dfma_flops, double *dmma_flops, double *mixed_flops);

/* (Beyond the paper: a test hook.)  The kernels' natural log (table-driven argument reduction after
 * P. T. P. Tang, ACM TOMS 16 (1990) 378, with a degree-5 series for
 * ln(1+r), |r| <= 2^-11) applied to n DEVICE doubles: out[i] = ln(in[i]) for
 * positive finite in[i].  Exposed for tests. */
int pdf_debug_log(pdfgpu_grid_t g, const double *in, int64_t n, double *out,
                  pdfgpu_stream_t stream);

/* (Beyond the paper: a test hook.)  The cells the kernels' knot searches give
 * for n DEVICE points x, q2 (positive, finite): x_cell[i], q_cell[i] DEVICE
 * int32, the largest cell whose lower knot is at or below the point (0 below
 * the grid, the last cell above it; a Q^2 on an internal threshold is in the
 * upper subgrid's first cell), and in guided (HOST [2], may be NULL) whether
 * the x and the Q^2 search run through a guide table (else by bisection). */
int pdf_debug_cells(pdfgpu_grid_t g, const double *x, const double *q2, int64_t n, int32_t *x_cell,
                    int32_t *q_cell, int32_t *guided, pdfgpu_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* PDFGPU_H */
