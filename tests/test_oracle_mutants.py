"""The pins are strong enough to catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of ``oracle/pdf_oracle.c`` (a dropped
or flipped term, a wrong index, a wrong tie-break...), builds it into a
separate shared object on the CPU, and runs a compact set of the pins against
it: at least one must fail.  The unmodified oracle passes all of them."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle.oracle as O
from oracle.bruteforce import ExactGrid
from paper_2012_08221_gb300 import synth
from tests.tinygrids import fill, tiny_two_sub

SRC = os.path.join(os.path.dirname(O.__file__), "pdf_oracle.c")

MUTANTS = {
    "hermite h10 sign": ("double h10 = t * s2;", "double h10 = -t * s2;"),
    "hermite h01 coefficient": ("double h01 = t2 * (3.0 - 2.0 * t);", "double h01 = t2 * (2.0 - 2.0 * t);"),
    "hermite h00 factor": ("double h00 = s2 * (1.0 + 2.0 * t);", "double h00 = s2 * (1.0 + t);"),
    "hermite derivative e10 sign": ("double e10 = s * (1.0 - 3.0 * t);", "double e10 = s * (1.0 + 3.0 * t);"),
    "hermite derivative dropped": ("return h00 * g0 + h10 * dz * d0 + h01 * g1 + h11 * dz * d1;",
                                   "return h00 * g0 + h10 * dz * d0 + h01 * g1;"),
    "interior slope one-sided": (
        "return 0.5 * ((gp - g0) / (z[k + 1] - z[k]) + (g0 - gm) / (z[k] - z[k - 1]));",
        "return (gp - g0) / (z[k + 1] - z[k]);"),
    "first-knot slope zero": ("if (k == 0) return (gp - g0) / (z[1] - z[0]);", "if (k == 0) return 0.0;"),
    "last-knot slope transposed": ("if (k == n - 1) return (g0 - gm) / (z[n - 1] - z[n - 2]);",
                                   "if (k == n - 1) return (gm - g0) / (z[n - 1] - z[n - 2]);"),
    "threshold to lower subgrid": ("        if (W[g->row0[j]] <= w) s = j;\n    int n = g->n_q[s], r0 = g->row0[s];",
                                   "        if (W[g->row0[j]] < w) s = j;\n    int n = g->n_q[s], r0 = g->row0[s];"),
    "w extrapolation rows": ("int r0 = w < W[0] ? 0 : last - 1;", "int r0 = w < W[0] ? 1 : last - 1;"),
    "u extrapolation columns": ("int k0 = u < U[0] ? 0 : n - 2;", "int k0 = u < U[0] ? 1 : n - 2;"),
    "w-derivative sign": ("if (dw) *dw = (B1 - B0) / dz;\n        if (du)",
                          "if (dw) *dw = (B0 - B1) / dz;\n        if (du)"),
    "row stencil shifted": ("double gm = k > 0 ? val(a, row, k - 1) : 0.0;",
                            "double gm = k > 1 ? val(a, row, k - 2) : 0.0;"),
}


LUMI_MUTANTS = {
    "luminosity pairs a with a": ("double f2 = orc_xfxq2_uw(g, member, -pa, u2, w, NULL, NULL);",
                                  "double f2 = orc_xfxq2_uw(g, member, pa, u2, w, NULL, NULL);"),
    "second parton's rapidity sign": ("*u2 = h - y;", "*u2 = h + y;"),
    "tail replaces the wrong parton's x": ("if (flags & 2u) *u1 = ln_x1;", "if (flags & 2u) *u2 = ln_x1;"),
    "factorisation scale ignores the tail": ("if (flags & 1u) *w = ln_mu2;", "if (flags & 1u) *w = ln_tau + ln_s;"),
}


VEGAS_MUTANTS = {
    "VEGAS Jacobian without the bin count": ("jac *= n_bins * width;", "jac *= width;"),
    "VEGAS bin index off by one": ("double vn = v[2 * i + d] * n_bins;\n            int b = (int)vn;",
                                   "double vn = v[2 * i + d] * n_bins;\n            int b = (int)vn + 1;"),
    "general VEGAS map without the bin count in the Jacobian": ("j *= n_bins * width;", "j *= width;"),
    "general VEGAS map bin index off by one": ("double vn = v[i * dim + d] * n_bins;\n            int b = (int)vn;",
                                               "double vn = v[i * dim + d] * n_bins;\n            int b = (int)vn + 1;"),
    "general VEGAS accumulate drops the square": ("out[2 + d * n_bins + bins[i * dim + d]] += wi * wi;",
                                                  "out[2 + d * n_bins + bins[i * dim + d]] += wi;"),
    "VEGAS tau mapped the other way": ("double ln_tau = (1.0 - r[0]) * ln_tau_min;",
                                       "double ln_tau = r[0] * ln_tau_min;"),
    "VEGAS second moment ignores the shift": ("out[1] += (wt - shift) * (wt - shift);", "out[1] += wt * wt;"),
    "general VEGAS second moment ignores the shift": ("out[1] += (wi - shift) * (wi - shift);",
                                                      "out[1] += wi * wi;"),
}


GRAD_MUTANTS = {
    "chain rule multiplies by x": ("*dx = du / x;", "*dx = du * x;"),
    "alpha_s derivative left in ln Q^2": ("*dq2 = dw / q2;\n    return v;\n}\n\ndouble orc_alphas(",
                                          "*dq2 = dw;\n    return v;\n}\n\ndouble orc_alphas("),
    "indicator scan drops the last stencil knot": (
        "*c1 = k + 3 > g->n_x - 1 ? g->n_x - 1 : k + 3;", "*c1 = k + 1 > g->n_x - 1 ? g->n_x - 1 : k + 1;"),
    "grid gradient ignores the point weights": ("double t = gw[i] * wt;", "double t = wt;"),
}


CONT_MUTANTS = {
    "continuation anchored at the wrong knot": ("double y = y0 * exp(t * lr);", "double y = y1 * exp(t * lr);"),
    "continuation threshold on one value only": ("if (y0 > CONT_MIN && y1 > CONT_MIN) {",
                                                 "if (y0 > CONT_MIN) {"),
    "corners continued by a straight line in u": (
        "double A0 = wdir(a, &c0, w, &dw0, NULL), A1 = wdir(a, &c1, w, &dw1, NULL);\n        double dz = U[k0 + 1] - U[k0];\n        if (g->extrap == 3) {",
        "double A0 = wdir(a, &c0, w, &dw0, NULL), A1 = wdir(a, &c1, w, &dw1, NULL);\n        double dz = U[k0 + 1] - U[k0];\n        if (g->extrap == 3 && w >= g->W[0] && w <= g->W[g->rows - 1]) {"),
}


def build_variant(tmp, text):
    src = os.path.join(tmp, "orc.c")
    with open(src, "w") as f:
        f.write(text)
    so = os.path.join(tmp, "liborc_variant.so")
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", src, "-o", so, "-lm"],
                   check=True)
    return O.load_library(so)


def pin_failures():
    """Names of the compact pins that fail with the currently loaded oracle."""
    fails = []
    # knot values, including thresholds, on a two-subgrid grid
    g = tiny_two_sub(seed=41, dup_equal=False)
    o = O.OracleGrid.from_synth(g)
    starts = np.concatenate([[0], np.cumsum(g.n_q)[:-1]])
    for r in range(g.n_rows):
        row = r + 1 if any(r == s + n - 1 for s, n in zip(starts[:-1], g.n_q[:-1])) else r
        for k in range(g.n_x):
            if o.xfxq2(g.pids[0], g.x_knots[k], g.q_knots[r] ** 2) != g.values[0, row, k, 0]:
                fails.append("knots")
                break
        if fails:
            break
    # log-bilinear data everywhere (inside and outside), with derivatives
    gl = fill(synth.grid_small(), lambda U, W: 0.7 - 0.3 * U + 0.05 * W + 0.01 * U * W)
    ol = O.OracleGrid.from_synth(gl)
    rng = np.random.default_rng(42)
    for u, w in zip(rng.uniform(-22, 0, 200), rng.uniform(-1, 22, 200)):
        v, du, dw = ol.xfxq2_uw(0, u, w)
        if (abs(v - (0.7 - 0.3 * u + 0.05 * w + 0.01 * u * w)) > 1e-12 or
                abs(du - (-0.3 + 0.01 * w)) > 1e-11 or abs(dw - (0.05 + 0.01 * u)) > 1e-11):
            fails.append("bilinear")
            break
    # quadratic in u: interior exact, first interval h^2 t (1-t)^2
    gq = fill(synth.grid_small(), lambda U, W: U * U + 0 * W)
    oq = O.OracleGrid.from_synth(gq)
    U = np.log(gq.x_knots)
    h = U[1] - U[0]
    for k, t in [(0, 0.3), (10, 0.4), (30, 0.8)]:
        u = U[k] + t * (U[k + 1] - U[k])
        want = u * u + (h * h * t * (1 - t) ** 2 if k == 0 else 0.0)
        if abs(oq.xfxq2_uw(0, u, math.log(50.0))[0] - want) > 1e-11 * (1 + u * u):
            fails.append("quadratic")
            break
    # exact-rational brute force on the two-subgrid grid
    Wsub = [o.W[0:3], o.W[3:6]]
    ex = ExactGrid(o.U, Wsub, [g.values[0, 0:3, :, 0], g.values[0, 3:6, :, 0]])
    for u, w in zip(rng.uniform(o.U[0] - 1, 0, 40), rng.uniform(o.W[0] - 1, o.W[-1] + 1, 40)):
        if abs(o.xfxq2_uw(g.pids[0], u, w)[0] - float(ex.eval(u, w)[0])) > 1e-13:
            fails.append("brute force")
            break
    return fails


FLAVOUR_MUTANTS = {
    "a grid's gluon listed as 21 not recognised": (
        "static int grid_pid(const orc_grid *g, int a) { return g->pids[a] == 21 ? 0 : g->pids[a]; }",
        "static int grid_pid(const orc_grid *g, int a) { return g->pids[a]; }"),
    "a query's pid 21 not mapped to the gluon": ("    if (pid == 21) pid = 0;\n", ""),
}


def flavour_pin_fails():
    """Gluon as 0 or 21, in the query and in the grid's flavour list."""
    g0 = tiny_two_sub(seed=43)
    p21 = g0.pids.copy()
    p21[p21 == 0] = 21
    g21 = synth.Grid(g0.x_knots, g0.n_q, g0.q_knots, p21, g0.values, g0.alphas, "g21")
    o0, o21 = O.OracleGrid.from_synth(g0), O.OracleGrid.from_synth(g21)
    x, q2 = np.array([3e-4, 0.02, 0.5]), np.array([1.5, 4.0, 30.0])
    ref = o0.xfxq2_batch([0], x, q2)
    return not (np.array_equal(o0.xfxq2_batch([21], x, q2), ref) and
                np.array_equal(o21.xfxq2_batch([0], x, q2), ref) and
                np.array_equal(o21.xfxq2_batch([21], x, q2), ref) and np.any(ref != 0.0))


def test_unmodified_oracle_passes_the_flavour_pin():
    assert not flavour_pin_fails()


@pytest.mark.parametrize("name", sorted(FLAVOUR_MUTANTS))
def test_planted_flavour_mistake_is_caught(name, tmp_path, swap_oracle):
    old, new = FLAVOUR_MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site not unique: {name}"
    O._lib = build_variant(str(tmp_path), text.replace(old, new))
    assert flavour_pin_fails(), f"no pin catches: {name}"


@pytest.fixture
def swap_oracle():
    saved = O._lib
    yield
    O._lib = saved


def test_unmodified_oracle_passes_the_compact_pins():
    assert pin_failures() == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path, swap_oracle):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site not unique: {name}"
    O._lib = build_variant(str(tmp_path), text.replace(old, new))
    assert pin_failures(), f"no pin catches: {name}"
    shutil.rmtree(tmp_path, ignore_errors=True)


def lumi_pin_fails():
    """The closed-form luminosity pin (flavour-dependent log-bilinear data)."""
    from tests.closed_forms import bilinear_flavour_grid, luminosity
    g, params = bilinear_flavour_grid(synth.grid_nnpdf())
    o = O.OracleGrid.from_synth(g)
    ev = synth.events_lhc(2000, seed=81, tail=0.3)
    _, lum, _ = o.lumi(ev)
    want, mag, _ = luminosity(g.pids, params, ev)
    return not np.all(np.abs(lum - want) <= 1e-13 * mag + 1e-15)


def test_unmodified_oracle_passes_the_luminosity_pin():
    assert not lumi_pin_fails()


@pytest.mark.parametrize("name", sorted(LUMI_MUTANTS))
def test_planted_luminosity_mistake_is_caught(name, tmp_path, swap_oracle):
    old, new = LUMI_MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site not unique: {name}"
    O._lib = build_variant(str(tmp_path), text.replace(old, new))
    assert lumi_pin_fails(), f"no pin catches: {name}"
    shutil.rmtree(tmp_path, ignore_errors=True)


def vegas_pins_fail():
    """The two closed-form VEGAS pins: identity map sample by sample, and a
    non-uniform map integrated exactly by a midpoint lattice."""
    from tests import test_oracle_vegas as V
    try:
        V.test_identity_map_on_constant_grid_is_the_closed_form()
        V.test_non_uniform_map_midpoint_rule_is_exact()
        V.test_general_map_midpoint_lattice_is_exact_for_multilinear_integrands()
        V.test_general_map_and_accumulate_reproduce_the_fused_luminosity_sums()
        V.test_second_moment_about_a_shift()
    except AssertionError:
        return True
    return False


def test_unmodified_oracle_passes_the_vegas_pins():
    assert not vegas_pins_fail()


@pytest.mark.parametrize("name", sorted(VEGAS_MUTANTS))
def test_planted_vegas_mistake_is_caught(name, tmp_path, swap_oracle):
    old, new = VEGAS_MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site not unique: {name}"
    O._lib = build_variant(str(tmp_path), text.replace(old, new))
    assert vegas_pins_fail(), f"no pin catches: {name}"
    shutil.rmtree(tmp_path, ignore_errors=True)


def gradient_pins_fail():
    """The derivative pins: central differences of x*f and alpha_s, the
    linear response of one grid value, and the full indicator scan."""
    from tests import test_oracle_pins as P
    small, nnpdf = synth.grid_small(), synth.grid_nnpdf()
    try:
        P.test_gradients_against_central_differences(small)
        P.test_grid_gradient_is_linear_response(small)
        P.test_alphas_derivative_against_central_differences(nnpdf)
        P.test_window_holds_every_nonzero_weight()
    except AssertionError:
        return True
    return False


def test_unmodified_oracle_passes_the_gradient_pins():
    assert not gradient_pins_fail()


@pytest.mark.parametrize("name", sorted(GRAD_MUTANTS))
def test_planted_gradient_mistake_is_caught(name, tmp_path, swap_oracle):
    old, new = GRAD_MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site not unique: {name}"
    O._lib = build_variant(str(tmp_path), text.replace(old, new))
    assert gradient_pins_fail(), f"no pin catches: {name}"
    shutil.rmtree(tmp_path, ignore_errors=True)


def continuation_pins_fail():
    from tests import test_oracle_modes as M
    try:
        M.test_continuation_reproduces_power_laws_outside()
        M.test_continuation_inside_equals_linear_and_falls_back_where_not_positive()
    except AssertionError:
        return True
    return False


def test_unmodified_oracle_passes_the_continuation_pins():
    assert not continuation_pins_fail()


@pytest.mark.parametrize("name", sorted(CONT_MUTANTS))
def test_planted_continuation_mistake_is_caught(name, tmp_path, swap_oracle):
    old, new = CONT_MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site not unique: {name}"
    O._lib = build_variant(str(tmp_path), text.replace(old, new))
    assert continuation_pins_fail(), f"no pin catches: {name}"
    shutil.rmtree(tmp_path, ignore_errors=True)


KAPPA_MUTANTS = {
    "kappa takes every pid's values from the first pid's column": (
        "int col = pid_column(g, pointwise ? pids[i] : pids[p]);",
        "int col = pid_column(g, pointwise ? pids[i] : pids[0]);"),
    "kappa reads member 0 whatever the member": (
        "const double *vm = g->values + (size_t)member * g->rows * stride;",
        "const double *vm = g->values;"),
    "kappa keeps the sign of negative weights": (
        "kappa[i * np + p] += fabs(wt * vm[(size_t)r * stride + (size_t)k * g->n_flav + col]);",
        "kappa[i * np + p] += wt * fabs(vm[(size_t)r * stride + (size_t)k * g->n_flav + col]);"),
    "kappa scan drops the last stencil knot": (
        "for (int k = c0; k <= c1; ++k) {\n                double wt = orc_cell_weight_uw(g, r, k, u, w);\n"
        "                if (wt == 0.0) continue;\n                for (int p = 0; p < np; ++p) {",
        "for (int k = c0; k < c1; ++k) {\n                double wt = orc_cell_weight_uw(g, r, k, u, w);\n"
        "                if (wt == 0.0) continue;\n                for (int p = 0; p < np; ++p) {"),
    "pointwise gradient magnitudes without the point weight": (
        "double t = gw[i] * wt;\n                grad[((size_t)r * g->n_x + k) * g->n_flav + col] += absval ? fabs(t) : t;",
        "double t = gw[i] * wt;\n                grad[((size_t)r * g->n_x + k) * g->n_flav + col] += absval ? fabs(wt) : t;"),
    "matrix-form gradient magnitudes keep the sign": (
        "double t = gout[i * n_pid + p] * wt;\n                    grad[((size_t)r * g->n_x + k) * g->n_flav + col] "
        "+= absval ? fabs(t) : t;",
        "double t = gout[i * n_pid + p] * wt;\n                    grad[((size_t)r * g->n_x + k) * g->n_flav + col] "
        "+= absval ? t : t;"),
    "luminosity gradient magnitudes without the partner factor": (
        "grad[((size_t)r * g->n_x + k) * F + b] += absval ? fabs(t) : t;",
        "grad[((size_t)r * g->n_x + k) * F + b] += absval ? fabs(wt) : t;"),
    "alpha_s kappa keeps the sign of negative weights": (
        "sum += fabs(wdir(&a, &c, w, NULL, NULL) * g->alphas[r]);",
        "sum += wdir(&a, &c, w, NULL, NULL) * g->alphas[r];"),
    "alpha_s kappa takes every weight's value from the first knot of the window": (
        "sum += fabs(wdir(&a, &c, w, NULL, NULL) * g->alphas[r]);",
        "sum += fabs(wdir(&a, &c, w, NULL, NULL) * g->alphas[r0]);"),
}


def kappa_pins_fail():
    """The tolerance-scale pins: kappa, alpha_s kappa and the |term| sums of
    the gradients against exact weights, and kappa at knots."""
    from tests import test_oracle_kappa as K
    if K.kappa_vs_exact_weights(K.GRIDS[1], n=6) >= 1e-13:
        return True
    try:
        K.test_kappa_at_knots_is_the_magnitude_of_the_value(K.GRIDS[1])
    except AssertionError:
        return True
    return (K.dgrid_absval_vs_exact(n=6) >= 1e-13 or K.lumi_absval_vs_exact(n=5) >= 1e-13 or
            K.alphas_kappa_vs_exact(n=16) >= 1e-13)


def test_unmodified_oracle_passes_the_kappa_pins():
    assert not kappa_pins_fail()


@pytest.mark.parametrize("name", sorted(KAPPA_MUTANTS))
def test_planted_kappa_mistake_is_caught(name, tmp_path, swap_oracle):
    old, new = KAPPA_MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site not unique: {name}"
    O._lib = build_variant(str(tmp_path), text.replace(old, new))
    assert kappa_pins_fail(), f"no pin catches: {name}"
    shutil.rmtree(tmp_path, ignore_errors=True)
