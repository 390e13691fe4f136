"""Plant one plausible mistake at a time in a copy of the oracle and check that
at least one pin catches it (CPU only; the committed oracle is untouched).

Each mutation is a textual substitution that must match exactly once in the
oracle source, so a refactor of the oracle that removes the mutated line is
reported instead of silently passing.
"""
import os

import pytest

import oracle
import pins

MUTANTS = {
    # depth operator X
    "drop_minus_2s": ("*mid = (n2_m[l] - 1.0) - 2.0 * s;", "*mid = (n2_m[l] - 1.0);"),
    "drop_minus_1": ("*mid = (n2_m[l] - 1.0) - 2.0 * s;", "*mid = n2_m[l] - 2.0 * s;"),
    "s_without_k0": ("const double s = 1.0 / ((k0 * dz) * (k0 * dz));",
                     "const double s = 1.0 / (dz * dz);"),
    "x_lower_index": ("if (l > 0) xw = xw + lo * wm[l - 1];", "if (l > 0) xw = xw + lo * wm[l];"),
    # the scheme's coefficients
    "delta_sign": ("const cplx delta = I * (k0 * dr);", "const cplx delta = -I * (k0 * dr);"),
    "alpha_beta_swapped": ("const cplx alpha = 0.25 - delta / 4.0;",
                           "const cplx alpha = 0.25 + delta / 4.0;"),
    "beta_times_w": ("rhs[l] = wm[l] + beta * xw;", "rhs[l] = wm[l] + beta * wm[l];"),
    "y_factor_sign": ("dg[m] = 1.0 - yfac * (-2.0 * c);", "dg[m] = 1.0 + yfac * (-2.0 * c);"),
    # azimuth operator Y
    "c_without_r": ("const double c = 1.0 / ((k0 * rstar * dtheta) * (k0 * rstar * dtheta));",
                    "const double c = 1.0 / ((k0 * dtheta) * (k0 * dtheta));"),
    "theta_wrong_neighbour": ("+ theta_nb(u, Nz, Nt, periodic, m, -1, l));",
                              "+ theta_nb(u, Nz, Nt, periodic, m, +1, l));"),
    "periodic_corner_missing": ("cplx lo = (periodic || m > 0) ? c : 0.0;",
                                "cplx lo = (m > 0) ? c : 0.0;"),
    # range bookkeeping
    "rstar_at_rj": ("double rstar = r0 + (double)(j + 1) * dr;", "double rstar = r0 + (double)j * dr;"),
    # range interpolation of the medium
    "interp_t_reversed": ("double t = (r - slice_r[k]) / (slice_r[k + 1] - slice_r[k]);",
                          "double t = (slice_r[k + 1] - r) / (slice_r[k + 1] - slice_r[k]);"),
    "interp_weights_swapped": ("out[i] = (1.0 - t) * a[i] + t * b[i];",
                               "out[i] = t * a[i] + (1.0 - t) * b[i];"),
    "interp_same_slice": ("*b = n2 + (size_t)(k + 1) * npts;", "*b = n2 + (size_t)k * npts;"),
    "interp_ignored": ("        if (interp) {", "        if (0) {"),
    "interp_hold_first": ("if (k + 1 >= K || r < slice_r[k]) {", "if (k + 1 >= K) {"),
    # the Taylor form of Eq. 3 and its banded solve
    "taylor_x2_sign": ("- (delta / 4.0) * xr[b] + (delta / 16.0) * x2[b];", "- (delta / 4.0) * xr[b] - (delta / 16.0) * x2[b];"),
    "taylor_drop_x2_rhs": ("rhs[l] = wm[l] + (delta / 4.0) * xw - (delta / 16.0) * x2w;",
                           "rhs[l] = wm[l] + (delta / 4.0) * xw;"),
    "x2_wrong_band": ("if (k + 1 < Nz) x2[(k + 1) - l + 2] += xlk * khi;", "if (k + 1 < Nz) x2[(k + 1) - l + 2] += xlk * kmid;"),
    "penta_no_interchange": ("        if (p != 0)\n            for (int c = j; c <= ju; ++c) {",
                             "        if (0)\n            for (int c = j; c <= ju; ++c) {"),
    "penta_forward_sign": ("for (int t = 1; t <= km; ++t) b[j + t] = b[j + t] - AB(PB_KV + t, j) * b[j];",
                           "for (int t = 1; t <= km; ++t) b[j + t] = b[j + t] + AB(PB_KV + t, j) * b[j];"),
    # solvers
    "backsub_index": ("- u2[i] * b[i + 2]) / d[i];", "- u2[i] * b[i + 1]) / d[i];"),
    "swap_fill_sign": ("if (i + 2 < n) u1[i + 1] = 0.0 - mult * r_i2;",
                       "if (i + 2 < n) u1[i + 1] = 0.0 + mult * r_i2;"),
    "sm_sign": ("for (int i = 0; i < n; ++i) b[i] = b[i] - f * z[i];",
                "for (int i = 0; i < n; ++i) b[i] = b[i] + f * z[i];"),
    "sm_corner_gamma": ("tdiag[n - 1] = diag[n - 1] - corner_bl * corner_tr / gamma;",
                        "tdiag[n - 1] = diag[n - 1];"),
}


@pytest.fixture(scope="module")
def source():
    with open(os.path.join(os.path.dirname(oracle.__file__), "pe3d_oracle.c")) as f:
        return f.read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, source, name):
    find, repl = MUTANTS[name]
    assert source.count(find) == 1, f"mutation anchor for {name} not unique in the oracle"
    src = tmp_path / f"mut_{name}.c"
    src.write_text(source.replace(find, repl))
    lib = oracle.OracleLib(oracle.build(str(src), str(tmp_path / f"mut_{name}.so")))
    failed = []
    for check, fn in pins.ALL_CHECKS.items():
        try:
            err = fn(lib)
        except (RuntimeError, FloatingPointError, ValueError):
            err = float("inf")
        if not err < pins.TOLS[check]:
            failed.append(check)
    assert failed, f"mutant {name} passed every pin"
