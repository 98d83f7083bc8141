"""Plant plausible mistakes in copies of the oracle and check that the pins
catch each one.

Every mutant is a copy of oracle/oracle.c with one edit, compiled with gcc
into a temporary library and swapped in for the real one while a set of
independent checks runs (brute force over images, two-body closed form,
Newton's third law, lattice symmetry, exact binning, finite differences of
the Plummer and spline adjoints, the lattice constant of the far-field
tensor, far + near against the Ewald sum). A mutant that passes every check would mean the pins cannot
see that mistake. CPU only.
"""
import os
import subprocess

import pytest

import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")
FAR = os.path.join(os.path.dirname(oracle.__file__), "farfield.c")

MUTANTS = {
    "drop_eps2": ("double s = ddx * ddx + ddy * ddy + ddz * ddz + eps2;",
                  "double s = ddx * ddx + ddy * ddy + ddz * ddz + 0.0 * eps2 + 1e-300;"),
    "sign_of_delta": ("double ddx = (pos[3 * j + 0] - pos[3 * i + 0]) + sx;",
                      "double ddx = (pos[3 * i + 0] - pos[3 * j + 0]) + sx;"),
    "wrong_image_sign": ("double sx = (double)((tx - wx) / cpd) * L;\n            double sy = (double)((ty - wy) / cpd) * L;\n            double sz = (double)((tz - wz) / cpd) * L;\n            int64_t cc = ((int64_t)wx * cpd + wy) * cpd + wz;\n            for (int64_t k = start[cc]",
                         "double sx = -(double)((tx - wx) / cpd) * L;\n            double sy = (double)((ty - wy) / cpd) * L;\n            double sz = (double)((tz - wz) / cpd) * L;\n            int64_t cc = ((int64_t)wx * cpd + wy) * cpd + wz;\n            for (int64_t k = start[cc]"),
    "radius_short": ("        for (int dx = -R; dx <= R; ++dx)\n        for (int dy = -R; dy <= R; ++dy)\n        for (int dz = -R; dz <= R; ++dz) {\n            int tx = cx + dx, ty = cy + dy, tz = cz + dz;\n            int wx = wrap(tx, cpd), wy = wrap(ty, cpd), wz = wrap(tz, cpd);\n            double sx = (double)((tx - wx) / cpd) * L;\n            double sy = (double)((ty - wy) / cpd) * L;\n            double sz = (double)((tz - wz) / cpd) * L;\n            int64_t cc = ((int64_t)wx * cpd + wy) * cpd + wz;\n            for (int64_t k = start[cc]",
                     "        for (int dx = -R; dx <= R; ++dx)\n        for (int dy = -R; dy <= R; ++dy)\n        for (int dz = -R; dz < R; ++dz) {\n            int tx = cx + dx, ty = cy + dy, tz = cz + dz;\n            int wx = wrap(tx, cpd), wy = wrap(ty, cpd), wz = wrap(tz, cpd);\n            double sx = (double)((tx - wx) / cpd) * L;\n            double sy = (double)((ty - wy) / cpd) * L;\n            double sz = (double)((tz - wz) / cpd) * L;\n            int64_t cc = ((int64_t)wx * cpd + wy) * cpd + wz;\n            for (int64_t k = start[cc]"),
    "transposed_cell_id": ("cid[i] = (int32_t)(((int64_t)c3[0] * cpd + c3[1]) * cpd + c3[2]);",
                           "cid[i] = (int32_t)(((int64_t)c3[2] * cpd + c3[1]) * cpd + c3[0]);"),
    "sink_mass_instead": ("double mj = mass ? mass[j] : m0;\n                double f = mj / (s * sqrt(s));",
                          "double mj = mass ? mass[i] : m0;\n                double f = mj / (s * sqrt(s));"),
    "power_minus_one": ("double f = mj / (s * sqrt(s));", "double f = mj / s;"),
    "unstable_sort": ("    for (int64_t i = 0; i < n; ++i) {\n        int64_t k = cursor[cid[i]]++;\n        perm[k] = i;\n    }",
                      "    for (int64_t i = n - 1; i >= 0; --i) {\n        int64_t k = cursor[cid[i]]++;\n        perm[k] = i;\n    }"),
    "floor_to_round": ("    int c = (int)floor(u);\n    if (c >= cpd) c = cpd - 1;",
                       "    int c = (int)floor(u + 0.5);\n    if (c >= cpd) c = cpd - 1;"),
    "vjp_swap_masses": ("u[a] = mk * w[3 * j + a] - mj * w[3 * k + a];",
                        "u[a] = mj * w[3 * j + a] - mk * w[3 * k + a];"),
    "vjp_drop_factor3": ("gx += s32 * u[0] - 3.0 * s52 * D[0] * Du;",
                         "gx += s32 * u[0] - 1.0 * s52 * D[0] * Du;"),
    "vjp_sign": ("for (int a = 0; a < 3; ++a) u[a] = mk * w[3 * j + a] - mj * w[3 * k + a];",
                 "for (int a = 0; a < 3; ++a) u[a] = mj * w[3 * k + a] - mk * w[3 * j + a];"),
    "vjp_spline_inner_slope": ("dfr = (-15.0 + 12.0 * uu) / (eps2 * eps2 * r);",
                               "dfr = (-15.0 + 6.0 * uu) / (eps2 * eps2 * r);"),
    "vjp_spline_outer_power": ("dfr = -3.0 * f / r2;", "dfr = -2.0 * f / r2;"),
    "vjp_spline_sign": ("gx += f * u[0] + dfr * D[0] * Du;", "gx += f * u[0] - dfr * D[0] * Du;"),
    # far field (farfield.c)
    "far_multipole_sign": ("coef[m] = (((a + b + c) & 1) ? -1.0 : 1.0) /", "coef[m] = 1.0 /"),
    "far_offset_direction": ("const int64_t e = ((int64_t)((cx - x2 + cpd) % cpd) * cpd",
                             "const int64_t e = ((int64_t)((x2 - cx + cpd) % cpd) * cpd"),
    "far_taylor_factorial": ("const double yj = pow(y[0], ja) * pow(y[1], jb) * pow(y[2], jc) /\n                                  (factorial(ja) * factorial(jb) * factorial(jc));",
                             "const double yj = pow(y[0], ja) * pow(y[1], jb) * pow(y[2], jc) /\n                                  (factorial(ja) * factorial(jb));"),
    "far_recip_phase": ("case 1: re = -sn; break;", "case 1: re = sn; break;"),
    "far_no_background": ("out[0] -= M_PI / (alpha * alpha * V);", "out[0] -= 0.0;"),
    "far_near_image_kept": ("            g_minus_erf(r, alpha, Q, g);\n        } else {",
                            "            g_minus_erf(r, alpha, Q, g);\n            for (int jj = 0; jj <= Q; ++jj) g[jj] *= 0.5;\n        } else {"),
    "far_near_block_lopsided": ("fabs(s[1]) <= R && fabs(s[2]) <= R;", "fabs(s[1]) <= R && s[2] >= -R && s[2] < R;"),
}


def _build(name, tmp):
    old, new = MUTANTS[name]
    files = []
    hits = 0
    for path in (SRC, FAR):
        src = open(path).read()
        if old in src:
            src = src.replace(old, new, 1)
            hits += 1
        c = tmp / f"{name}_{os.path.basename(path)}"
        c.write_text(src)
        files.append(str(c))
    assert hits == 1, name
    so = tmp / f"{name}.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                    *files, "-o", str(so), "-lm"], check=True)
    return str(so)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    so = _build(name, tmp_path)
    saved_lib, saved_path = oracle._lib, oracle._LIB
    try:
        oracle._lib = None
        oracle._LIB = so
        # keep oracle.build() from recompiling over the mutant
        orig_build = oracle.build
        oracle.build = lambda force=False: so
        failed = _run_pins(first_only=True)
    finally:
        oracle.build = orig_build
        oracle._lib = saved_lib
        oracle._LIB = saved_path
    assert failed, f"mutant {name} passed every pin"


def _run_pins(first_only=False):
    """The pins of test_oracle_pins.py (and of the spline and far-field pin
    files), evaluated without pytest; returns the list of pins that the
    current oracle library fails (only the first with ``first_only``)."""
    import test_oracle_pins as P
    import test_oracle_spline_kde as S
    import test_oracle_farfield as F
    failed = []
    checks = [
        ("binning", lambda: P.test_binning_exact_containment_and_stability(oracle, 9, 1.0)),
        ("brute", lambda: P.test_accel_matches_brute_force_images(oracle, 7, 2, 300, True)),
        ("two_body", lambda: P.test_two_body_closed_form_across_face(oracle, 0.5)),
        ("golden", lambda: P.test_golden_two_body_values(oracle)),
        ("open", lambda: P.test_open_boundary_reduction(oracle)),
        ("lattice", lambda: P.test_lattice_symmetry_zero(oracle)),
        ("newton", lambda: P.test_newton_third_law(oracle)),
        ("vjp_fd", lambda: P.test_vjp_two_body_finite_difference(oracle)),
        ("vjp_spline_fd", lambda: S.test_spline_vjp_central_differences(oracle)),
        ("far_lattice_constant", lambda: F.test_tensor_origin_value_is_the_cubic_lattice_constant(5)),
        ("far_parity", F.test_tensor_has_the_parity_of_its_order),
        ("far_lattice", F.test_far_field_of_a_perfect_lattice_vanishes),
        ("far_vs_ewald", F.test_far_plus_near_equals_ewald_and_converges_with_order),
        ("far_cell_shift", F.test_far_field_follows_a_whole_cell_shift),
    ]
    for nm, fn in checks:
        try:
            fn()
        except Exception:
            failed.append(nm)
            if first_only:
                break
    return failed


def test_real_oracle_passes_the_same_pins():
    assert _run_pins() == []
