"""The pins must catch plausible mistakes in the oracle.

Each case copies the oracle's C source, plants one mistake (a dropped term,
a wrong sign or index, a transposed operand, a changed order), compiles the
copy on the CPU and runs the pin tests against it: at least one pin must
fail.  The real oracle is never modified.
"""
import importlib.util
import os
import shutil

import pytest

import tests.test_oracle_ax as tax
import tests.test_oracle_dssum_cg as tdc
import tests.test_oracle_gll as tgl
import tests.test_oracle_pcg as tpc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = {
    "dxm1_for_dxtm1": ("acc = acc + D[l * n + i] * ur", "acc = acc + D[i * n + l] * ur"),
    "dropped_g3_wt": ("ur[p] = g[0 * n3 + p] * wr + g[1 * n3 + p] * ws + g[2 * n3 + p] * wt;",
                      "ur[p] = g[0 * n3 + p] * wr + g[1 * n3 + p] * ws;"),
    "swapped_gxyz_component": ("us[p] = g[1 * n3 + p] * wr + g[3 * n3 + p] * ws",
                               "us[p] = g[2 * n3 + p] * wr + g[3 * n3 + p] * ws"),
    "ws_wrong_index": ("ws = ws + D[j * n + l] * ue[i + n * (l + (long)n * k)];",
                       "ws = ws + D[j * n + l] * ue[l + n * (i + (long)n * k)];"),
    "metric_transposed": ("g = g + Jinv[b][m] * Jinv[c][m];", "g = g + Jinv[m][b] * Jinv[m][c];"),
    "weight_formula": ("w[i] = (double)(2.0L / ((long double)N * (N + 1) * p * p));",
                       "w[i] = (double)(2.0L / ((long double)N * (N + 2) * p * p));"),
    "dmat_corner_sign": ("v = -(long double)N * (N + 1) / 4.0L;", "v = (long double)N * (N + 1) / 4.0L;"),
    "dssum_reverse_order": ("for (long q = 0; q < E * n3; q++) acc[gid[q]] = acc[gid[q]] + w[q];",
                            "for (long q = E * n3 - 1; q >= 0; q--) acc[gid[q]] = acc[gid[q]] + w[q];"),
    "mask_misses_z_faces": ("gy == 0 || gy == NY - 1 ||\n                          gz == 0 || gz == NZ - 1;",
                            "gy == 0 || gy == NY - 1;"),
    "cg_beta_inverted": ("double beta = (it == 1) ? 0.0 : rho / rho_old;\n        for (long q = 0; q < npts; q++) p[q] = r[q] + beta * p[q];",
                         "double beta = (it == 1) ? 0.0 : rho_old / rho;\n        for (long q = 0; q < npts; q++) p[q] = r[q] + beta * p[q];"),
    "cg_residual_sign": ("r[q] = r[q] - alpha * w[q];\n        }\n        rho_old = rho;\n        rho = nbo_dot_c(Ex, Ey, Ez, n, r, r);",
                         "r[q] = r[q] + alpha * w[q];\n        }\n        rho_old = rho;\n        rho = nbo_dot_c(Ex, Ey, Ez, n, r, r);"),
    "diag_drops_cross_term": ("+ 2.0 * D[j * n + j] * D[k * n + k] * g[4 * n3 + p];",
                              ";"),
    "pcg_z_from_w": ("z[q] = minv[q] * r[q];\n        }", "z[q] = minv[q] * w[q];\n        }"),
    "gid_wrong_local_index": ("long gy = (long)ey * (n - 1) + j;\n            long gz = (long)ez * (n - 1) + k;\n            gid[",
                              "long gy = (long)ey * (n - 1) + i;\n            long gz = (long)ez * (n - 1) + k;\n            gid["),
}

PINS = [
    lambda o: tgl.test_gll_quadrature_exactness(o, 6),
    lambda o: tgl.test_gll_nodes_are_lobatto_points(o, 6),
    lambda o: tgl.test_dmat_differentiates_polynomials(o, 6),
    lambda o: tax.test_ax_constant_nullspace_and_symmetry(o, 5),
    lambda o: tax.test_ax_dense_element_matrix_bruteforce(o, 3),
    lambda o: tax.test_ax_exact_stiffness_affine(o, 4),
    lambda o: tax.test_isoparametric_identity_perturbed(o, 4),
    lambda o: tdc.test_numbering_multiplicity_mask(o, (3, 2, 1), 4),
    lambda o: tdc.test_dssum_canonical_order_bruteforce(o, (2, 2, 2), 3),
    lambda o: tdc.test_cg_matches_dense_solve(o, (2, 2, 2), 3),
    lambda o: tdc.test_cg_energy_error_decreases_and_fixed_iterations(o),
    lambda o: tpc.test_diag_matches_bruteforce_element_matrix(o, 3),
    lambda o: tpc.test_jacobi_pcg_dense_solve_and_iterations(o),
]


def load_mutant(tmp_path, old, new):
    src = open(os.path.join(ROOT, "oracle", "nekbone_oracle.c")).read()
    assert src.count(old) == 1, "mutation anchor must match exactly once"
    d = tmp_path / "oracle_mut"
    d.mkdir()
    (d / "nekbone_oracle.c").write_text(src.replace(old, new))
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), d / "__init__.py")
    spec = importlib.util.spec_from_file_location(f"oracle_mut_{id(d)}", d / "__init__.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    return mod


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(tmp_path, name):
    old, new = MUTATIONS[name]
    mut = load_mutant(tmp_path, old, new)
    caught = []
    for pin in PINS:
        try:
            pin(mut)
        except (AssertionError, ValueError, IndexError):
            caught.append(pin)
    assert caught, f"no pin caught mutation {name}"
