"""Planted mistakes: each is a plausible slip in the oracle's scheme or its sub-cycling
(a dropped term, a wrong sign or index, a wrong factor, a missing step), planted into a scratch copy of the oracle's C
source, which is compiled and loaded in place of the real one for the test; the pin
named beside it must then fail.  The real oracle passes every one of these pins."""
import os
import shutil

import numpy as np
import pytest

import test_oracle_hydro as H
import test_oracle_refine as RF
import test_oracle_mlp as M
import test_oracle_poisson as P
import test_oracle_riemann as R
import test_oracle_tree as TR
import test_oracle_subcycle as S
import test_oracle_truncation as T

# (file, exact text, replacement): the predictor and face states of hydro.c
PREDICTOR = {
    "density_divergence_dropped": (
        "hydro.c",
        "Wt[0] = r - h * (u * D[0][0] + r * D[0][1] + v * D[1][0] + r * D[1][2] + w * D[2][0] + r * D[2][3]);",
        "Wt[0] = r - h * (u * D[0][0] + v * D[1][0] + w * D[2][0]);"),
    "density_advection_dropped_x": ("hydro.c", "Wt[0] = r - h * (u * D[0][0] + ", "Wt[0] = r - h * ("),
    "velocity_advection_dropped_x": ("hydro.c", "Wt[1] = u - h * (u * D[0][1] + ", "Wt[1] = u - h * ("),
    "pressure_gradient_dropped_x": ("hydro.c", "+ w * D[2][1] + D[0][4] / r);", "+ w * D[2][1]);"),
    "pressure_divergence_dropped": ("hydro.c", " + gamma * p * (D[0][1] + D[1][2] + D[2][3]));", ");"),
    "predictor_full_step": ("hydro.c", "double h = 0.5 * lam;", "double h = lam;"),
    "face_states_swapped": ("hydro.c", "side ? Wt[v] + 0.5 * D[d][v] : Wt[v] - 0.5 * D[d][v];",
                            "side ? Wt[v] - 0.5 * D[d][v] : Wt[v] + 0.5 * D[d][v];"),
}
OTHER = {
    "interpolation_sign": (("hydro.c", "r = r + (pos[d] ? 0.25 * m : -0.25 * m);",
                            "r = r + (pos[d] ? -0.25 * m : 0.25 * m);"),
                           lambda O: H.test_ghost_interpolation_mean_and_linear(O)),
    "reflux_sign": (("hydro.c", "side ? u_new[(int64_t)v * ncell + C] - lam * corr",
                     "side ? u_new[(int64_t)v * ncell + C] + lam * corr"),
                    lambda O: H.test_conservation_periodic(O, True)),
    "restriction_factor": (("hydro.c", "u_new[(int64_t)v * ncell + o * 8 + c] = 0.125 * sum;",
                            "u_new[(int64_t)v * ncell + o * 8 + c] = 0.25 * sum;"),
                           lambda O: H.test_refined_cells_hold_the_mean_of_their_children(O)),
    "restriction_coarse_level_first": (("hydro.c",
                                        "for (int l = t->levelmax - 1; l >= 1; l--) or_reflux_restrict(t, p, l, reg, u_new, dt);",
                                        "for (int l = 1; l <= t->levelmax - 1; l++) or_reflux_restrict(t, p, l, reg, u_new, dt);"),
                                       lambda O: H.test_refined_cells_hold_the_mean_of_their_children(O)),
    "courant_over_refined_cells_too": (("hydro.c",
                                        "            if (t->son[cid] >= 0) continue;\n            double U[NV], W[NV];\n"
                                        "            load(u, ncell, cid, U);",
                                        "            double U[NV], W[NV];\n            load(u, ncell, cid, U);"),
                                       lambda O: H.test_courant_over_leaves_only(O)),
    # HLLC (riemann.c): each caught by the reflection symmetry that maps a branch onto its partner
    "hllc_left_speed_from_the_wrong_wave": (("riemann.c", "double SL = fmin(uL - cL, uR - cR);",
                                             "double SL = fmin(uL - cL, uR + cR);"),
                                            lambda O: R.test_hllc_mirror_symmetry(O)),
    "hllc_right_star_with_the_left_density": (("riemann.c", "double f = rR * (SR - uR) / (SR - Sstar);",
                                               "double f = rL * (SR - uR) / (SR - Sstar);"),
                                              lambda O: R.test_hllc_mirror_symmetry(O)),
    "hllc_right_star_with_the_left_speed": (("riemann.c",
                                             "for (int v = 0; v < 5; v++) F[v] = FR[v] + SR * (Us[v] - UR[v]);",
                                             "for (int v = 0; v < 5; v++) F[v] = FR[v] + SL * (Us[v] - UR[v]);"),
                                            lambda O: R.test_hllc_mirror_symmetry(O)),
    "hllc_contact_speed_sign": (("riemann.c", "double Sstar = (pR - pL + rL", "double Sstar = (pL - pR + rL"),
                                lambda O: R.test_hllc_close_to_exact_for_weak_waves(O)),
    # the uniform-box path (box.c), checked against the exact solution on its own
    "box_pressure_divergence_dropped": (("box.c", " + gamma * p * (D[0][1] + D[1][2] + D[2][3]));", ");"),
                                        lambda O: T.test_box_step_local_error_is_third_order(O)),
    # refinement (refine.c)
    "refinement_mass_with_dx_squared": (("refine.c", "flag[cell] = u[cell] * (dx * dx * dx) > mass_thr;",
                                         "flag[cell] = u[cell] * (dx * dx) > mass_thr;"),
                                        lambda O: RF.test_new_octs_match_set_construction(O, True, 1)),
    # octree and Hilbert key (tree.c)
    "hilbert_gray_code_order": (("tree.c", "    X[1] ^= X[0];\n    X[2] ^= X[1];", "    X[2] ^= X[1];\n    X[1] ^= X[0];"),
                                lambda O: TR.test_hilbert_bijection_and_adjacency(O, 3)),
    "octree_child_bits_swapped": (("tree.c", "return o * 8 + (X & 1) + 2 * (Y & 1) + 4 * (Z & 1);",
                                   "return o * 8 + (X & 1) + 4 * (Y & 1) + 2 * (Z & 1);"),
                                  lambda O: TR.test_tables_match_brute_force(O, 0)),
    # surrogate network and Adam (mlp.c)
    "silu_derivative": (("mlp.c", "gz[j] = g[j] * sg * (1.0 + z[L][j] * (1.0 - sg));",
                         "gz[j] = g[j] * sg * (1.0 + z[L][j] * sg);"),
                        lambda O: M.test_backward_matches_finite_differences(O)),
    "features_pressure_reference_min": (("mlp.c", "double pref = WL[4] > WR[4] ? WL[4] : WR[4];",
                                         "double pref = WL[4] < WR[4] ? WL[4] : WR[4];"),
                                        lambda O: M.test_features_worked_examples(O)),
    "features_mean_velocity_left_only": (("mlp.c", "double ubar = 0.5 * (WL[1] + WR[1]);", "double ubar = WL[1];"),
                                         lambda O: M.test_features_worked_examples(O)),
    "adam_without_bias_correction": (("mlp.c", "double mh = m[i] / c1, vh = v[i] / c2;", "double mh = m[i], vh = v[i];"),
                                     lambda O: M.test_adam_first_step(O)),
    # Poisson solvers (poisson.c)
    "preconditioner_centre_weight": (("poisson.c",
                                      "u[c] = (13.0 / 12.0) * r[c] + nb_sum(r, nx, ny, nz, i, j, k) / 6.0;",
                                      "u[c] = r[c] + nb_sum(r, nx, ny, nz, i, j, k) / 6.0;"),
                                     lambda O: P.test_preconditioner_is_incomplete_kkt(O)),
    "ppcg_step_length_recurrence": (("poisson.c", "alpha = gamma / (delta - beta * gamma / alpha_old);",
                                     "alpha = gamma / (delta - beta * gamma * alpha_old);"),
                                    lambda O: P.test_iterates_match_scipy_cg(O, 0)),
    # level sub-cycling (subcycle.c)
    "subcycle_no_time_interpolation": (("subcycle.c", "U[i] = 0.5 * (U[i] + N[i]);", "U[i] = U[i];"),
                                       lambda O: S.test_wave_through_refinement_bands(O)),
    "subcycle_ghosts_at_the_new_time": (("subcycle.c", "U[i] = 0.5 * (U[i] + N[i]);", "U[i] = N[i];"),
                                        lambda O: S.test_wave_through_refinement_bands(O)),
    "subcycle_fine_step_not_halved": (("subcycle.c",
                                       "x.dt[l] = l >= t->levelmin ? ldexp(dtb, -(l - t->levelmin)) : dtb;",
                                       "x.dt[l] = dtb;"),
                                      lambda O: S.test_wave_through_refinement_bands(O)),
    "subcycle_first_fine_step_not_corrected": (("subcycle.c",
                                                "        or_reflux_restrict(t, x->p, c, x->reg, x->U, x->dt[c + 1]);\n",
                                                ""),
                                               lambda O: S.test_wave_through_refinement_bands(O)),
    "subcycle_reflux_with_the_coarse_step": (("subcycle.c",
                                              "        advance(x, c + 1);\n"
                                              "        or_reflux_restrict(t, x->p, c, x->reg, x->N, x->dt[c + 1]);\n    }",
                                              "        advance(x, c + 1);\n"
                                              "        or_reflux_restrict(t, x->p, c, x->reg, x->N, x->dt[c]);\n    }"),
                                             lambda O: S.test_conservation(O)),
    "subcycle_courant_not_scaled_by_level": (("subcycle.c", "double r = ldexp(dx / sig, l - t->levelmin);",
                                              "double r = dx / sig;"),
                                             lambda O: S.test_time_step_closed_form(O)),
}


@pytest.fixture
def planted(oracle, tmp_path, monkeypatch):
    """Returns a function that plants one mistake and loads the mutated oracle."""
    def plant(fname, old, new):
        for s in oracle._SRC + ["oracle.h"]:
            shutil.copy(os.path.join(oracle._HERE, s), tmp_path)
        path = os.path.join(tmp_path, fname)
        src = open(path).read()
        assert src.count(old) == 1, "the planted text must match exactly once"
        open(path, "w").write(src.replace(old, new))
        monkeypatch.setattr(oracle, "_HERE", str(tmp_path))
        monkeypatch.setattr(oracle, "_LIB_PATH", os.path.join(tmp_path, "liboracle.so"))
        monkeypatch.setattr(oracle, "_lib", None)
        return oracle
    return plant


@pytest.mark.parametrize("name", sorted(PREDICTOR))
def test_predictor_mistakes_fail_the_exact_solution_pin(planted, name):
    O = planted(*PREDICTOR[name])
    e5, e6 = T.octree_errors(O, 5), T.octree_errors(O, 6)
    order = np.log2(e5 / e6)
    assert not np.all(order > 2.8), (name, order)


@pytest.mark.parametrize("name", sorted(OTHER))
def test_other_mistakes_fail_their_pin(planted, name):
    mutation, pin = OTHER[name]
    O = planted(*mutation)
    with pytest.raises(AssertionError):
        pin(O)
