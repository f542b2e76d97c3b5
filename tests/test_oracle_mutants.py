"""The oracle's pins catch plausible mistakes (CPU).

Each entry plants one mistake in a copy of ``oracle/fsp_oracle.cpp``: a flipped sign, a
transposed operand or index, a dropped term, or a mistyped digit in a printed coefficient.
The copy is built with the oracle's own flags. Then the pins named beside the mistake run
against it, through ``FSP_ORACLE_LIB``, and at least one of them must fail. The unmodified
oracle passes the same pins in the rest of the suite.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fsp_oracle.cpp")

ADV = "test_oracle_advection.py::"
EUL = "test_oracle_euler.py::"
MBK = "test_oracle_multiblock.py::"
W7 = "test_oracle_weno7.py::"
TAN = "test_oracle_tangent.py::"
FLO = "test_oracle_flops.py::"
VJP = "test_oracle_vjp.py::"
OPT = "test_oracle_options.py::"
D3 = "test_oracle_3d.py::"
W74 = "test_oracle_weno7_4mp.py::"

# (name, text in the oracle, planted replacement, pins that catch it: tests/ node ids)
MUTANTS = [
    # printed coefficients (Section 3, Appendix)
    ("h5_1mp_sign", "-29.0L / 480", "29.0L / 480", [ADV + "test_table3[2]", ADV + "test_table3_orders[2-5]"]),
    ("h3_2mp_midpoint", "{1.0L - 1.0L / 6, -1.0L / 6}", "{1.0L + 1.0L / 6, -1.0L / 6}",
     [ADV + "test_table3[1]", ADV + "test_table3_orders[1-3]"]),
    ("central5_sign", "-13.0L / 320", "13.0L / 320",
     [EUL + "test_metrics_exact_on_affine_grid[True-2]", EUL + "test_metrics_exact_on_polynomial_grid[2]"]),
    ("central3_2mp_mid", "{11.0L / 12, -1.0L / 12}", "{11.0L / 12, 1.0L / 12}",
     [EUL + "test_metrics_exact_on_affine_grid[True-1]", EUL + "test_metrics_exact_on_polynomial_grid[1]"]),
    ("h7_digit", "-7481.0L / 107520", "-7418.0L / 107520",
     [EUL + "test_free_stream_preservation_randomized_grid[0-4]", EUL + "test_design_order_on_curved_grid[4-7-ns4]"]),
    ("is4_digit", "{3169, -6518, 2989}", "{3169, -6518, 2998}", [W7 + "test_r4_indicators_follow_the_definition"]),
    # midpoint interpolation and metrics (Sections 2.3-2.4)
    ("interp6_index", "cst<T>(3) * phi(-2) - cst<T>(25) * phi(-1)", "cst<T>(3) * phi(-1) - cst<T>(25) * phi(-2)",
     [EUL + "test_metrics_exact_on_polynomial_grid[2]", EUL + "test_mirror_symmetry[2]"]),
    ("interp4_digit", "cst<T>(9) * phi(1) - phi(2)) / cst<T>(16)", "cst<T>(9) * phi(1) - phi(2)) / cst<T>(15)",
     [EUL + "test_metrics_exact_on_affine_grid[True-0]", EUL + "test_metrics_exact_on_polynomial_grid[0]"]),
    ("metric_eta_x_sign", "M[2 * plane + o] = -y_xi;", "M[2 * plane + o] = y_xi;",
     [EUL + "test_metrics_exact_on_polynomial_grid[0]", EUL + "test_free_stream_preservation_randomized_grid[0-0]"]),
    ("metric_dir_swap", "y_xi = central_D(P, C, 0, 1, i, j);", "y_xi = central_D(P, C, 1, 1, i, j);",
     [EUL + "test_metrics_exact_on_affine_grid[True-0]", EUL + "test_metrics_exact_on_polynomial_grid[0]"]),
    ("metric_sign", "M[1 * plane + o] = -x_eta;", "M[1 * plane + o] = x_eta;",
     [EUL + "test_metrics_exact_on_affine_grid[True-0]", EUL + "test_metrics_exact_on_polynomial_grid[0]"]),
    ("jacobian_sign", "M[4 * plane + o] = x_xi * y_eta - x_eta * y_xi;",
     "M[4 * plane + o] = x_xi * y_eta + x_eta * y_xi;",
     [EUL + "test_metrics_exact_on_polynomial_grid[0]", MBK + "test_small_cylinder_blocks_are_valid"]),
    # Euler flux, spectral radius, eigenvectors (Sections 2.1, 2.3, 3.4)
    ("flux_metric_swap", "f[1] = rho * u * U + mx * p;", "f[1] = rho * u * U + my * p;",
     [EUL + "test_mirror_symmetry[0]", EUL + "test_transpose_symmetry[0]"]),
    ("flux_y_pressure", "f[2] = rho * v * U + my * p;", "f[2] = rho * v * U + mx * p;",
     [EUL + "test_mirror_symmetry[0]", EUL + "test_rotation_equivariance[0]"]),
    ("flux_energy_drop", "f[3] = (q[3] + p) * U;", "f[3] = q[3] * U;",
     [EUL + "test_linear_weights_reduce_to_linear_upwind_operator[0]", EUL + "test_sod_against_exact_solution[0]"]),
    ("spectral_norm_drop", "return fabs(mx * u + my * v) + c * sqrt(mx * mx + my * my);",
     "return fabs(mx * u + my * v) + c;",
     [EUL + "test_linear_weights_reduce_to_linear_upwind_operator[0]", EUL + "test_line_lambda_closed_form"]),
    ("eig_right_index", "R[2][0] = v - c * ny;", "R[2][0] = v - c * nx;",
     [EUL + "test_free_stream_preservation_randomized_grid[0-0]", EUL + "test_table4_free_stream_on_paper_grid[0]"]),
    ("eig_left_sign", "L[1][3] = -b1;", "L[1][3] = b1;",
     [EUL + "test_free_stream_preservation_randomized_grid[0-0]", EUL + "test_table4_free_stream_on_paper_grid[2]"]),
    # WENO interpolation (Eqs. 3.10-3.15, 3.22-3.23, Table 1)
    ("is1_sign", "T d2 = db - da, d1 = da + db;", "T d2 = db - da, d1 = da - db;",
     [ADV + "test_table3[0]", ADV + "test_table3_orders[0-3]"]),
    ("is0_sign", "T d2 = db - da, d1 = cst<T>(3) * db - da;", "T d2 = db - da, d1 = cst<T>(3) * db + da;",
     [ADV + "test_table3[0]", ADV + "test_table3_orders[0-3]"]),
    ("candidate_index", "cst<T>(b3[k][l]) * uj[k + l - 2]", "cst<T>(b3[k][l]) * uj[k + l - 1]",
     [ADV + "test_table3[2]", ADV + "test_table3_orders[2-5]"]),
    ("linear_weights_swap", "{1.0L / 16, 10.0L / 16, 5.0L / 16}", "{1.0L / 16, 5.0L / 16, 10.0L / 16}",
     [ADV + "test_table3[2]", ADV + "test_table3_orders[2-5]"]),
    ("b2_digit", "{{-0.5L, 1.5L}, {0.5L, 0.5L}}", "{{-0.5L, 1.5L}, {0.5L, 1.5L}}",
     [ADV + "test_table3[0]", ADV + "test_table3_orders[0-3]"]),
    ("c2_swap", "static const long double c2[2] = {0.25L, 0.75L};", "static const long double c2[2] = {0.75L, 0.25L};",
     [ADV + "test_table3[0]", EUL + "test_linear_weights_reduce_to_linear_upwind_operator[0]"]),
    ("ppm_renorm_drop", "for (int k = 0; k < r; ++k) w[k] = g[k] / sg;", "for (int k = 0; k < r; ++k) w[k] = g[k];",
     [ADV + "test_table3[2]", EUL + "test_table4_free_stream_on_paper_grid[2]"]),
    ("alpha_cube", "a[k] = Ck[k] / (d * d); s = s + a[k];", "a[k] = Ck[k] / (d * d * d); s = s + a[k];",
     [ADV + "test_table3[0]"]),
    ("cand2_index", "cst<T>(b2[k][l]) * uj[k + l - 1]", "cst<T>(b2[k][l]) * uj[k + l]",
     [ADV + "test_table3[0]", ADV + "test_table3_orders[0-3]"]),
    ("alpha_square_drop", "a[k] = Ck[k] / (d * d);", "a[k] = Ck[k] / d;", [ADV + "test_table3[0]"]),
    ("ppm3_sign", "return C * (cst<T>(1) + s * s * s);", "return C * (cst<T>(1) - s * s * s);",
     [ADV + "test_table3[2]", EUL + "test_rk3_third_order_in_time"]),
    ("ppm2_sign", "T d = w - C; return C - d * d / (C - cst<T>(1));", "T d = w - C; return C + d * d / (C - cst<T>(1));",
     [ADV + "test_table3[0]", EUL + "test_table4_free_stream_on_paper_grid[0]"]),
    # splitting and the right-hand side (Sections 2.3, 3, 3.4)
    ("lf_alpha_drop", "return F.P.alpha * best;", "return best;",
     [EUL + "test_linear_weights_reduce_to_linear_upwind_operator[0]", EUL + "test_line_lambda_closed_form"]),
    ("split_sign", "fm[4 * (s + 4) + v] = cst<T>(0.5L) * (f[v] - A * qs[v]);",
     "fm[4 * (s + 4) + v] = cst<T>(0.5L) * (f[v] + A * qs[v]);",
     [EUL + "test_mirror_symmetry[0]", EUL + "test_linear_weights_reduce_to_linear_upwind_operator[0]"]),
    ("minus_side_eigen", "const int ce = side == 0 ? c0 : c0 + 1;", "const int ce = side == 0 ? c0 : c0;",
     [EUL + "test_mirror_symmetry[0]"]),
    ("h2mp_plus_index", "hp = hp + cst<T>(S.hmid[-m]) * fpm[4 * (p + m + 2) + v];",
     "hp = hp + cst<T>(S.hmid[-m]) * fpm[4 * (p - m + 2) + v];",
     [EUL + "test_free_stream_preservation_randomized_grid[0-1]", EUL + "test_mirror_symmetry[1]"]),
    ("h2mp_minus_index", "hm = hm + cst<T>(S.hmid[-m]) * fmm[4 * (p - m + 2) + v];",
     "hm = hm + cst<T>(S.hmid[-m]) * fmm[4 * (p + m + 2) + v];",
     [EUL + "test_free_stream_preservation_randomized_grid[0-1]", EUL + "test_mirror_symmetry[1]"]),
    ("line_max_min", "if (s == 0 || sp > best) best = sp;", "if (s == 0 || sp < best) best = sp;",
     [EUL + "test_linear_weights_reduce_to_linear_upwind_operator[0]"]),
    ("direction_swap", "  nx = mbx / mb;\n  ny = mby / mb;", "  nx = mby / mb;\n  ny = mbx / mb;",
     [EUL + "test_rotation_equivariance[2]"]),
    ("mirror_stencil", "const int node = side == 0 ? c0 + m : c0 + 1 - m;",
     "const int node = side == 0 ? c0 + m : c0 + 1 + m;",
     [EUL + "test_mirror_symmetry[0]", EUL + "test_linear_weights_reduce_to_linear_upwind_operator[0]"]),
    ("h_minus_index", "fm[4 * (p + 1 - k + 4) + v]", "fm[4 * (p + k + 4) + v]",
     [EUL + "test_free_stream_preservation_randomized_grid[0-0]", EUL + "test_table4_free_stream_on_paper_grid[0]"]),
    ("difference_index", "R[o] = R[o] + (Hh[4 * (s + 2) + v] - Hh[4 * (s + 1) + v]);",
     "R[o] = R[o] + (Hh[4 * (s + 2) + v] - Hh[4 * (s + 0) + v]);",
     [EUL + "test_free_stream_preservation_randomized_grid[0-0]", EUL + "test_conservation_periodic"]),
    ("jacobian_multiply", "dQ[o] = -R[o] / Jinv;", "dQ[o] = -R[o] * Jinv;",
     [EUL + "test_conservation_periodic", EUL + "test_linear_weights_reduce_to_linear_upwind_operator[0]"]),
    ("midpoint_metric_shift", "return mxs[c0 + l]; });", "return mxs[c0 + l + 1]; });",
     [EUL + "test_free_stream_preservation_randomized_grid[0-0]", EUL + "test_table4_free_stream_on_paper_grid[0]"]),
    # seventh-order pieces (Appendix)
    ("ppm4_sign", "return C - d * d * d * d / (e * e * e);", "return C + d * d * d * d / (e * e * e);",
     [W7 + "test_fourth_order_mapping[0.015625]", EUL + "test_rotation_equivariance[4]"]),
    ("c4_digit", "{1.0L / 64, 21.0L / 64, 35.0L / 64, 7.0L / 64}", "{1.0L / 64, 21.0L / 64, 35.0L / 64, 8.0L / 64}",
     [W7 + "test_table_a1_candidates_and_linear_weights", W7 + "test_seventh_order_advection"]),
    ("b4_sign", "{-1.0L / 16, 9.0L / 16, 9.0L / 16, -1.0L / 16}", "{-1.0L / 16, 9.0L / 16, 9.0L / 16, 1.0L / 16}",
     [W7 + "test_table_a1_candidates_and_linear_weights", W7 + "test_weno7_constant_and_step"]),
    ("interp8_digit", "cst<T>(49) * phi(-2) - cst<T>(245) * phi(-1)", "cst<T>(49) * phi(-2) - cst<T>(254) * phi(-1)",
     [EUL + "test_metrics_exact_on_affine_grid[True-4]", EUL + "test_metrics_exact_on_polynomial_grid[4]"]),
    ("cand4_index", "tab4.b[k][l] * uj[k + l - 3]", "tab4.b[k][l] * uj[k + l - 2]",
     [EUL + "test_free_stream_preservation_randomized_grid[0-4]", EUL + "test_mirror_symmetry[4]"]),
    ("is4_scale", "cst<T>(IS4[q][a][b] / 2880.0L)", "cst<T>(IS4[q][a][b] / 2800.0L)",
     [W7 + "test_r4_indicators_follow_the_definition"]),
    ("is4_symmetric_digit", "{-31718, 45076, -16958}", "{-31718, 45067, -16958}",
     [W7 + "test_r4_indicators_follow_the_definition"]),
    # boundary rules, ghost coordinates and linked faces (readings)
    ("slipwall_mirror", "int sm = 2 * b - s;", "int sm = 2 * b - s - 1;",
     [EUL + "test_slip_wall_is_a_symmetry_plane[2]"]),
    ("slipwall_sign", "out[2] = out[2] - cst<T>(2) * un * ny;", "out[2] = out[2] + cst<T>(2) * un * ny;",
     [EUL + "test_slip_wall_is_a_symmetry_plane[2]"]),
    ("farfield_inflow", "if (vn < T(0))", "if (vn > T(0))",
     [EUL + "test_far_field_is_dirichlet_on_inflow_and_transmissive_on_outflow[2]"]),
    ("transmissive_node", "case BC_TRANSMISSIVE: rd(b, out); return;",
     "case BC_TRANSMISSIVE: rd(s < 0 ? 1 : n - 2, out); return;",
     [EUL + "test_transmissive_face_is_a_constant_continuation[2]"]),
    ("ghost_reflect", "at(ib, j, X0, Y0); at(2 * ib - i, j, X1, Y1);", "at(ib, j, X0, Y0); at(2 * ib - i + 1, j, X1, Y1);",
     [EUL + "test_metrics_exact_on_affine_grid[False-0]"]),
    ("period_sign", "X = X + T(double(q)) * per[0][0];", "X = X - T(double(q)) * per[0][0];",
     [EUL + "test_metrics_exact_on_affine_grid[True-0]", EUL + "test_transpose_symmetry[0]"]),
    ("link_reverse", "if (L.rev) t = nt - 1 - t;", "if (!L.rev) t = nt - 1 - t;",
     [MBK + "test_reversed_link_metrics_on_randomised_grid", MBK + "test_reversed_link_rhs"]),
    ("link_depth", "else if (L.face == 1) depth = nni - 1 - k;", "else if (L.face == 1) depth = nni - 2 - k;",
     [MBK + "test_cut_grid_reproduces_rhs[0]", MBK + "test_reversed_link_rhs"]),
    ("dirichlet_face", "case BC_DIRICHLET: for (int v = 0; v < 4; ++v) out[v] = P.bcq[face][v]; return;",
     "case BC_DIRICHLET: for (int v = 0; v < 4; ++v) out[v] = P.bcq[0][v]; return;",
     [EUL + "test_dirichlet_face_holds_its_own_state[2]"]),
    ("link_offset_sign", "X = X + T(L.off[0]); Y = Y + T(L.off[1]);", "X = X - T(L.off[0]); Y = Y + T(L.off[1]);",
     [MBK + "test_cut_periodic_grid_reproduces_metrics[0]", MBK + "test_cut_grid_reproduces_rhs[0]"]),
    # forward tangents (the dual numbers behind the adjoint checks)
    ("dual_product", "a.d * b.v + a.v * b.d", "a.d * b.v + a.d * b.d",
     [TAN + "test_rhs_tangent_matches_finite_differences[0]", TAN + "test_metrics_tangent_matches_finite_differences[0]"]),
    ("dual_quotient", "(a.d - q * b.d) / b.v", "(a.d + q * b.d) / b.v",
     [TAN + "test_rhs_tangent_matches_finite_differences[0]", TAN + "test_rk3_tangent_matches_finite_differences"]),
    ("dual_sqrt", "a.d / (2.0 * s)", "a.d / s",
     [TAN + "test_rhs_tangent_matches_finite_differences[0]", TAN + "test_rk3_tangent_matches_finite_differences"]),
    # options: free parameter, WENO-Z, midpoint splittings
    ("alpha5_digit", "n[2] = 5 * a / 32 - 13.0L / 60;", "n[2] = 5 * a / 32 - 13.0L / 50;",
     [OPT + "test_alpha_accuracy_relations[0.7]", OPT + "test_alpha_one_is_the_printed_scheme[2]"]),
    ("alpha_csd_index", "(nk(d) - nk(d + 1) + nk(1 - d) - nk(-d)) / 2", "(nk(d) - nk(d + 1) + nk(-d) - nk(1 - d)) / 2",
     [OPT + "test_alpha_one_is_the_printed_scheme[0]", OPT + "test_alpha_central_operator_is_exact_and_preserves_free_stream[0]"]),
    ("wenoz_tau", "fabs(IS[0] - IS[r - 1])", "fabs(IS[0] - IS[1])",
     [OPT + "test_weno_z_weights_approach_the_linear_ones[3-9]", OPT + "test_weno_z_design_order[2-5]"]),
    ("sw_acoustic", "l[2] * (u + c * nx));", "l[2] * (u - c * nx));",
     [OPT + "test_midpoint_splittings_are_consistent[1]", OPT + "test_midpoint_splittings_sod[1]"]),
    ("vl_energy", "(gamma * gamma - cst<T>(1))", "(gamma * gamma + cst<T>(1))",
     [OPT + "test_midpoint_splittings_are_consistent[2]", OPT + "test_midpoint_splittings_upwind_limits"]),
    # the four-midpoint seventh-order scheme (Appendix, scheme (3))
    ("s74_node_digit", "-108.0L / 420", "-106.0L / 420",
     [W74 + "test_h_reproduces_the_flux_through_degree_six", W74 + "test_printed_central_operator_is_the_central_part_of_h"]),
    ("s74_mirror_index", "cst<T>(S.hmidx[0]) * fmm[4 * (p + 2 + 2) + v]", "cst<T>(S.hmidx[0]) * fmm[4 * (p - 2 + 2) + v]",
     [W74 + "test_design_order_on_a_curved_grid"]),
    ("s74_central_b52", "if (S.cmid3 != 0.0L) d = d + cst<T>(S.cmid3) * (mid(2) - mid(-3));",
     "if (S.cmid3 != 0.0L) d = d + cst<T>(S.cmid3) * (mid(2) - mid(-2));",
     [W74 + "test_free_stream_and_conservation"]),
    # three dimensions (Sections 2.1-2.2)
    ("d3_metric_sign", "(dprod(b, a, p, q) - dprod(a, b, p, q) + dprod(a, b, q, p) - dprod(b, a, q, p))",
     "(dprod(b, a, p, q) + dprod(a, b, p, q) + dprod(a, b, q, p) - dprod(b, a, q, p))",
     [D3 + "test_metrics_exact_on_affine_grids[bc0]", D3 + "test_free_stream_on_randomised_cube[2]"]),
    ("d3_jacobian_third", "M[9 * plane + E4.at(i, j, k)] = Jv / cst<T>(3);", "M[9 * plane + E4.at(i, j, k)] = Jv / cst<T>(2);",
     [D3 + "test_metrics_exact_on_affine_grids[bc0]"]),
    ("d3_ghost_reflection", "return cst<T>(2) * coord3(P, X, c, id[0], id[1], id[2]) - coord3(P, X, c, m[0], m[1], m[2]);",
     "return coord3(P, X, c, m[0], m[1], m[2]);", [D3 + "test_metrics_exact_on_affine_grids[bc1]"]),
    ("d3_tangent_axis", "if (fabs(n[i]) < fabs(n[a])) a = i;", "if (fabs(n[i]) > fabs(n[a])) a = i;",
     [D3 + "test_eigenvectors[n1]"]),
    ("d3_left_shear", "L[1][0] = T(1) - b2; L[2][0] = -U1; L[3][0] = -U2;", "L[1][0] = T(1) - b2; L[2][0] = U1; L[3][0] = -U2;",
     [D3 + "test_eigenvectors[n0]", D3 + "test_extruded_grid_reduces_to_two_dimensions[2]"]),
    ("d3_w_momentum_flux", "f[3] = rho * w * U + m[2] * p;", "f[3] = rho * w * U + m[1] * p;",
     [D3 + "test_rotation_with_linear_weights[0]", D3 + "test_design_order_stationary_vortex[2-4.0]"]),
    ("d3_mid_metric_component", "mm[c] = interp_mid<T>(P.scheme, P.interp, [&](int l) { return ms[3 * (c0 + l) + c]; });",
     "mm[c] = interp_mid<T>(P.scheme, P.interp, [&](int l) { return ms[3 * (c0 + l)]; });",
     [D3 + "test_free_stream_on_randomised_cube[2]"]),
    ("d3_spectral_w", "fabs(m[0] * u + m[1] * v + m[2] * w) + c", "fabs(m[0] * u + m[1] * v + m[1] * w) + c",
     [D3 + "test_rotation_with_linear_weights[0]"]),
    # reverse mode (the tape behind the oracle's adjoints)
    ("rev_sub_sign", "rev_rec(a.v - b.v, a.i, 1.0, b.i, -1.0, 1)", "rev_rec(a.v - b.v, a.i, 1.0, b.i, 1.0, 1)",
     [VJP + "test_rhs_vjp_is_the_transposed_tangent[False-0]", VJP + "test_rhs_vjp_matches_finite_differences"]),
    ("rev_product_swap", "rev_rec(a.v * b.v, a.i, b.v, b.i, a.v, 2)", "rev_rec(a.v * b.v, a.i, a.v, b.i, b.v, 2)",
     [VJP + "test_rhs_vjp_is_the_transposed_tangent[False-0]", VJP + "test_metrics_vjp_is_the_transposed_tangent[0]"]),
    ("rev_quotient_sign", "1.0 / b.v, b.i, -q / b.v", "1.0 / b.v, b.i, q / b.v",
     [VJP + "test_rhs_vjp_is_the_transposed_tangent[False-0]", VJP + "test_rk3_vjp_is_the_transposed_tangent"]),
    ("rev_sqrt_half", "s > 0 ? 0.5 / s : 0.0", "s > 0 ? 1.0 / s : 0.0",
     [VJP + "test_rhs_vjp_is_the_transposed_tangent[False-0]", VJP + "test_rhs_vjp_matches_finite_differences"]),
    ("rev_sweep_operand", "if (r.b >= 0) adj[r.b] += r.pb * g;", "if (r.b >= 0) adj[r.b] += r.pa * g;",
     [VJP + "test_rhs_vjp_is_the_transposed_tangent[False-0]", VJP + "test_metrics_vjp_is_the_transposed_tangent[0]"]),
    # the operation counter (the roofline's algorithmic flops)
    ("count_sqrt_drop", "inline Counted sqrt(Counted a) { ++g_flops; return", "inline Counted sqrt(Counted a) { return",
     [FLO + "test_closed_forms[2]"]),
    ("count_div_drop", "inline Counted operator/(Counted a, Counted b) { ++g_flops;",
     "inline Counted operator/(Counted a, Counted b) {", [FLO + "test_closed_forms[2]"]),
    # time stepping (Section 6)
    ("rk3_weights", "cst<T>(0.75L) * Q[k] + cst<T>(0.25L) * (Q1[k] + dt * R[k])",
     "cst<T>(0.25L) * Q[k] + cst<T>(0.75L) * (Q1[k] + dt * R[k])",
     [EUL + "test_rk3_third_order_in_time", EUL + "test_sod_against_exact_solution[0]"]),
    ("rk3_last_stage", "cst<T>(2.0L / 3) * (Q2[k] + dt * R[k]);", "cst<T>(2.0L / 3) * (Q2[k] + dt * R[k] * cst<T>(0.5L));",
     [EUL + "test_rk3_third_order_in_time", EUL + "test_sod_against_exact_solution[0]"]),
    ("cfl_one_direction", "spectral(q, F.met(2, i, j), F.met(3, i, j), P.gamma)) / F.met(4, i, j);",
     "T(0) * spectral(q, F.met(2, i, j), F.met(3, i, j), P.gamma)) / F.met(4, i, j);",
     [EUL + "test_line_lambda_closed_form"]),
    ("cfl_invert", "return cfl / best;", "return cfl * best;",
     [EUL + "test_line_lambda_closed_form", EUL + "test_sod_against_exact_solution[0]"]),
]


def _build(tmp, name, old, new, src):
    d = os.path.join(tmp, name)
    os.makedirs(d, exist_ok=True)
    cpp, so = os.path.join(d, "fsp_oracle.cpp"), os.path.join(d, "libfsp_oracle.so")
    with open(cpp, "w") as f:
        f.write(src.replace(old, new))
    r = subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", so, cpp],
                       capture_output=True, text=True)
    return so if r.returncode == 0 else None


def _pins_fail(so, pins):
    env = dict(os.environ, FSP_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider",
                        *[os.path.join("tests", t) for t in pins]],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode != 0, (r.stdout.strip().splitlines() or [""])[-1]


def test_every_planted_mistake_is_caught(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("g++ is needed to build the mutated oracles")
    with open(SRC) as f:
        src = f.read()
    for name, old, new, _ in MUTANTS:
        assert src.count(old) == 1, f"{name}: the planted text must occur once in the oracle"
    workers = min(8, os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(workers) as ex:
        libs = list(ex.map(lambda m: _build(str(tmp_path), m[0], m[1], m[2], src), MUTANTS))
    assert all(libs), [m[0] for m, so in zip(MUTANTS, libs) if so is None]
    with cf.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(lambda a: _pins_fail(a[0], a[1][3]), zip(libs, MUTANTS)))
    missed = [(m[0], last) for m, (caught, last) in zip(MUTANTS, results) if not caught]
    assert not missed, f"mistakes the pins did not catch: {missed}"
