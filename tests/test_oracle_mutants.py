"""Mistakes planted in the oracle, on the CPU: each entry below changes one
thing in a copy of oracle/teuk_oracle.c the way a slip in writing it could
(a dropped term, a wrong sign, index, constant or power, transposed or swapped
operands), compiles the copy, and runs the oracle's pins against it (through
TEUK_ORACLE_LIB). Every planted mistake must make at least one pin fail, and
the unaltered copy must pass the same pins, so that the pins tie every part of
the oracle to the paper and to the mathematics rather than to itself.
The pins each mistake is run against are listed beside it. LD_MUTANTS do the
same for the extended-precision oracle (oracle/teuk_oracle_ld.c, loaded
through TEUK_ORACLE_LD_LIB), including slips that would quietly drop its
extra precision."""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

import oracle as o

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "teuk_oracle.c")
SRC_LD = os.path.join(ROOT, "oracle", "teuk_oracle_ld.c")

P = "tests/test_oracle_pins.py::"
PH = "tests/test_oracle_physics.py::"
HY = "tests/test_oracle_hyperboloidal.py::"

SYM = PH + "test_coefficients_match_symbolic_derivation"
SYM_HYP = HY + "test_hyperboloidal_coefficients_match_teukolsky_equation"
SYM_PHI = HY + "test_rescaled_field_in_rstar_matches_teukolsky_equation"
EIGEN = PH + "test_theta_operator_on_spin_weighted_harmonics"
ASSEMBLY = PH + "test_assembly_matches_printed_real_matrices"

# (name, text in the oracle source, replacement, pins)
MUTANTS = [
    # tortoise coordinate, Sec. 2.2
    ("tortoise: sign of the r_- logarithm",
     "- (2.0 * M * rm / (rp - rm)) * log((x + rp - rm) / (2.0 * M));",
     "+ (2.0 * M * rm / (rp - rm)) * log((x + rp - rm) / (2.0 * M));",
     [P + "test_tortoise_derivative_and_inverse"]),
    ("tortoise: sign of the extremal pole term",
     "- 2.0 * M * M * exp(-y);", "+ 2.0 * M * M * exp(-y);",
     [P + "test_tortoise_derivative_and_inverse"]),
    ("tortoise: r - r_- written r - r_+ in the logarithm",
     "log((x + rp - rm) / (2.0 * M));", "log(x / (2.0 * M));",
     [P + "test_tortoise_derivative_and_inverse"]),
    ("Delta: r - r_- factor written r - r_+",
     "double Delta = x * (x + 2.0 * sqrt(fmax(M * M - a * a, 0.0)));",
     "double Delta = x * x;", [SYM]),
    # coefficients in r*, Eq. teuk0
    ("B*: (r - M) written (r + M)", "2.0 * s * (r - M) * varpi) / Sigma2",
     "2.0 * s * (r + M) * varpi) / Sigma2", [SYM]),
    ("Bt: sign of the i s a Delta cos term", "- 2.0 * I * s * a * Delta * cs) / Sigma2",
     "+ 2.0 * I * s * a * Delta * cs) / Sigma2", [SYM]),
    ("Bt: dropped M a m term", "(-4.0 * I * M * a * m * r\n",
     "(0.0 * I * M * a * m * r\n", [SYM]),
    ("C: sign of the pole potential", "Delta * (s - mc * mc / (sn * sn))",
     "Delta * (s + mc * mc / (sn * sn))", [SYM]),
    ("C: s cos(theta) in (m + s cos) dropped", "double mc = m + s * cs;\n    double complex C = (4.0",
     "double mc = m;\n    double complex C = (4.0", [SYM]),
    ("K: sign of b b_*", "Bstar - b * b_star - b * Bt", "Bstar + b * b_star - b * Bt", [SYM]),
    ("db/dr: sign of the Sigma2 derivative", "- varpi * dSigma2_dr / (2.0 * Sigma2 * Sigma)",
     "+ varpi * dSigma2_dr / (2.0 * Sigma2 * Sigma)", [SYM]),
    ("rescaled field: dropped B* g1 in C", "C = C + Axx * g2 + Bstar * g1;",
     "C = C + Axx * g2;", [SYM_PHI]),
    ("rescaled field: dropped g1^2", "double g2 = (Delta / varpi) * dg1_dr + g1 * g1;",
     "double g2 = (Delta / varpi) * dg1_dr;", [SYM_PHI]),
    # hyperboloidal coefficients, Sec. 2.2 / Eq. near_final
    ("hyperboloidal Bt: sign of (1 - H')", "I * (2.0 * m * a * (1.0 - Hp)",
     "I * (2.0 * m * a * (Hp - 1.0)", [SYM_HYP]),
    ("hyperboloidal C: dropped 2 a^2 x^2", "+ 2.0 * a * a * x * x\n                        - 2.0 * I",
     "\n                        - 2.0 * I", [SYM_HYP]),
    ("hyperboloidal K: b for c in the last term", "Br - b * Bt - c * db", "Br - b * Bt - b * db",
     [SYM_HYP]),
    ("hyperboloidal c: W for W^2", "double c = W * W * E / D;", "double c = W * E / D;",
     [HY + "test_speeds_vanish_on_the_horizon_and_at_scri", SYM_HYP]),
    ("hyperboloidal G: 8M^2/S for 4M^2/S", "8.0 * M * M / S - 2.0 * M * W\n                      + a",
     "4.0 * M * M / S - 2.0 * M * W\n                      + a", [SYM_HYP]),
    ("ghost extrapolation: cubic for quartic", "#define EXTRAP_DEG 4", "#define EXTRAP_DEG 3",
     [HY + "test_extrapolated_ghosts_keep_linear_weights_exact_to_degree_four"]),
    # rounding to the weight formats
    ("bfloat16: 9 significant bits", "round_to_format(x, 8, -126,", "round_to_format(x, 9, -126,",
     [P + "test_round_w_matches_numpy_and_torch"]),
    ("rounding: truncation for nearest", "double q = nearbyint(ldexp(x, p - 1 - E));",
     "double q = trunc(ldexp(x, p - 1 - E));", [P + "test_round_w_matches_numpy_and_torch"]),
    ("binary16: subnormal exponent", "round_to_format(x, 11, -14,", "round_to_format(x, 11, -15,",
     [P + "test_round_w_matches_numpy_and_torch"]),
    # WENO5 weights and fluxes, Sec. 3.1.2-3.1.3
    ("linear weights transposed", "D_LIN[3] = {0.1, 0.6, 0.3}", "D_LIN[3] = {0.3, 0.6, 0.1}",
     [P + "test_smooth_weights_approach_linear_weights_at_second_order",
      P + "test_fifth_order_convergence_on_periodic_advection"]),
    ("IS_0: 3 f_j written 2 f_j",
     "IS[0] = 13.0 / 12.0 * pow(f[0] - 2 * f[1] + f[2], 2)\n              + 0.25 * pow(f[0] - 4 * f[1] + 3 * f[2], 2);",
     "IS[0] = 13.0 / 12.0 * pow(f[0] - 2 * f[1] + f[2], 2)\n              + 0.25 * pow(f[0] - 4 * f[1] + 2 * f[2], 2);",
     [P + "test_smooth_weights_approach_linear_weights_at_second_order"]),
    ("alpha: (eps + IS) not squared", "alpha[k] = D_LIN[k] / pow(eps + IS[k], 2);",
     "alpha[k] = D_LIN[k] / pow(eps + IS[k], 1);",
     [P + "test_reduced_reading_in_binary64_equals_paper_formula"]),
    ("candidate q_1: wrong node", "q[1] = (-f[1] + 5.0 * f[2] + 2.0 * f[3]) / 6.0;",
     "q[1] = (-f[1] + 5.0 * f[2] + 2.0 * f[4]) / 6.0;",
     [P + "test_each_candidate_stencil_exact_to_degree_three"]),
    ("negative-direction q_0 mirrored wrongly", "q[0] = (11.0 * f[2] - 7.0 * f[3] + 2.0 * f[4]) / 6.0;",
     "q[0] = (11.0 * f[4] - 7.0 * f[3] + 2.0 * f[2]) / 6.0;",
     [P + "test_each_candidate_stencil_exact_to_degree_three"]),
    ("omega_1: sign of omega_2", "w[1] = 1.0 - w[0] - w[2];", "w[1] = 1.0 - w[0] + w[2];",
     [P + "test_reduced_weights_within_rounding_of_fp64_weights"]),
    ("reduced IS_1: f_{j-1} - f_{j+1} as a difference", "b = RW(xh[1] + xh[2]);",
     "b = RW(xh[1] - xh[2]);", [P + "test_reduced_weights_within_rounding_of_fp64_weights"]),
    ("reduced mirror: last two swapped", "x[2] = t1; x[3] = t0;", "x[2] = t0; x[3] = t1;",
     [P + "test_reduced_weights_within_rounding_of_fp64_weights"]),
    ("reduced eps: scaled by 2^-e", "double eh = ldexp(eps, -2 * e);",
     "double eh = ldexp(eps, -e);", [P + "test_reduced_reading_in_binary64_equals_paper_formula"]),
    ("flux difference divided by 2h", "D[i] = (fh[i + 1] - fh[i]) / h;",
     "D[i] = (fh[i + 1] - fh[i]) / (2.0 * h);", [P + "test_linear_scheme_exact_to_degree_five"]),
    ("negative direction on the positive stencil", "&ext[i - 2 + 3] : &ext[i - 1 + 3]",
     "&ext[i - 2 + 3] : &ext[i - 2 + 3]", [P + "test_linear_scheme_exact_to_degree_five"]),
    ("r* ghosts zero instead of edge copies", "else ext[k + 3] = f[k < 0 ? 0 : n - 1];",
     "else ext[k + 3] = 0.0;", [PH + "test_constant_scalar_state_is_stationary"]),
    # FD6 + KO8, Sec. 3.1.1
    ("FD6: sign of u_{j-3}", "+ 9.0 * u[-2] - u[-3])", "+ 9.0 * u[-2] + u[-3])",
     [P + "test_fd6_exact_to_degree_six_and_sixth_order"]),
    ("KO8: h^8 for h^7", "Q[j] = sigma * pow(h, 7) * b[j + G] / 256.0;",
     "Q[j] = sigma * pow(h, 8) * b[j + G] / 256.0;",
     [P + "test_ko8_annihilates_degree_seven_and_has_its_fourier_symbol"]),
    ("KO8 added instead of subtracted", "F[2 * plane + p] = creal(Fpi) - Qc[2 * nr + i];",
     "F[2 * plane + p] = creal(Fpi) + Qc[2 * nr + i];",
     [PH + "test_kreiss_oliger_term_damps_in_the_right_hand_side"]),
    # right-hand side assembly, Eq. evln and Sec. 3.1.2
    ("pole parity inverted", "double sigma = ((g->m + g->s) % 2 == 0) ? 1.0 : -1.0;\n\n#pragma",
     "double sigma = ((g->m + g->s) % 2 == 0) ? -1.0 : 1.0;\n\n#pragma", [EIGEN]),
    ("theta second difference: -20 for -30", "- 30.0 * nb[2]", "- 20.0 * nb[2]", [EIGEN]),
    ("theta first difference: sign", "(nb[0] - 8.0 * nb[1] + 8.0 * nb[3] - nb[4])",
     "(-nb[0] + 8.0 * nb[1] - 8.0 * nb[3] + nb[4])", [EIGEN]),
    ("pole ghost mirrored on the node", "if (jj < 0) { jj = -1 - jj; sg = sigma; }\n            if (jj >= nth) { jj = 2 * nth - 1 - jj; sg = sigma; }\n            rows",
     "if (jj < 0) { jj = -jj; sg = sigma; }\n            if (jj >= nth) { jj = 2 * nth - 1 - jj; sg = sigma; }\n            rows",
     [EIGEN]),
    ("Psi rows: sign of b D", "double complex Fpsi = pi - b * Dpsi;",
     "double complex Fpsi = pi + b * Dpsi;", [ASSEMBLY]),
    ("pi rows: b for c", "double complex Fpi = cpi * Dpi", "double complex Fpi = b * Dpi", [ASSEMBLY]),
    ("pi rows: upwinded like Psi", "int dir = (c < 2) ? +1 : -1;", "int dir = +1;",
     [PH + "test_price_tail_exponent_schwarzschild_l0"]),
    ("pi rows: Bt acting on Psi", "+ Bth * psi_th + Bt * pi + C * psi;",
     "+ Bth * psi_th + Bt * psi + C * psi;", [ASSEMBLY]),
    ("pi rows: dropped C Psi", "+ Bth * psi_th + Bt * pi + C * psi;",
     "+ Bth * psi_th + Bt * pi;", [ASSEMBLY]),
    # time integrators, Sec. 3.2
    ("SSP-RK(3,3): stage-2 weights swapped", "u2[k] = 0.75 * u[k] + 0.25 * (u1[k] + dt * Fv[k]);",
     "u2[k] = 0.25 * u[k] + 0.75 * (u1[k] + dt * Fv[k]);",
     [P + "test_ssprk33_stability_polynomial"]),
    ("SSP-RK(3,3): last stage from u1", "u[k] = u[k] / 3.0 + 2.0 / 3.0 * (u2[k] + dt * Fv[k]);",
     "u[k] = u[k] / 3.0 + 2.0 / 3.0 * (u1[k] + dt * Fv[k]);",
     [P + "test_ssprk33_stability_polynomial"]),
    ("SSP-RK(10,4): dt/6 for dt/15 in u5", "2.0 / 5.0 * u4[k] + dt / 15.0 * F4[k];",
     "2.0 / 5.0 * u4[k] + dt / 6.0 * F4[k];", [P + "test_ssprk104_fourth_order_convergence"]),
    ("SSP-RK(10,4): dt/6 for dt/10 at the end", "+ 3.0 / 50.0 * dt * F4[k] + dt / 10.0 * Fv[k];",
     "+ 3.0 / 50.0 * dt * F4[k] + dt / 6.0 * Fv[k];", [P + "test_ssprk104_fourth_order_convergence"]),
    ("r(r*): bisection sides swapped", "if (rstar_of_lnx(mid, M, a) < rs) lo = mid; else hi = mid;",
     "if (rstar_of_lnx(mid, M, a) < rs) hi = mid; else lo = mid;",
     [P + "test_tortoise_derivative_and_inverse"]),
    ("rescaled field: 2 A** g1 written A** g1", "Bstar = Bstar + 2.0 * Axx * g1;",
     "Bstar = Bstar + Axx * g1;", [SYM_PHI]),
    ("rescaled field: dropped a^2/r in N", "double N = 2.0 * s * (r - M) + Delta / r;",
     "double N = 2.0 * s * (r - M) + (Delta - a * a) / r;", [SYM_PHI]),
    ("hyperboloidal b in the complex step: rho for rho^2",
     "return rho * rho * delta / E;", "return rho * delta / E;", [SYM_HYP]),
    ("hyperboloidal sigma: sign under the root",
     "double sig = sqrt(w * w - a * a * x * x * delta * sn2);",
     "double sig = sqrt(w * w + a * a * x * x * delta * sn2);", [SYM_HYP]),
    ("hyperboloidal D: sign of a^2 sin^2", "double D = Hp * G - a * a * sn2;",
     "double D = Hp * G + a * a * sn2;", [SYM_HYP]),
    ("hyperboloidal B^r: (1 + s) written (1 - s)", "2.0 * W * W * (M * (1 + s) - a * a * x)",
     "2.0 * W * W * (M * (1 - s) - a * a * x)", [SYM_HYP]),
    ("rho(r): S/r for r/S", "return r / (1.0 + r / S);", "return r / (1.0 + S / r);",
     [HY + "test_speeds_vanish_on_the_horizon_and_at_scri"]),
    ("theta nodes on a node-centred grid", "double th = (j + 0.5) * M_PI / nth;\n            double c[10];",
     "double th = (j + 1.0) * M_PI / (nth + 1);\n            double c[10];", [EIGEN]),
    ("theta spacing pi/(nth - 1)", "double dth = M_PI / nth;\n    double sigma",
     "double dth = M_PI / (nth - 1);\n    double sigma", [EIGEN]),
    ("radial spacing over nr", "double h = (g->rs_max - g->rs_min) / (nr - 1);\n    double dth",
     "double h = (g->rs_max - g->rs_min) / nr;\n    double dth", [ASSEMBLY]),
    ("theta WENO: downwind", "int dir = (-Bth_here < 0.0) ? -1 : +1;",
     "int dir = (-Bth_here < 0.0) ? +1 : -1;",
     [PH + "test_theta_weno_stencil_lies_upwind"]),
    ("negative-direction IS_0: wrong node",
     "IS[0] = 13.0 / 12.0 * pow(f[2] - 2 * f[3] + f[4], 2)",
     "IS[0] = 13.0 / 12.0 * pow(f[1] - 2 * f[3] + f[4], 2)",
     [P + "test_fifth_order_convergence_on_periodic_advection"]),
    ("reduced IS: 1/2 for 1/4", "c14 = 0.25,", "c14 = 0.5,",
     [P + "test_reduced_weights_within_rounding_of_fp64_weights"]),
    ("rounding: subnormal spacing ignored", "if (E < emin) E = emin;", "",
     [P + "test_round_w_matches_numpy_and_torch"]),
    ("rounding: no overflow to infinity", "if (fabs(y) > maxfinite) return copysign(INFINITY, x);",
     "", [P + "test_round_w_matches_numpy_and_torch"]),
    ("FD6: 30 h for 60 h", "/ (60.0 * h);", "/ (30.0 * h);",
     [P + "test_fd6_exact_to_degree_six_and_sixth_order"]),
    ("KO8: three D- for four", "for (int r = 0; r < 4; ++r)\n        for (int k = m - 1;",
     "for (int r = 0; r < 3; ++r)\n        for (int k = m - 1;",
     [P + "test_ko8_annihilates_degree_seven_and_has_its_fourier_symbol"]),
    ("SSP-RK(3,3): half step in stage 1", "u1[k] = u[k] + dt * Fv[k];",
     "u1[k] = u[k] + 0.5 * dt * Fv[k];", [P + "test_ssprk33_stability_polynomial"]),
    ("SSP-RK(10,4): three stages before u5", "for (int i = 1; i <= 4; ++i) {",
     "for (int i = 1; i <= 3; ++i) {", [P + "test_ssprk104_fourth_order_convergence"]),
    ("test equation: sign of Im lambda", "F[0] = c->lr * y[0] - c->li * y[1];",
     "F[0] = c->lr * y[0] + c->li * y[1];", [P + "test_ssprk33_stability_polynomial"]),
    ("advection: backwards", "F[i] = -(double)c->dir * F[i];", "F[i] = (double)c->dir * F[i];",
     [P + "test_fifth_order_convergence_on_periodic_advection"]),
    ("observe: horizon gather one node in", "horizon[6 * j + c] = u[c * plane + row];",
     "horizon[6 * j + c] = u[c * plane + row + 1];",
     [PH + "test_observe_gathers_nodes_and_one_sided_derivative"]),
    ("FD6 on the slices with edge-copy ghosts",
     "g->coords == 1 ? 2 : 0, &Dc[c * nr], &Qc[c * nr]);", "0, &Dc[c * nr], &Qc[c * nr]);",
     [ASSEMBLY]),
    ("WENO on the slices with edge-copy ghosts",
     "g->eps, g->coords == 1 ? 2 : 0, NULL, &Dc[c * nr],", "g->eps, 0, NULL, &Dc[c * nr],",
     [ASSEMBLY]),
    ("theta WENO: pole ghost mirrored on the node",
     "if (jj < 0) { jj = -1 - jj; sg = sigma; }\n                    if (jj >= nth)",
     "if (jj < 0) { jj = -jj; sg = sigma; }\n                    if (jj >= nth)",
     [PH + "test_theta_weno_option_on_spin_weighted_harmonics"]),
    ("theta WENO: direction from Ath instead of Bth", "double Bth_here = coef[8 * plane + p];",
     "double Bth_here = coef[7 * plane + p];", [PH + "test_theta_weno_stencil_lies_upwind"]),
    ("theta WENO: flux difference over 2 dtheta", "d[c] = (fp - fm) / dth;",
     "d[c] = (fp - fm) / (2.0 * dth);", [PH + "test_theta_weno_option_on_spin_weighted_harmonics"]),
    ("hyperboloidal db/drho: a real-size complex step", "double hstep = 1e-30;",
     "double hstep = 1e-2;", [SYM_HYP]),
    # observation, Sec. 4
    ("observe: one-sided derivative over h", "horizon[6 * j + 4 + c] = (-3.0 * f[0] + 4.0 * f[1] - f[2]) / (2.0 * h);",
     "horizon[6 * j + 4 + c] = (-3.0 * f[0] + 4.0 * f[1] - f[2]) / h;",
     [PH + "test_observe_gathers_nodes_and_one_sided_derivative"]),
    ("observe: truncated node index", "long ie = lround((rs_ext - g->rs_min) / h);",
     "long ie = (long)((rs_ext - g->rs_min) / h);",
     [PH + "test_observe_gathers_nodes_and_one_sided_derivative"]),
]


LD = "tests/test_oracle_ld.py::"
LD_FLUX = LD + "test_flux_of_linear_data_in_closed_form"
LD_LIN = LD + "test_rhs_of_linear_state_in_closed_form"
LD_RHS = LD + "test_rhs_agrees_with_binary64_oracle"
LD_EVO = LD + "test_evolution_agrees_with_binary64_oracle"
LD_PREC = LD + "test_evolution_carries_the_extended_precision"

LD_MUTANTS = [
    ("ld: candidate value q1 over 5", "q[1] = (-g[1] + 5 * g[2] + 2 * g[3]) / 6.0L;",
     "q[1] = (-g[1] + 5 * g[2] + 2 * g[3]) / 5.0L;", [LD_FLUX]),
    ("ld: q2 with g3 and g4 swapped", "q[2] = (2 * g[2] + 5 * g[3] - g[4]) / 6.0L;",
     "q[2] = (2 * g[2] + 5 * g[4] - g[3]) / 6.0L;", [LD_FLUX]),
    ("ld: linear weights reversed", "const real d[3] = {0.1L, 0.6L, 0.3L};",
     "const real d[3] = {0.3L, 0.6L, 0.1L};", [LD_RHS]),
    ("ld: IS0 second term 3 -> 2", "t = g[0] - 4 * g[1] + 3 * g[2];",
     "t = g[0] - 4 * g[1] + 2 * g[2];", [LD_RHS]),
    ("ld: alpha with the first power", "alpha[k] = d[k] / (e * e);",
     "alpha[k] = d[k] / e;", [LD_RHS]),
    ("ld: negative-direction stencil one node left", "dir > 0 ? &ext[i + 1] : &ext[i + 2]",
     "dir > 0 ? &ext[i + 1] : &ext[i + 1]", [LD_LIN, LD_RHS]),
    ("ld: quartic ghost through the wrong nodes", "const int x0 = k < 0 ? 0 : n - 5;",
     "const int x0 = k < 0 ? 0 : n - 6;", [LD_RHS]),
    ("ld: sign of b D_Psi", "const creal_t Fpsi = pi - b * Dpsi;",
     "const creal_t Fpsi = pi + b * Dpsi;", [LD_LIN, LD_RHS]),
    ("ld: C multiplies pi", "+ Bt * pi + C * psi;", "+ Bt * pi + C * pi;", [LD_LIN, LD_RHS]),
    ("ld: sign of the theta first derivative",
     "(nb[0] - 8 * nb[1] + 8 * nb[3] - nb[4]) / (12 * dth)",
     "(nb[4] - 8 * nb[3] + 8 * nb[1] - nb[0]) / (12 * dth)", [LD_RHS]),
    ("ld: pole mirror off by one", "if (jj < 0) { jj = -1 - jj; s = sigma; }",
     "if (jj < 0) { jj = -jj; s = sigma; }", [LD_RHS]),
    ("ld: stage 2 combines u1 for u", "u2[k] = 0.75L * u[k] + 0.25L * (u1[k] + dt * Fv[k]);",
     "u2[k] = 0.75L * u1[k] + 0.25L * (u1[k] + dt * Fv[k]);", [LD_EVO]),
    ("ld: stage 1 through binary64", "u1[k] = u[k] + dt * Fv[k];",
     "u1[k] = (double)u[k] + dt * Fv[k];", [LD_PREC]),
    ("ld: stage 3 through binary64", "u[k] = u[k] / 3 + 2 * (u2[k] + dt * Fv[k]) / 3;",
     "u[k] = (double)(u[k] / 3 + 2 * (u2[k] + dt * Fv[k]) / 3);", [LD_PREC]),
    ("ld: flux accumulated in binary64", "real fh = 0.0L;", "double fh = 0.0L;",
     [LD_FLUX, LD_LIN]),
]


def _run_pins(lib_path, pins, var="TEUK_ORACLE_LIB"):
    env = dict(os.environ, OMP_NUM_THREADS="2")
    env[var] = lib_path
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
           *pins]
    out = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return out.returncode, out.stdout[-2000:]


def _compile(tmp, tag, text):
    src = os.path.join(tmp, f"oracle_{tag}.c")
    with open(src, "w") as fh:
        fh.write(text)
    return o.build(force=True, src=src, out=os.path.join(tmp, f"liboracle_{tag}.so"))


def test_mutants_are_distinct_single_edits():
    text = open(SRC).read()
    names = [m[0] for m in MUTANTS]
    assert len(set(names)) == len(names)
    for name, old, new, pins in MUTANTS:
        assert text.count(old) == 1, name
        assert old != new and pins, name


@pytest.mark.slow
def test_every_planted_mistake_fails_a_pin(tmp_path):
    text = open(SRC).read()
    tmp = str(tmp_path)
    all_pins = sorted({p for m in MUTANTS for p in m[3]})
    jobs = [("original", text, all_pins)]
    for k, (name, old, new, pins) in enumerate(MUTANTS):
        jobs.append((name, text.replace(old, new), pins))

    def job(k):
        _, mutated, pins = jobs[k]
        return _run_pins(_compile(tmp, str(k), mutated), pins)

    workers = max(1, min(8, (os.cpu_count() or 2) // 2))
    with cf.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(job, range(len(jobs))))
    rc0, log0 = results[0]
    assert rc0 == 0, "the unaltered oracle fails its pins:\n" + log0
    survivors = [(j[0], rc, log) for j, (rc, log) in zip(jobs[1:], results[1:]) if rc != 1]
    assert not survivors, "\n\n".join(f"{n}: pytest exit {rc}\n{log}" for n, rc, log in survivors)


def test_ld_mutants_are_distinct_single_edits():
    text = open(SRC_LD).read()
    names = [m[0] for m in LD_MUTANTS]
    assert len(set(names)) == len(names)
    for name, old, new, pins in LD_MUTANTS:
        assert text.count(old) == 1, name
        assert old != new and pins, name


@pytest.mark.slow
def test_every_planted_ld_mistake_fails_a_pin(tmp_path):
    text = open(SRC_LD).read()
    tmp = str(tmp_path)
    all_pins = sorted({p for m in LD_MUTANTS for p in m[3]})
    jobs = [("original", text, all_pins)]
    for name, old, new, pins in LD_MUTANTS:
        jobs.append((name, text.replace(old, new), pins))

    def job(k):
        _, mutated, pins = jobs[k]
        src = os.path.join(tmp, f"oracle_ld_{k}.c")
        with open(src, "w") as fh:
            fh.write(mutated)
        lib = o.build_ld(force=True, src=src, out=os.path.join(tmp, f"liboracle_ld_{k}.so"))
        return _run_pins(lib, pins, "TEUK_ORACLE_LD_LIB")

    workers = max(1, min(8, (os.cpu_count() or 2) // 2))
    with cf.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(job, range(len(jobs))))
    rc0, log0 = results[0]
    assert rc0 == 0, "the unaltered extended oracle fails its pins:\n" + log0
    survivors = [(j[0], rc, log) for j, (rc, log) in zip(jobs[1:], results[1:]) if rc != 1]
    assert not survivors, "\n\n".join(f"{n}: pytest exit {rc}\n{log}" for n, rc, log in survivors)
