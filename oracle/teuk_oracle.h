/*
 * Plain FP64 CPU oracle for the mixed-precision WENO5 Teukolsky stage operator
 * (Field, Gottlieb, Grant, Isherwood, Khanna, arXiv 2010.04760).
 *
 * TEST INFRASTRUCTURE ONLY. This library exists to check the CUDA path. Only the
 * test suite, __graft_entry__.smoke() and bench.py (its cpu_baseline leg and its
 * reference arm) may load it. It shares no code, header, table or helper with the
 * CUDA library; the two are independent implementations of the same equations.
 *
 * Array layout used by every 2-D routine: component-major planes
 *   u[c][j][i], c in {Psi_R, Psi_I, pi_R, pi_I}, j = theta row (0..nth-1),
 *   i = r* index (0..nr-1, fastest).
 * Coefficient layout (complex first-order form, see orc_coeff_point):
 *   coef[k][j][i], k = 0..9 : b, K_re, K_im, Bt_re, Bt_im, C_re, C_im, Ath, Bth,
 *   c (the pi rows' speed; c = b in r*).
 * The radial coordinate is r* (coords 0) or the hyperboloidal rho (coords 1);
 * rs_min, rs_max hold its range either way.
 *
 * Weight precision codes: 0 = binary64 (paper formulas), 1 = binary32,
 * 2 = binary16, 3 = bfloat16 (reduced-precision reading, see teuk_oracle.c),
 * 4 = the reduced-precision reading carried out in binary64 (used only to show
 * that the reading is the paper's formula rearranged).
 *
 * Parity status: every routine is pinned by the tests in tests/test_oracle_pins.py,
 * tests/test_oracle_physics.py and tests/test_oracle_hyperboloidal.py (and
 * tests/test_oracle_mutants.py shows that single-edit mistakes planted in each
 * routine of a copy of teuk_oracle.c make those pins fail), except the
 * Aretakis-charge interpretation of the horizon gather in r*, which is "parity
 * unpinned" (the extremal horizon is not on an r* grid). On the hyperboloidal
 * grid the horizon is node 0 and the Aretakis laws are pinned.
 */
#ifndef TEUK_ORACLE_H
#define TEUK_ORACLE_H

typedef struct {
    int nr, nth;             /* grid points in r* and theta                      */
    double rs_min, rs_max;   /* r* domain (units of M)                           */
    double M, a;             /* black-hole mass and spin                         */
    int s, m;                /* spin weight and azimuthal mode number            */
    double eps;              /* WENO epsilon                                     */
    int wprec;               /* weight precision code                            */
    int theta_mode;          /* 0: centred dtheta; 1: WENO5 dtheta (reading)     */
    int scheme;              /* 0: WENO5 in r*; 1: FD6 + KO8 (Sec. 3.1.1)        */
    double ko_sigma;         /* Kreiss-Oliger sigma of scheme 1                  */
    int coords;              /* 0: BL t and r*; 1: hyperboloidal (tau, rho)      */
    int field;               /* 0: Psi; 1: Phi = r Delta^s Psi (always in 1)     */
    double S;                /* hyperboloidal slice parameter (coords 1)         */
} orc_grid;

double orc_rstar_of_r(double r, double M, double a);
double orc_r_of_rstar(double rs, double M, double a);
double orc_x_of_rstar(double rs, double M, double a);   /* r - r_+ at r*      */
void   orc_coeff_point(double r, double th, double M, double a, int s, int m,
                       int field, double out[10]);
double orc_rho_of_r(double r, double S);
void   orc_coeff_point_hyp(double rho, double th, double M, double a, double S,
                           int s, int m, double out[10]);
void   orc_coefficients(const orc_grid* g, double* coef);
double orc_round_w(int wprec, double x);
void   orc_weno5_weights(int wprec, int dir, const double* f5, double eps,
                         double w[3]);
double orc_weno5_flux(int wprec, int dir, const double* f5, double eps,
                      const double* force_w, double w_out[3], double q_out[3]);
void   orc_fd6_ko8_1d(const double* f, int n, double h, double sigma, int bc,
                      double* D, double* Q);
void   orc_weno5_deriv_1d(const double* f, int n, double h, int dir, int wprec,
                          double eps, int bc, const double* force_w,
                          double* D, double* w_out, double* q_out);
void   orc_rhs(const orc_grid* g, const double* coef, const double* u, double* F);
void   orc_rk3_step(const orc_grid* g, const double* coef, double dt, double* u,
                    long nsteps);
void   orc_rk3_linear(double lam_re, double lam_im, double dt, long nsteps,
                      double y[2]);
void   orc_rk104_step(const orc_grid* g, const double* coef, double dt, double* u,
                      long nsteps);
void   orc_rk104_linear(double lam_re, double lam_im, double dt, long nsteps,
                        double y[2]);
void   orc_advect_1d(double* f, int n, double h, double dt, long nsteps, int dir,
                     int wprec, double eps);
void   orc_observe(const orc_grid* g, const double* u, double rs_ext,
                   double* wave, double* horizon);
int    orc_num_threads(void);

#endif
