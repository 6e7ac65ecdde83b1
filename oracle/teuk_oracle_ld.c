/*
 * Extended-precision state evolution for the oracle: the WENO5 Teukolsky
 * right-hand side and SSP-RK(3,3) step of teuk_oracle.c with every state
 * quantity, weight and flux in C `long double` (binary128 on aarch64 Linux,
 * the x87 64-bit-significand format on x86-64; orc_ld_mant_dig reports which).
 *
 * TEST INFRASTRUCTURE ONLY, like teuk_oracle.c: it measures the round-off of
 * the binary64 state itself. The paper keeps its state in quad precision
 * because at late times the multipoles of the field sit 15-20 decades apart
 * and binary64 round-off would swamp the fast-decaying ones (Sec. 2.3, the
 * paragraph on high-precision numerics); its mixed-precision scheme keeps the
 * state and the flux assembly in the high precision and only the weights in
 * the low one (Sec. 3.1.3). Evolving the same discretisation here with a wider
 * state and comparing with the binary64 evolution gives the binary64 state's
 * own error, the quantity the paper's quad baseline controls.
 *
 * Scope: the configurations whose state error is measured: WENO5 in the
 * radial coordinate (scheme 0), centred fourth-order theta derivatives
 * (theta_mode 0), weights in the state's precision (the paper's formulas,
 * Sec. 3.1.2; g->wprec is not consulted), both coordinate systems (ghosts:
 * edge copies in r*, the quartic through the five edge nodes on the
 * hyperboloidal grid), SSP-RK(3,3) (Sec. 3.2). Other schemes return -1.
 * The discrete problem is the binary64 codes' own: the coefficients are the
 * binary64 arrays of orc_coefficients and the spacings h and dtheta, eps and
 * dt the binary64 values those codes use, all promoted exactly, so that the
 * two evolutions differ only in the precision of the state arithmetic.
 *
 * Layout as in teuk_oracle.h: u[c][j][i], c = Psi_R, Psi_I, pi_R, pi_I.
 */
#include <complex.h>
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "teuk_oracle.h"

typedef long double real;
typedef long double complex creal_t;

int orc_ld_mant_dig(void) { return LDBL_MANT_DIG; }

/* WENO5 numerical flux at j+1/2 (Sec. 3.1.2). dir = +1: f = f_{j-2..j+2};
 * dir = -1: f = f_{j-1..j+3} (the mirror image). Smoothness indicators IS_k,
 * alpha_k = d_k / (eps + IS_k)^2, omega_k = alpha_k / sum alpha, and the
 * third-order candidate values q_k, all in long double. */
static real weno5_flux(int dir, const real* f, real eps) {
    /* the positive-direction stencil: g = f; the negative one mirrored */
    real g[5];
    for (int k = 0; k < 5; ++k) g[k] = dir > 0 ? f[k] : f[4 - k];
    const real d[3] = {0.1L, 0.6L, 0.3L};
    real IS[3], q[3], alpha[3], sum = 0.0L;
    real t;
    t = g[0] - 2 * g[1] + g[2];
    IS[0] = 13.0L / 12.0L * t * t;
    t = g[0] - 4 * g[1] + 3 * g[2];
    IS[0] += 0.25L * t * t;
    t = g[1] - 2 * g[2] + g[3];
    IS[1] = 13.0L / 12.0L * t * t;
    t = g[1] - g[3];
    IS[1] += 0.25L * t * t;
    t = g[2] - 2 * g[3] + g[4];
    IS[2] = 13.0L / 12.0L * t * t;
    t = 3 * g[2] - 4 * g[3] + g[4];
    IS[2] += 0.25L * t * t;
    q[0] = (2 * g[0] - 7 * g[1] + 11 * g[2]) / 6.0L;
    q[1] = (-g[1] + 5 * g[2] + 2 * g[3]) / 6.0L;
    q[2] = (2 * g[2] + 5 * g[3] - g[4]) / 6.0L;
    for (int k = 0; k < 3; ++k) {
        const real e = eps + IS[k];
        alpha[k] = d[k] / (e * e);
        sum += alpha[k];
    }
    real fh = 0.0L;
    for (int k = 0; k < 3; ++k) fh += alpha[k] / sum * q[k];
    return fh;
}

/* The flux above for a caller: eps and the result by pointer, so that no
 * conversion through binary64 touches them. */
void orc_ld_weno5_flux(int dir, const real* f, const real* eps, real* out) {
    *out = weno5_flux(dir, f, *eps);
}

/* Lagrange extrapolation of the quartic through the five edge nodes to the
 * ghost index k (k < 0 or k >= n). */
static real ghost_quartic(const real* f, int n, int k) {
    const int x0 = k < 0 ? 0 : n - 5;
    real v = 0.0L;
    for (int j = x0; j < x0 + 5; ++j) {
        real L = 1.0L;
        for (int l = x0; l < x0 + 5; ++l)
            if (l != j) L *= (real)(k - l) / (real)(j - l);
        v += L * f[j];
    }
    return v;
}

/* D_i = (fhat_{i+1/2} - fhat_{i-1/2}) / h along one radial line. */
static void weno5_deriv(const real* f, int n, real h, int dir, real eps, int hyp,
                        real* ext, real* fh, real* D) {
    for (int k = -3; k < n + 3; ++k) {
        if (k >= 0 && k < n) ext[k + 3] = f[k];
        else if (hyp) ext[k + 3] = ghost_quartic(f, n, k);
        else ext[k + 3] = f[k < 0 ? 0 : n - 1];
    }
    for (int i = -1; i < n; ++i)
        fh[i + 1] = weno5_flux(dir, dir > 0 ? &ext[i + 1] : &ext[i + 2], eps);
    for (int i = 0; i < n; ++i) D[i] = (fh[i + 1] - fh[i]) / h;
}

/* F(u) = -(M du/dx + L u + A u) (Eq. evln) in complex first-order form,
 *   F_Psi = pi - b D_Psi,
 *   F_pi  = c D_pi + K D_Psi + Ath Psi_thth + Bth Psi_th + Bt pi + C Psi,
 * Psi rows with the positive-direction flux, pi rows with the negative one;
 * theta derivatives fourth-order centred, rows past a pole mirrored with
 * parity (-1)^(m+s). */
int orc_ld_rhs(const orc_grid* g, const double* coef, const real* u, real* F) {
    if (g->scheme != 0 || g->theta_mode != 0) return -1;
    const int nr = g->nr, nth = g->nth;
    const long plane = (long)nr * nth;
    const real h = (g->rs_max - g->rs_min) / (nr - 1);        /* binary64 spacings */
    const real dth = M_PI / nth;
    const real sigma = ((g->m + g->s) % 2 == 0) ? 1.0L : -1.0L;
    const int hyp = g->coords == 1;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < nth; ++j) {
        real* Dc = (real*)malloc(sizeof(real) * 4 * nr);
        real* ext = (real*)malloc(sizeof(real) * (nr + 6));
        real* fh = (real*)malloc(sizeof(real) * (nr + 1));
        for (int c = 0; c < 4; ++c)
            weno5_deriv(&u[c * plane + (long)j * nr], nr, h, c < 2 ? +1 : -1, (real)g->eps,
                        hyp, ext, fh, &Dc[c * nr]);
        int rows[5];
        real sg[5];
        for (int k = -2; k <= 2; ++k) {
            int jj = j + k;
            real s = 1.0L;
            if (jj < 0) { jj = -1 - jj; s = sigma; }
            if (jj >= nth) { jj = 2 * nth - 1 - jj; s = sigma; }
            rows[k + 2] = jj;
            sg[k + 2] = s;
        }
        for (int i = 0; i < nr; ++i) {
            const long p = (long)j * nr + i;
            const creal_t psi = u[p] + I * u[plane + p];
            const creal_t pi = u[2 * plane + p] + I * u[3 * plane + p];
            const creal_t Dpsi = Dc[i] + I * Dc[nr + i];
            const creal_t Dpi = Dc[2 * nr + i] + I * Dc[3 * nr + i];
            creal_t nb[5];
            for (int k = 0; k < 5; ++k) {
                const long q = (long)rows[k] * nr + i;
                nb[k] = sg[k] * (u[q] + I * u[plane + q]);
            }
            const creal_t psi_th = (nb[0] - 8 * nb[1] + 8 * nb[3] - nb[4]) / (12 * dth);
            const creal_t psi_thth =
                (-nb[0] + 16 * nb[1] - 30 * nb[2] + 16 * nb[3] - nb[4]) / (12 * dth * dth);
            const real b = coef[p];
            const creal_t K = coef[plane + p] + I * (real)coef[2 * plane + p];
            const creal_t Bt = coef[3 * plane + p] + I * (real)coef[4 * plane + p];
            const creal_t C = coef[5 * plane + p] + I * (real)coef[6 * plane + p];
            const real Ath = coef[7 * plane + p], Bth = coef[8 * plane + p];
            const real cpi = coef[9 * plane + p];
            const creal_t Fpsi = pi - b * Dpsi;
            const creal_t Fpi = cpi * Dpi + K * Dpsi + Ath * psi_thth + Bth * psi_th
                                + Bt * pi + C * psi;
            F[p] = creall(Fpsi);
            F[plane + p] = cimagl(Fpsi);
            F[2 * plane + p] = creall(Fpi);
            F[3 * plane + p] = cimagl(Fpi);
        }
        free(Dc);
        free(ext);
        free(fh);
    }
    return 0;
}

/* SSP-RK(3,3) in Shu-Osher form (Sec. 3.2). */
int orc_ld_rk3_step(const orc_grid* g, const double* coef, double dt_in, real* u,
                    long nsteps) {
    if (g->scheme != 0 || g->theta_mode != 0) return -1;
    const long n = 4L * g->nr * g->nth;
    const real dt = dt_in;
    real* u1 = (real*)malloc(sizeof(real) * n);
    real* u2 = (real*)malloc(sizeof(real) * n);
    real* Fv = (real*)malloc(sizeof(real) * n);
    for (long step = 0; step < nsteps; ++step) {
        orc_ld_rhs(g, coef, u, Fv);
        for (long k = 0; k < n; ++k) u1[k] = u[k] + dt * Fv[k];
        orc_ld_rhs(g, coef, u1, Fv);
        for (long k = 0; k < n; ++k) u2[k] = 0.75L * u[k] + 0.25L * (u1[k] + dt * Fv[k]);
        orc_ld_rhs(g, coef, u2, Fv);
        for (long k = 0; k < n; ++k) u[k] = u[k] / 3 + 2 * (u2[k] + dt * Fv[k]) / 3;
    }
    free(u1);
    free(u2);
    free(Fv);
    return 0;
}
