/*
 * Plain FP64 CPU oracle for the mixed-precision WENO5 Teukolsky stage operator
 * of arXiv 2010.04760. TEST INFRASTRUCTURE ONLY: only the test suite,
 * __graft_entry__.smoke() and bench.py (cpu_baseline leg, reference arm) may
 * load it; the product (CUDA) path never does. It shares no code with the CUDA
 * library. Every routine follows the paper's steps in the paper's order, with
 * plain loops; the passage each one follows is cited beside it.
 *
 * Readings of points the paper leaves open:
 *  - Coordinates (coords 0): Boyer-Lindquist time t, tortoise r*, ingoing
 *    azimuth phi~ (Sec. 2.2). coords 1: the paper's hyperboloidal slices
 *    (tau, rho) of Sec. 2.2, whose coefficients (Eq. near_final) the paper
 *    does not print; they are derived here from Eq. teuk0 for the field
 *    Phi = r Delta^s Psi (the paper's Phi of Sec. 4 at s = -2), and the grid
 *    runs from the horizon rho_+ to at most scri (rho = S). The "4 ln" of the
 *    slice's height function is read as 4 M ln (the paper sets M = 1).
 *  - Field (field 1): Phi = r Delta^s Psi in either coordinate system.
 *  - First-order variable pi = Psi_t + b Psi_* with b the larger root of
 *    b^2 + Atr b - Arr = 0 (b = +sqrt(A**) > 0 in r*), so the Psi rows move
 *    with speed +b (outgoing) and the pi rows with -c, c = Atr + b (ingoing);
 *    in r* c = b, as Sec. 3.1 states.
 *  - Radial boundaries: in r*, ghost values copy the edge value (zeroth-order
 *    extrapolation). On the hyperboloidal grid both ends are outflow
 *    boundaries (horizon and scri); ghosts extrapolate the polynomial through
 *    the edge nodes. theta: cell-centred grid, ghost rows mirror across the
 *    poles with parity (-1)^(m+s).
 *  - theta derivatives: fourth-order centred differences (the paper says
 *    centred differences without an order). Optional theta WENO
 *    (theta_mode 1): the first derivative in the Bth term is the WENO5
 *    derivative along theta, upwinded by the sign of the term's speed -Bth
 *    (the term read as -(-Bth) dPsi/dtheta), with weights in the same
 *    precision as in r*; the second derivative stays centred.
 *  - Reduced-precision weights: first differences formed in binary64, scaled
 *    by a power of two, rounded to the weight format; smoothness indicators,
 *    epsilon, alpha and omega computed in that format with every operation
 *    rounded; alpha normalised by the smallest (eps + IS). omega_0, omega_2
 *    promoted to binary64 and omega_1 = 1 - omega_0 - omega_2 there (Sec. 3.1.3).
 *  - WENO epsilon: a parameter (1e-6 by default), unstated in the paper.
 *  - Comparison scheme (scheme 1, Sec. 3.1.1): the sixth-order centred radial
 *    derivative for all four components and the Kreiss-Oliger term
 *    sigma h^7 D+^4 D-^4 / 256 subtracted from every component's right-hand
 *    side (the sign that damps), with the same ghosts as for WENO (edge
 *    copies in r*, the quartic extrapolation on the hyperboloidal grid).
 */
#include <math.h>
#include <complex.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include "teuk_oracle.h"

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Tortoise coordinate, r* = int (r^2+a^2)/Delta dr (Sec. 2.2). Integration  */
/* constant: the one that makes r* -> r + 2M ln(r/2M - 1) at a = 0. Written  */
/* in y = ln(r - r_+): towards the horizon r - r_+ falls off exponentially    */
/* in r* (e-folding length 2M r_+/(r_+ - r_-)), below the spacing of binary64 */
/* numbers near r_+ once r* is a few tens of M negative, so r itself cannot  */
/* carry it and Delta = (r - r_+)(r - r_-) must be formed from r - r_+.       */
/* ------------------------------------------------------------------------ */
static double rstar_of_lnx(double y, double M, double a) {
    double x = exp(y);
    if (fabs(a) < M) {
        double d = sqrt(M * M - a * a);
        double rp = M + d, rm = M - d;
        return rp + x + (2.0 * M * rp / (rp - rm)) * (y - log(2.0 * M))
                 - (2.0 * M * rm / (rp - rm)) * log((x + rp - rm) / (2.0 * M));
    }
    /* extremal a = M: Delta = (r - M)^2 */
    return M + x + 2.0 * M * (y - log(M)) - 2.0 * M * M * exp(-y);
}

static double horizon_r(double M, double a) { return M + sqrt(fmax(M * M - a * a, 0.0)); }

double orc_rstar_of_r(double r, double M, double a) {
    return rstar_of_lnx(log(r - horizon_r(M, a)), M, a);
}

/* r - r_+ at r*, by bisection on y = ln(r - r_+) (y -> r* is monotone). */
double orc_x_of_rstar(double rs, double M, double a) {
    double lo = -1.0, hi = 1.0;
    while (rstar_of_lnx(lo, M, a) > rs && lo > -1.0e6) lo *= 2.0;
    while (rstar_of_lnx(hi, M, a) < rs) hi *= 2.0;
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (rstar_of_lnx(mid, M, a) < rs) lo = mid; else hi = mid;
    }
    return exp(0.5 * (lo + hi));
}

double orc_r_of_rstar(double rs, double M, double a) {
    return horizon_r(M, a) + orc_x_of_rstar(rs, M, a);
}

/* ------------------------------------------------------------------------ */
/* Coefficients of the first-order system (Eqs. final, evln; matrices M, A,  */
/* L) obtained from the Teukolsky master equation (Eq. teuk0) with           */
/* Psi = exp(i m phi~) psi(t, r*, theta):                                    */
/*   psi_tt = A** psi_** + B* psi_* + Ath psi_thth + Bth psi_th              */
/*            + Bt psi_t + C psi                                             */
/* with varpi = r^2+a^2, Delta = r^2-2Mr+a^2, Sigma2 = varpi^2 -             */
/* a^2 Delta sin^2(theta), and                                               */
/*   A** = varpi^2/Sigma2,                                                   */
/*   B*  = [2 r Delta + 2 i m a varpi + 2 s (r-M) varpi]/Sigma2,             */
/*   Ath = Delta/Sigma2, Bth = Delta cot(theta)/Sigma2,                      */
/*   Bt  = [-4 i M a m r - 2 s (r Delta - M (r^2-a^2)) - 2 i s a Delta       */
/*          cos(theta)]/Sigma2,                                              */
/*   C   = [4 i s m a (r-M) + Delta (s - (m + s cos)^2/sin^2)]/Sigma2.       */
/* First-order form (Sec. 2.3): pi = psi_t + b psi_*, b = sqrt(A**), so      */
/*   psi_t = pi - b psi_*,                                                   */
/*   pi_t  = b pi_* + K psi_* + Ath psi_thth + Bth psi_th + Bt pi + C psi,   */
/*   K = B* - b b_* - b Bt,  b_* = d b / d r* = (Delta/varpi) d b / d r.     */
/* field 1 evolves Phi = Psi / g, g = Delta^-s / r: with                      */
/*   g1 = (dg/dr*) / g = -(s Delta' + Delta/r)/varpi,                        */
/*   g2 = (d2g/dr*2) / g = dg1/dr* + g1^2,                                   */
/* the Phi equation has B* + 2 A** g1 in place of B* and C + A** g2 + B* g1  */
/* in place of C (Bt, Ath, Bth unchanged: there is no t-r* cross term).      */
/* out = {b, Re K, Im K, Re Bt, Im Bt, Re C, Im C, Ath, Bth, c}, c = b.      */
/* ------------------------------------------------------------------------ */
/* x = r - r_+ given beside r (Delta = x (x + r_+ - r_-), no cancellation). */
static void coeff_point_rx(double r, double x, double th, double M, double a, int s,
                           int m, int field, double out[10]) {
    double sn = sin(th), cs = cos(th);
    double varpi = r * r + a * a;
    double Delta = x * (x + 2.0 * sqrt(fmax(M * M - a * a, 0.0)));
    double Sigma2 = varpi * varpi - a * a * Delta * sn * sn;
    double Sigma = sqrt(Sigma2);

    double complex Bstar = (2.0 * r * Delta + 2.0 * I * m * a * varpi
                            + 2.0 * s * (r - M) * varpi) / Sigma2;
    double Ath = Delta / Sigma2;
    double Bth = Delta * (cs / sn) / Sigma2;
    double complex Bt = (-4.0 * I * M * a * m * r
                         - 2.0 * s * (r * Delta - M * (r * r - a * a))
                         - 2.0 * I * s * a * Delta * cs) / Sigma2;
    double mc = m + s * cs;
    double complex C = (4.0 * I * s * m * a * (r - M)
                        + Delta * (s - mc * mc / (sn * sn))) / Sigma2;
    double Axx = varpi * varpi / Sigma2;

    if (field == 1) {
        /* g1(r) = -N/varpi, N = 2s(r-M) + Delta/r */
        double N = 2.0 * s * (r - M) + Delta / r;
        double dN = 2.0 * s + 1.0 - a * a / (r * r);
        double g1 = -N / varpi;
        double dg1_dr = -(dN * varpi - N * 2.0 * r) / (varpi * varpi);
        double g2 = (Delta / varpi) * dg1_dr + g1 * g1;
        C = C + Axx * g2 + Bstar * g1;
        Bstar = Bstar + 2.0 * Axx * g1;
    }

    double b = varpi / Sigma;
    double dSigma2_dr = 2.0 * varpi * (2.0 * r) - a * a * sn * sn * 2.0 * (r - M);
    double db_dr = 2.0 * r / Sigma - varpi * dSigma2_dr / (2.0 * Sigma2 * Sigma);
    double b_star = (Delta / varpi) * db_dr;
    double complex K = Bstar - b * b_star - b * Bt;

    out[0] = b;
    out[1] = creal(K);  out[2] = cimag(K);
    out[3] = creal(Bt); out[4] = cimag(Bt);
    out[5] = creal(C);  out[6] = cimag(C);
    out[7] = Ath;       out[8] = Bth;
    out[9] = b;
}

void orc_coeff_point(double r, double th, double M, double a, int s, int m,
                     int field, double out[10]) {
    coeff_point_rx(r, r - horizon_r(M, a), th, M, a, s, m, field, out);
}

/* ------------------------------------------------------------------------ */
/* Hyperboloidal slices (Sec. 2.2): ingoing Kerr t~ = t - r + r*,            */
/* phi~ = phi + int a/Delta dr, then                                         */
/*   tau = t~ - r^2/(r+S) + 4M ln(S/(r+S)),   rho = r/(1 + r/S),             */
/* and the field Phi = r Delta^s Psi (Sec. 4). Written as                    */
/*   A^tt Phi_tt + A^tr Phi_tr + A^rr Phi_rr + Phi_thth + cot Phi_th         */
/*   + B^t Phi_t + B^r Phi_r + C Phi = 0   (t = tau, r = rho here)           */
/* this is Eq. near_final; dividing by D = -A^tt > 0 gives Eq. final.        */
/* Derived by the chain rule from Eq. teuk0 with tau = t + T(r),             */
/* T' = varpi/Delta - H', H' = 2 - W^2 + 4MW/S, rho' = W^2, W = S/(r+S)      */
/* = 1 - rho/S, and written in x = 1/r = 1/rho - 1/S, W and rho so that      */
/* every term stays finite and free of cancellation from the horizon to      */
/* scri (x = 0, W = 0, rho = S):                                             */
/*   delta = Delta/r^2 = 1 - 2Mx + a^2 x^2,  w = varpi/r^2 = 1 + a^2 x^2,    */
/*   sig = Sigma/r^2 = sqrt(w^2 - a^2 x^2 delta sin^2),                      */
/*   G  = 2 varpi - Delta H'                                                 */
/*      = rho (rho + 4M + 8M^2/S - 2MW + a^2 x (W - 4M/S)),                  */
/*   E  = Sigma + varpi - Delta H' = G - a^2 delta sin^2 / (sig + w),        */
/*   D  = H' G - a^2 sin^2,                                                  */
/*   A^tr = 2 W^2 (varpi - Delta H'),  A^rr = rho^2 W^2 delta,               */
/*   B^t = 2s rho (4M/S - W) - 2(1+s) M H' + 2a^2 x (H' - 1)                 */
/*         - 2 delta rho^2 (W - 2M/S)/S + i (2ma (1 - H') - 2sa cos),        */
/*   B^r = 2ima W^2 - 2W rho ((s+1) - W - rho x (2M - a^2 x)/S)              */
/*         + 2W^2 (M (1+s) - a^2 x),                                         */
/*   C   = s - (m + s cos)^2/sin^2 - 2(s+1) M x + 2a^2 x^2 - 2imax.          */
/* The principal symbol's discriminant is A^tr^2 - 4 A^rr A^tt               */
/* = 4 W^4 Sigma^2, so the roots of b^2 + (A^tr/D) b - A^rr/D = 0 are        */
/*   b = W^2 Delta / E = rho^2 delta / E  (outgoing, 0 on the horizon),      */
/*   -c, c = W^2 E / D                    (ingoing, 0 at scri).              */
/* First-order form with pi = Phi_tau + b Phi_rho:                           */
/*   Phi_tau = pi - b Phi_rho,                                               */
/*   pi_tau  = c pi_rho + K Phi_rho + Phi_thth/D + cot Phi_th/D              */
/*             + (B^t/D) pi + (C/D) Phi,  K = B^r/D - b B^t/D - c b_rho.     */
/* b_rho by the complex-step derivative (Squire and Trapp 1998):             */
/* b_rho = Im b(rho + i h)/h, exact to rounding for analytic b.              */
/* out = {b, Re K, Im K, Re Bt, Im Bt, Re C, Im C, Ath, Bth, c} with         */
/* Bt = B^t/D, C = C/D, Ath = 1/D, Bth = cot/D.                              */
/* ------------------------------------------------------------------------ */
double orc_rho_of_r(double r, double S) { return r / (1.0 + r / S); }

static double complex hyp_b(double complex rho, double sn2, double M, double a,
                            double S) {
    double complex x = 1.0 / rho - 1.0 / S;
    double complex W = 1.0 - rho / S;
    double complex delta = 1.0 - 2.0 * M * x + a * a * x * x;
    double complex w = 1.0 + a * a * x * x;
    double complex sig = csqrt(w * w - a * a * x * x * delta * sn2);
    double complex G = rho * (rho + 4.0 * M + 8.0 * M * M / S - 2.0 * M * W
                              + a * a * x * (W - 4.0 * M / S));
    double complex E = G - a * a * delta * sn2 / (sig + w);
    return rho * rho * delta / E;
}

void orc_coeff_point_hyp(double rho, double th, double M, double a, double S,
                         int s, int m, double out[10]) {
    double sn = sin(th), cs = cos(th), sn2 = sn * sn;
    double x = 1.0 / rho - 1.0 / S;
    double W = 1.0 - rho / S;
    double delta = 1.0 - 2.0 * M * x + a * a * x * x;
    double w = 1.0 + a * a * x * x;
    double sig = sqrt(w * w - a * a * x * x * delta * sn2);
    double Hp = 2.0 - W * W + 4.0 * M * W / S;
    double G = rho * (rho + 4.0 * M + 8.0 * M * M / S - 2.0 * M * W
                      + a * a * x * (W - 4.0 * M / S));
    double E = G - a * a * delta * sn2 / (sig + w);
    double D = Hp * G - a * a * sn2;

    double b = rho * rho * delta / E;
    double c = W * W * E / D;
    double hstep = 1e-30;
    double db = cimag(hyp_b(rho + I * hstep, sn2, M, a, S)) / hstep;

    double complex Bt = (2.0 * s * rho * (4.0 * M / S - W) - 2.0 * (1 + s) * M * Hp
                         + 2.0 * a * a * x * (Hp - 1.0)
                         - 2.0 * delta * rho * rho * (W - 2.0 * M / S) / S
                         + I * (2.0 * m * a * (1.0 - Hp) - 2.0 * s * a * cs)) / D;
    double complex Br = (2.0 * I * m * a * W * W
                         - 2.0 * W * rho * ((s + 1) - W - rho * x * (2.0 * M - a * a * x) / S)
                         + 2.0 * W * W * (M * (1 + s) - a * a * x)) / D;
    double mc = m + s * cs;
    double complex C = (s - mc * mc / sn2 - 2.0 * (s + 1) * M * x + 2.0 * a * a * x * x
                        - 2.0 * I * m * a * x) / D;
    double complex K = Br - b * Bt - c * db;

    out[0] = b;
    out[1] = creal(K);  out[2] = cimag(K);
    out[3] = creal(Bt); out[4] = cimag(Bt);
    out[5] = creal(C);  out[6] = cimag(C);
    out[7] = 1.0 / D;   out[8] = (cs / sn) / D;
    out[9] = c;
}

/* Grid (reading): x_i = x_min + i h, h = (x_max - x_min)/(nr-1), x = r* or  */
/* rho; theta_j = (j + 1/2) pi / nth (cell centred, never on a pole).       */
void orc_coefficients(const orc_grid* g, double* coef) {
    int nr = g->nr, nth = g->nth;
    double h = (g->rs_max - g->rs_min) / (nr - 1);
    long plane = (long)nr * nth;
    for (int i = 0; i < nr; ++i) {
        double x = g->rs_min + i * h;
        double xp = (g->coords == 1) ? 0.0 : orc_x_of_rstar(x, g->M, g->a);   /* r - r_+ */
        double r = horizon_r(g->M, g->a) + xp;
        for (int j = 0; j < nth; ++j) {
            double th = (j + 0.5) * M_PI / nth;
            double c[10];
            if (g->coords == 1)
                orc_coeff_point_hyp(x, th, g->M, g->a, g->S, g->s, g->m, c);
            else
                coeff_point_rx(r, xp, th, g->M, g->a, g->s, g->m, g->field, c);
            for (int k = 0; k < 10; ++k) coef[k * plane + (long)j * nr + i] = c[k];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Rounding to the weight format. A value is rounded to p significant bits  */
/* (round to nearest, ties to even), with the format's smallest normal       */
/* exponent emin fixing the subnormal spacing and overflow going to +-inf.   */
/* binary16: p = 11, emin = -14;  bfloat16: p = 8, emin = -126.              */
/* One arithmetic operation done in binary64 and then rounded this way is    */
/* the correctly rounded operation in the narrower format (53 >= 2p + 2).    */
/* ------------------------------------------------------------------------ */
static double round_to_format(double x, int p, int emin, double maxfinite) {
    if (x == 0.0 || !isfinite(x)) return x;
    int e2;
    frexp(x, &e2);                 /* |x| = f 2^e2, f in [0.5, 1) */
    int E = e2 - 1;                /* floor(log2 |x|) */
    if (E < emin) E = emin;        /* subnormal: fixed spacing 2^(emin-p+1) */
    double q = nearbyint(ldexp(x, p - 1 - E));   /* ties to even */
    double y = ldexp(q, E - (p - 1));
    if (fabs(y) > maxfinite) return copysign(INFINITY, x);
    return y;
}

double orc_round_w(int wprec, double x) {
    switch (wprec) {
    case 1: return (double)(float)x;
    case 2: return round_to_format(x, 11, -14, 65504.0);
    case 3: return round_to_format(x, 8, -126, ldexp(255.0, 120));
    default: return x;
    }
}

/* Range limits of the scaled epsilon (reading): eps_hat is clamped to       */
/* [tiny, huge] before rounding; both are powers of two.                     */
static void eps_range(int wprec, double* tiny, double* huge) {
    if (wprec == 2)      { *tiny = ldexp(1.0, -14);   *huge = ldexp(1.0, 15); }
    else if (wprec == 4) { *tiny = ldexp(1.0, -1022); *huge = ldexp(1.0, 1000); }
    else                 { *tiny = ldexp(1.0, -126);  *huge = ldexp(1.0, 100); }
}

/* ------------------------------------------------------------------------ */
/* WENO5 nonlinear weights (Sec. 3.1.2).                                     */
/* dir = +1: f5 = f_{j-2..j+2}, weights of the positive-direction flux at    */
/*           j+1/2; dir = -1: f5 = f_{j-1..j+3}, negative-direction flux.    */
/* w[k] = omega_k with the paper's indexing (omega^-_0 belongs to the        */
/* stencil f_{j+1}, f_{j+2}, f_{j+3}).                                       */
/* ------------------------------------------------------------------------ */
static const double D_LIN[3] = {0.1, 0.6, 0.3};

static void weights_fp64(int dir, const double* f, double eps, double w[3]) {
    double IS[3];
    if (dir > 0) {
        IS[0] = 13.0 / 12.0 * pow(f[0] - 2 * f[1] + f[2], 2)
              + 0.25 * pow(f[0] - 4 * f[1] + 3 * f[2], 2);
        IS[1] = 13.0 / 12.0 * pow(f[1] - 2 * f[2] + f[3], 2)
              + 0.25 * pow(f[1] - f[3], 2);
        IS[2] = 13.0 / 12.0 * pow(f[2] - 2 * f[3] + f[4], 2)
              + 0.25 * pow(3 * f[2] - 4 * f[3] + f[4], 2);
    } else {
        IS[0] = 13.0 / 12.0 * pow(f[2] - 2 * f[3] + f[4], 2)
              + 0.25 * pow(3 * f[2] - 4 * f[3] + f[4], 2);
        IS[1] = 13.0 / 12.0 * pow(f[1] - 2 * f[2] + f[3], 2)
              + 0.25 * pow(f[1] - f[3], 2);
        IS[2] = 13.0 / 12.0 * pow(f[0] - 2 * f[1] + f[2], 2)
              + 0.25 * pow(f[0] - 4 * f[1] + 3 * f[2], 2);
    }
    double alpha[3], sum = 0.0;
    for (int k = 0; k < 3; ++k) {
        alpha[k] = D_LIN[k] / pow(eps + IS[k], 2);
        sum += alpha[k];
    }
    for (int k = 0; k < 3; ++k) w[k] = alpha[k] / sum;
}

/* Reduced-precision weights (Sec. 3.1.3, reading above). The smoothness     */
/* indicators are the paper's, written with the stencil's first differences */
/* x: for dir = +1, x_k = f_{k+1} - f_k over f_{j-2..j+2}, and              */
/*   f_{j-2}-2f_{j-1}+f_j = x1-x0,   f_{j-2}-4f_{j-1}+3f_j = 3x1-x0,         */
/*   f_{j-1}-2f_j+f_{j+1} = x2-x1,   f_{j-1}-f_{j+1}      = -(x1+x2),        */
/*   f_j-2f_{j+1}+f_{j+2} = x3-x2,   3f_j-4f_{j+1}+f_{j+2} = x3-3x2.         */
/* For dir = -1 the same identities hold with the first differences taken   */
/* in reverse order (the negative-direction stencil is the mirror image).    */
static void weights_reduced(int wprec, int dir, const double* f, double eps,
                            double w[3]) {
    double x[4];
    for (int k = 0; k < 4; ++k) x[k] = f[k + 1] - f[k];      /* binary64 */
    if (dir < 0) {                                           /* mirror */
        double t0 = x[0], t1 = x[1];
        x[0] = x[3]; x[1] = x[2]; x[2] = t1; x[3] = t0;
    }
    double mx = 0.0;
    for (int k = 0; k < 4; ++k) mx = fmax(mx, fabs(x[k]));
    int e = 0;
    if (mx > 0.0) { int e2; frexp(mx, &e2); e = e2 - 1; }   /* 2^e <= mx < 2^(e+1) */

#define RW(v) orc_round_w(wprec, (v))
    double xh[4];
    for (int k = 0; k < 4; ++k) xh[k] = RW(ldexp(x[k], -e));
    double tiny, huge;
    eps_range(wprec, &tiny, &huge);
    double eh = ldexp(eps, -2 * e);
    if (eh < tiny) eh = tiny;
    if (eh > huge) eh = huge;
    eh = RW(eh);
    double c13 = RW(13.0 / 12.0), c14 = 0.25, d[3];
    for (int k = 0; k < 3; ++k) d[k] = RW(D_LIN[k]);

    double a, b, IS[3];
    a = RW(xh[1] - xh[0]);             b = RW(RW(3.0 * xh[1]) - xh[0]);
    IS[0] = RW(RW(c13 * RW(a * a)) + RW(c14 * RW(b * b)));
    a = RW(xh[2] - xh[1]);             b = RW(xh[1] + xh[2]);
    IS[1] = RW(RW(c13 * RW(a * a)) + RW(c14 * RW(b * b)));
    a = RW(xh[3] - xh[2]);             b = RW(RW(3.0 * xh[2]) - xh[3]);
    IS[2] = RW(RW(c13 * RW(a * a)) + RW(c14 * RW(b * b)));

    double t[3], tmin, alpha[3];
    for (int k = 0; k < 3; ++k) t[k] = RW(eh + IS[k]);
    tmin = fmin(t[0], fmin(t[1], t[2]));
    for (int k = 0; k < 3; ++k) {
        double rk = RW(tmin / t[k]);
        alpha[k] = RW(d[k] * RW(rk * rk));
    }
    double sum = RW(RW(alpha[0] + alpha[1]) + alpha[2]);
    for (int k = 0; k < 3; ++k) w[k] = RW(alpha[k] / sum);
#undef RW
}

void orc_weno5_weights(int wprec, int dir, const double* f5, double eps,
                       double w[3]) {
    if (wprec == 0) weights_fp64(dir, f5, eps, w);
    else weights_reduced(wprec, dir, f5, eps, w);
}

/* Numerical flux at j+1/2 from the candidate stencils (Sec. 3.1.2). With    */
/* reduced weights, omega_1 = 1 - omega_0 - omega_2 in binary64 so that the  */
/* weights sum to one in the high precision (Sec. 3.1.3).                    */
double orc_weno5_flux(int wprec, int dir, const double* f, double eps,
                      const double* force_w, double w_out[3], double q_out[3]) {
    double w[3], q[3];
    if (force_w) { w[0] = force_w[0]; w[1] = force_w[1]; w[2] = force_w[2]; }
    else orc_weno5_weights(wprec, dir, f, eps, w);
    if (!force_w && wprec != 0) w[1] = 1.0 - w[0] - w[2];
    if (dir > 0) {
        q[0] = (2.0 * f[0] - 7.0 * f[1] + 11.0 * f[2]) / 6.0;
        q[1] = (-f[1] + 5.0 * f[2] + 2.0 * f[3]) / 6.0;
        q[2] = (2.0 * f[2] + 5.0 * f[3] - f[4]) / 6.0;
    } else {
        q[2] = (-f[0] + 5.0 * f[1] + 2.0 * f[2]) / 6.0;
        q[1] = (2.0 * f[1] + 5.0 * f[2] - f[3]) / 6.0;
        q[0] = (11.0 * f[2] - 7.0 * f[3] + 2.0 * f[4]) / 6.0;
    }
    if (w_out) { w_out[0] = w[0]; w_out[1] = w[1]; w_out[2] = w[2]; }
    if (q_out) { q_out[0] = q[0]; q_out[1] = q[1]; q_out[2] = q[2]; }
    return w[0] * q[0] + w[1] * q[1] + w[2] * q[2];
}

/* Ghost value at index k outside 0..n-1 by Lagrange extrapolation of the  */
/* degree-q polynomial through the q+1 nearest edge nodes:                   */
/*   p(k) = sum_j f_j prod_{l != j} (k - x_l)/(x_j - x_l).                   */
/* The hyperboloidal grid uses q = 4 (reading: both of its ends are outflow  */
/* boundaries, which need no data; among degrees 0..4 the quartic gave the   */
/* fastest convergence of the horizon value under grid refinement).          */
#define EXTRAP_DEG 4
static double extrap_ghost(const double* f, int n, int k, int q) {
    int x0 = (k < 0) ? 0 : n - 1 - q;          /* nodes x0 .. x0+q */
    double v = 0.0;
    for (int j = x0; j <= x0 + q; ++j) {
        double L = 1.0;
        for (int l = x0; l <= x0 + q; ++l)
            if (l != j) L *= (double)(k - l) / (double)(j - l);
        v += L * f[j];
    }
    return v;
}

/* Derivative of one line, D_i = (fhat_{i+1/2} - fhat_{i-1/2}) / h           */
/* (Sec. 3.1.2). Ghosts (bc): 0 copies of the edge value, 1 periodic wrap,   */
/* 2 polynomial extrapolation (extrap_ghost).                                */
/* w_out / q_out (optional, 3 per interface) receive the weights and          */
/* candidate values of interface i+1/2 for i = 0..n-1.                       */
void orc_weno5_deriv_1d(const double* f, int n, double h, int dir, int wprec,
                        double eps, int bc, const double* force_w,
                        double* D, double* w_out, double* q_out) {
    double* ext = (double*)malloc(sizeof(double) * (n + 6));
    double* fh = (double*)malloc(sizeof(double) * (n + 1));
    for (int k = -3; k < n + 3; ++k) {
        if (k >= 0 && k < n) ext[k + 3] = f[k];
        else if (bc == 1) ext[k + 3] = f[((k % n) + n) % n];
        else if (bc == 2) ext[k + 3] = extrap_ghost(f, n, k, EXTRAP_DEG);
        else ext[k + 3] = f[k < 0 ? 0 : n - 1];
    }
    /* interface i+1/2 for i = -1 .. n-1, stored at fh[i+1] */
    for (int i = -1; i < n; ++i) {
        const double* st = (dir > 0) ? &ext[i - 2 + 3] : &ext[i - 1 + 3];
        double wl[3], ql[3];
        fh[i + 1] = orc_weno5_flux(wprec, dir, st, eps, force_w, wl, ql);
        if (i >= 0 && w_out) for (int k = 0; k < 3; ++k) w_out[3 * i + k] = wl[k];
        if (i >= 0 && q_out) for (int k = 0; k < 3; ++k) q_out[3 * i + k] = ql[k];
    }
    for (int i = 0; i < n; ++i) D[i] = (fh[i + 1] - fh[i]) / h;
    free(ext);
    free(fh);
}

/* ------------------------------------------------------------------------ */
/* Comparison scheme of Sec. 3.1.1: the sixth-order centred derivative        */
/*   D_j = (u_{j+3} - 9u_{j+2} + 45u_{j+1} - 45u_{j-1} + 9u_{j-2} - u_{j-3})     */
/*         / (60 h)                                                          */
/* and the Kreiss-Oliger operator Q = sigma h^7 D+^4 D-^4 / 256 with          */
/* D+ u_j = (u_{j+1} - u_j)/h, D- u_j = (u_j - u_{j-1})/h, applied here       */
/* literally (nested differences). Ghosts (bc): 0 edge copies, 1 periodic    */
/* wrap, 2 polynomial extrapolation (extrap_ghost).                          */
/* ------------------------------------------------------------------------ */
void orc_fd6_ko8_1d(const double* f, int n, double h, double sigma, int bc,
                    double* D, double* Q) {
    const int G = 4;                                  /* ghost width */
    int m = n + 2 * G;
    double* a = (double*)malloc(sizeof(double) * m);
    double* b = (double*)malloc(sizeof(double) * m);
    for (int k = -G; k < n + G; ++k) {
        if (k >= 0 && k < n) a[k + G] = f[k];
        else if (bc == 1) a[k + G] = f[((k % n) + n) % n];
        else if (bc == 2) a[k + G] = extrap_ghost(f, n, k, EXTRAP_DEG);
        else a[k + G] = f[k < 0 ? 0 : n - 1];
    }
    for (int j = 0; j < n; ++j) {
        const double* u = &a[j + G];
        D[j] = (u[3] - 9.0 * u[2] + 45.0 * u[1] - 45.0 * u[-1] + 9.0 * u[-2] - u[-3])
               / (60.0 * h);
    }
    /* D-^4 then D+^4 on the extended line (each application valid on a
     * shrinking range; the centre j = 0..n-1 stays valid after all eight) */
    memcpy(b, a, sizeof(double) * m);
    for (int r = 0; r < 4; ++r)
        for (int k = m - 1; k >= 1; --k) b[k] = (b[k] - b[k - 1]) / h;    /* D- */
    for (int r = 0; r < 4; ++r)
        for (int k = 0; k < m - 1; ++k) b[k] = (b[k + 1] - b[k]) / h;    /* D+ */
    for (int j = 0; j < n; ++j) Q[j] = sigma * pow(h, 7) * b[j + G] / 256.0;
    free(a);
    free(b);
}

/* ------------------------------------------------------------------------ */
/* Right-hand side F(u) of du/dt = F(u) = -(M du/dr* + L u + A u)            */
/* (Eq. evln). Psi components take the positive-direction WENO flux, pi      */
/* components the negative-direction one, by the sign of M's diagonal        */
/* (Sec. 3.1.2); m31, m32 use the same Psi derivative. theta derivatives are */
/* fourth-order centred with parity ghosts. Complex form:                    */
/*   F_Psi = pi - b D_Psi,                                                   */
/*   F_pi  = c D_pi + K D_Psi + Ath Psi_thth + Bth Psi_th + Bt pi + C Psi    */
/* (c = b in r*).                                                            */
/* ------------------------------------------------------------------------ */
void orc_rhs(const orc_grid* g, const double* coef, const double* u, double* F) {
    int nr = g->nr, nth = g->nth;
    long plane = (long)nr * nth;
    double h = (g->rs_max - g->rs_min) / (nr - 1);
    double dth = M_PI / nth;
    double sigma = ((g->m + g->s) % 2 == 0) ? 1.0 : -1.0;

#pragma omp parallel for schedule(static)
    for (int j = 0; j < nth; ++j) {
        double* Dc = (double*)malloc(sizeof(double) * 4 * nr);
        double* Qc = (double*)calloc(4 * (size_t)nr, sizeof(double));
        for (int c = 0; c < 4; ++c) {
            if (g->scheme == 1) {
                orc_fd6_ko8_1d(&u[c * plane + (long)j * nr], nr, h, g->ko_sigma,
                               g->coords == 1 ? 2 : 0, &Dc[c * nr], &Qc[c * nr]);
            } else {
                int dir = (c < 2) ? +1 : -1;
                orc_weno5_deriv_1d(&u[c * plane + (long)j * nr], nr, h, dir, g->wprec,
                                   g->eps, g->coords == 1 ? 2 : 0, NULL, &Dc[c * nr],
                                   NULL, NULL);
            }
        }
        /* rows j-2 .. j+2 of Psi, with ghosts across the poles */
        int rows[5];
        double sgn[5];
        for (int k = -2; k <= 2; ++k) {
            int jj = j + k;
            double sg = 1.0;
            if (jj < 0) { jj = -1 - jj; sg = sigma; }
            if (jj >= nth) { jj = 2 * nth - 1 - jj; sg = sigma; }
            rows[k + 2] = jj;
            sgn[k + 2] = sg;
        }
        for (int i = 0; i < nr; ++i) {
            long p = (long)j * nr + i;
            double complex psi = u[0 * plane + p] + I * u[1 * plane + p];
            double complex pi = u[2 * plane + p] + I * u[3 * plane + p];
            double complex Dpsi = Dc[0 * nr + i] + I * Dc[1 * nr + i];
            double complex Dpi = Dc[2 * nr + i] + I * Dc[3 * nr + i];
            double complex nb[5];
            for (int k = 0; k < 5; ++k) {
                long q = (long)rows[k] * nr + i;
                nb[k] = sgn[k] * (u[0 * plane + q] + I * u[1 * plane + q]);
            }
            double complex psi_th = (nb[0] - 8.0 * nb[1] + 8.0 * nb[3] - nb[4])
                                    / (12.0 * dth);
            if (g->theta_mode == 1) {
                /* WENO5 along theta: rows j-3 .. j+3 with parity ghosts */
                double line[2][7];
                for (int k = -3; k <= 3; ++k) {
                    int jj = j + k;
                    double sg = 1.0;
                    if (jj < 0) { jj = -1 - jj; sg = sigma; }
                    if (jj >= nth) { jj = 2 * nth - 1 - jj; sg = sigma; }
                    long q = (long)jj * nr + i;
                    line[0][k + 3] = sg * u[0 * plane + q];
                    line[1][k + 3] = sg * u[1 * plane + q];
                }
                double Bth_here = coef[8 * plane + p];
                int dir = (-Bth_here < 0.0) ? -1 : +1;
                double d[2];
                for (int c = 0; c < 2; ++c) {
                    /* interfaces j+1/2 and j-1/2 */
                    const double* sp = (dir > 0) ? &line[c][1] : &line[c][2];
                    const double* sm = (dir > 0) ? &line[c][0] : &line[c][1];
                    double fp = orc_weno5_flux(g->wprec, dir, sp, g->eps, NULL, NULL, NULL);
                    double fm = orc_weno5_flux(g->wprec, dir, sm, g->eps, NULL, NULL, NULL);
                    d[c] = (fp - fm) / dth;
                }
                psi_th = d[0] + I * d[1];
            }
            double complex psi_thth = (-nb[0] + 16.0 * nb[1] - 30.0 * nb[2]
                                       + 16.0 * nb[3] - nb[4]) / (12.0 * dth * dth);
            double b = coef[0 * plane + p];
            double complex K = coef[1 * plane + p] + I * coef[2 * plane + p];
            double complex Bt = coef[3 * plane + p] + I * coef[4 * plane + p];
            double complex C = coef[5 * plane + p] + I * coef[6 * plane + p];
            double Ath = coef[7 * plane + p], Bth = coef[8 * plane + p];
            double cpi = coef[9 * plane + p];

            double complex Fpsi = pi - b * Dpsi;
            double complex Fpi = cpi * Dpi + K * Dpsi + Ath * psi_thth
                                 + Bth * psi_th + Bt * pi + C * psi;
            /* scheme 1: the Kreiss-Oliger term is subtracted (dissipative sign) */
            F[0 * plane + p] = creal(Fpsi) - Qc[0 * nr + i];
            F[1 * plane + p] = cimag(Fpsi) - Qc[1 * nr + i];
            F[2 * plane + p] = creal(Fpi) - Qc[2 * nr + i];
            F[3 * plane + p] = cimag(Fpi) - Qc[3 * nr + i];
        }
        free(Dc);
        free(Qc);
    }
}

/* ------------------------------------------------------------------------ */
/* SSP-RK(3,3) in Shu-Osher form (Sec. 3.2):                                 */
/*   u1 = u + dt F(u); u2 = 3/4 u + 1/4 (u1 + dt F(u1));                     */
/*   u^{n+1} = 1/3 u + 2/3 (u2 + dt F(u2)).                                  */
/* One routine serves the PDE and the scalar test equation.                  */
/* ------------------------------------------------------------------------ */
typedef void (*rhs_fn)(const void* ctx, const double* u, double* F);

static void ssprk3(long n, double* u, double dt, long nsteps, rhs_fn rhs,
                   const void* ctx) {
    double* u1 = (double*)malloc(sizeof(double) * n);
    double* u2 = (double*)malloc(sizeof(double) * n);
    double* Fv = (double*)malloc(sizeof(double) * n);
    for (long step = 0; step < nsteps; ++step) {
        rhs(ctx, u, Fv);
        for (long k = 0; k < n; ++k) u1[k] = u[k] + dt * Fv[k];
        rhs(ctx, u1, Fv);
        for (long k = 0; k < n; ++k)
            u2[k] = 0.75 * u[k] + 0.25 * (u1[k] + dt * Fv[k]);
        rhs(ctx, u2, Fv);
        for (long k = 0; k < n; ++k)
            u[k] = u[k] / 3.0 + 2.0 / 3.0 * (u2[k] + dt * Fv[k]);
    }
    free(u1);
    free(u2);
    free(Fv);
}

typedef struct { const orc_grid* g; const double* coef; } pde_ctx;

static void pde_rhs(const void* ctx, const double* u, double* F) {
    const pde_ctx* c = (const pde_ctx*)ctx;
    orc_rhs(c->g, c->coef, u, F);
}

void orc_rk3_step(const orc_grid* g, const double* coef, double dt, double* u,
                  long nsteps) {
    pde_ctx c = {g, coef};
    ssprk3(4L * g->nr * g->nth, u, dt, nsteps, pde_rhs, &c);
}

/* ------------------------------------------------------------------------ */
/* SSP-RK(10,4), low-storage ten-stage fourth-order method as printed in     */
/* Sec. 3.2 (Shu-Osher form):                                                */
/*   u1 = u + dt/6 F(u); u_i = u_{i-1} + dt/6 F(u_{i-1}), i = 2..4;           */
/*   u5 = 3/5 u + 2/5 u4 + dt/15 F(u4);                                      */
/*   u_i = u_{i-1} + dt/6 F(u_{i-1}), i = 6..9;                              */
/*   u^{n+1} = u/25 + 9/25 u4 + 3/5 u9 + 3/50 dt F(u4) + dt/10 F(u9).        */
/* ------------------------------------------------------------------------ */
static void ssprk104(long n, double* u, double dt, long nsteps, rhs_fn rhs,
                     const void* ctx) {
    double* ui = (double*)malloc(sizeof(double) * n);
    double* u4 = (double*)malloc(sizeof(double) * n);
    double* F4 = (double*)malloc(sizeof(double) * n);
    double* Fv = (double*)malloc(sizeof(double) * n);
    for (long step = 0; step < nsteps; ++step) {
        memcpy(ui, u, sizeof(double) * n);
        for (int i = 1; i <= 4; ++i) {
            rhs(ctx, ui, Fv);
            for (long k = 0; k < n; ++k) ui[k] = ui[k] + dt / 6.0 * Fv[k];
        }
        memcpy(u4, ui, sizeof(double) * n);
        rhs(ctx, u4, F4);
        for (long k = 0; k < n; ++k)
            ui[k] = 3.0 / 5.0 * u[k] + 2.0 / 5.0 * u4[k] + dt / 15.0 * F4[k];
        for (int i = 6; i <= 9; ++i) {
            rhs(ctx, ui, Fv);
            for (long k = 0; k < n; ++k) ui[k] = ui[k] + dt / 6.0 * Fv[k];
        }
        rhs(ctx, ui, Fv);
        for (long k = 0; k < n; ++k)
            u[k] = u[k] / 25.0 + 9.0 / 25.0 * u4[k] + 3.0 / 5.0 * ui[k]
                 + 3.0 / 50.0 * dt * F4[k] + dt / 10.0 * Fv[k];
    }
    free(ui);
    free(u4);
    free(F4);
    free(Fv);
}

void orc_rk104_step(const orc_grid* g, const double* coef, double dt, double* u,
                    long nsteps) {
    pde_ctx c = {g, coef};
    ssprk104(4L * g->nr * g->nth, u, dt, nsteps, pde_rhs, &c);
}

typedef struct { double lr, li; } lin_ctx;

static void lin_rhs(const void* ctx, const double* y, double* F) {
    const lin_ctx* c = (const lin_ctx*)ctx;
    F[0] = c->lr * y[0] - c->li * y[1];
    F[1] = c->lr * y[1] + c->li * y[0];
}

/* y' = lambda y for complex lambda; y = {Re, Im}. */
void orc_rk3_linear(double lam_re, double lam_im, double dt, long nsteps,
                    double y[2]) {
    lin_ctx c = {lam_re, lam_im};
    ssprk3(2, y, dt, nsteps, lin_rhs, &c);
}

void orc_rk104_linear(double lam_re, double lam_im, double dt, long nsteps,
                      double y[2]) {
    lin_ctx c = {lam_re, lam_im};
    ssprk104(2, y, dt, nsteps, lin_rhs, &c);
}

typedef struct { int n, dir, wprec; double h, eps; } adv_ctx;

static void adv_rhs(const void* ctx, const double* u, double* F) {
    const adv_ctx* c = (const adv_ctx*)ctx;
    orc_weno5_deriv_1d(u, c->n, c->h, c->dir, c->wprec, c->eps, 1, NULL, F,
                       NULL, NULL);
    for (int i = 0; i < c->n; ++i) F[i] = -(double)c->dir * F[i];
}

/* Periodic linear advection u_t + dir u_x = 0 with the dir-upwinded flux.   */
void orc_advect_1d(double* f, int n, double h, double dt, long nsteps, int dir,
                   int wprec, double eps) {
    adv_ctx c = {n, dir, wprec, h, eps};
    ssprk3(n, f, dt, nsteps, adv_rhs, &c);
}

/* ------------------------------------------------------------------------ */
/* Observation (Sec. 4): Psi along theta at the r* node nearest rs_ext, and  */
/* at the innermost node Psi, pi and dPsi/dr* (one-sided second order).      */
/* wave[2j+{0,1}] = Psi; horizon[6j + {0..5}] = Psi, pi, Psi_*.              */
/* ------------------------------------------------------------------------ */
void orc_observe(const orc_grid* g, const double* u, double rs_ext, double* wave,
                 double* horizon) {
    int nr = g->nr, nth = g->nth;
    long plane = (long)nr * nth;
    double h = (g->rs_max - g->rs_min) / (nr - 1);
    long ie = lround((rs_ext - g->rs_min) / h);
    if (ie < 0) ie = 0;
    if (ie > nr - 1) ie = nr - 1;
    for (int j = 0; j < nth; ++j) {
        long row = (long)j * nr;
        wave[2 * j] = u[0 * plane + row + ie];
        wave[2 * j + 1] = u[1 * plane + row + ie];
        for (int c = 0; c < 4; ++c) horizon[6 * j + c] = u[c * plane + row];
        for (int c = 0; c < 2; ++c) {
            const double* f = &u[c * plane + row];
            horizon[6 * j + 4 + c] = (-3.0 * f[0] + 4.0 * f[1] - f[2]) / (2.0 * h);
        }
    }
}
