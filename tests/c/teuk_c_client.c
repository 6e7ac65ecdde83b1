/*
 * A plain C client of the C ABI (include/teuk.h), built and run by
 * tests/test_host_abi.py (host-side calls, no GPU) and tests/test_gpu_parity.py
 * (the "gpu" mode). It uses nothing but the header's declarations: parameters
 * for the 2048 x 128 Kerr workload, the stability rule and the coefficient
 * array; the same on the hyperboloidal slices, whose range [0, 0] stands for
 * the whole slice from the horizon to scri (the client never computes rho_+);
 * with "gpu", a handle with the seeded Gaussian initial data, 40 steps
 * (graph replay plus direct launches), the observation at r* = 50 M and on the
 * innermost node, a checkpoint round trip, and a hyperboloidal handle observed
 * on the horizon and at scri.
 *
 * Output: "key value" lines read by the tests. Exit status 0 on success.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "teuk.h"

#define CHECK(call)                                                              \
    do {                                                                         \
        teuk_status st_ = (call);                                                \
        if (st_ != TEUK_OK) {                                                    \
            fprintf(stderr, "%s failed: %s (%s)\n", #call, teuk_status_str(st_), \
                    teuk_last_error());                                          \
            return 2;                                                            \
        }                                                                        \
    } while (0)

static teuk_params kerr_params(void) {
    teuk_params p;
    memset(&p, 0, sizeof p);
    p.nr = 2048;
    p.ntheta = 128;
    p.rstar_min = -100.0;
    p.rstar_max = 300.0;
    p.M = 1.0;
    p.a = 0.999;
    p.s = -2;
    p.m = 2;
    p.cfl = 0.5;
    p.dt = 0.0;
    p.eps = 1e-6;
    p.wprec = TEUK_W_FP32;
    p.theta_mode = TEUK_THETA_CENTERED4;
    p.rk = TEUK_RK_SSP33;
    p.scheme = TEUK_SCHEME_WENO5;
    p.ko_sigma = 0.01;
    p.coords = TEUK_COORDS_RSTAR;
    p.field = TEUK_FIELD_PSI;
    p.hyp_S = 20.0;
    return p;
}

/* The paper's extremal run on the hyperboloidal slices (Sec. 4), reduced to
 * 512 x 16 nodes; range [0, 0]: the library takes [rho_+, S]. */
static teuk_params hyp_params(void) {
    teuk_params p = kerr_params();
    p.nr = 512;
    p.ntheta = 16;
    p.rstar_min = 0.0;
    p.rstar_max = 0.0;
    p.a = 1.0;
    p.m = 0;
    p.coords = TEUK_COORDS_HYPERBOLOIDAL;
    p.field = TEUK_FIELD_PHI;
    return p;
}

static int host_mode(void) {
    teuk_params p = kerr_params();
    CHECK(teuk_check_params(&p));
    double dt = 0.0;
    CHECK(teuk_stable_dt(&p, &dt));
    size_t n = teuk_coeff_count(&p);
    double* coef = (double*)malloc(n * sizeof(double));
    if (!coef) return 3;
    CHECK(teuk_build_coefficients(&p, dt, coef));
    double sum = 0.0;
    for (size_t k = 0; k < n; ++k) sum += fabs(coef[k]);
    free(coef);
    printf("dt %.17g\n", dt);
    printf("coef_count %zu\n", n);
    printf("coef_abs_sum %.17g\n", sum);
    /* an invalid parameter set is reported, not fatal */
    teuk_params bad = p;
    bad.nr = 3;
    teuk_status st = teuk_check_params(&bad);
    printf("bad_status %d\n", (int)st);
    printf("bad_message_nonempty %d\n", teuk_last_error()[0] != '\0');
    /* the whole hyperboloidal slice without computing rho_+ here */
    teuk_params q = hyp_params();
    CHECK(teuk_check_params(&q));
    double dth = 0.0, rhop = 0.0;
    CHECK(teuk_stable_dt(&q, &dth));
    CHECK(teuk_horizon_rho(q.M, q.a, q.hyp_S, &rhop));
    printf("hyp_dt %.17g\n", dth);
    printf("horizon_rho %.17g\n", rhop);
    return 0;
}

static int gpu_mode(void) {
    teuk_params p = kerr_params();
    teuk_handle* h = NULL;
    CHECK(teuk_create(&p, NULL, &h));
    const double coeffs[2] = {1.0, 0.5};                /* one l = 2 term */
    CHECK(teuk_set_gaussian(h, 30.0, 3.0, coeffs, 1, 0));
    CHECK(teuk_step(h, 40));
    double* wave = (double*)malloc(2 * (size_t)p.ntheta * sizeof(double));
    double* hor = (double*)malloc(6 * (size_t)p.ntheta * sizeof(double));
    double t = 0.0;
    CHECK(teuk_observe(h, 50.0, wave, hor, &t));
    double wsum = 0.0;
    for (int k = 0; k < 2 * p.ntheta; ++k) wsum += fabs(wave[k]);
    printf("t %.17g\n", t);
    printf("wave_abs_sum %.17g\n", wsum);
    /* checkpoint round trip: save, step 5, restore, step 5 -> same bits */
    size_t n = 4 * (size_t)p.nr * p.ntheta;
    double* u0 = (double*)malloc(n * sizeof(double));
    double* u1 = (double*)malloc(n * sizeof(double));
    double* u2 = (double*)malloc(n * sizeof(double));
    double t0 = 0.0, t1 = 0.0;
    CHECK(teuk_get_state(h, u0, &t0));
    CHECK(teuk_step(h, 5));
    CHECK(teuk_get_state(h, u1, &t1));
    CHECK(teuk_set_state(h, u0, t0));
    CHECK(teuk_step(h, 5));
    CHECK(teuk_get_state(h, u2, NULL));
    printf("restart_bitwise %d\n", memcmp(u1, u2, n * sizeof(double)) == 0);
    CHECK(teuk_check_finite(h));
    /* the C ABI reports a bad call through its status */
    printf("neg_steps_status %d\n", (int)teuk_step(h, -1));
    CHECK(teuk_destroy(h));
    /* a handle on the whole hyperboloidal slice: the library fills the range */
    teuk_params q = hyp_params();
    teuk_handle* hh = NULL;
    CHECK(teuk_create(&q, NULL, &hh));
    teuk_params got;
    CHECK(teuk_get_info(hh, &got, NULL, NULL));
    printf("hyp_range %.17g %.17g\n", got.rstar_min, got.rstar_max);
    const double c1[2] = {1.0, 0.0};
    CHECK(teuk_set_gaussian(hh, 1.0, 0.22, c1, 1, 0));
    CHECK(teuk_step(hh, 20));
    double* hw = (double*)malloc(2 * (size_t)q.ntheta * sizeof(double));
    double* hh6 = (double*)malloc(6 * (size_t)q.ntheta * sizeof(double));
    CHECK(teuk_observe(hh, got.rstar_max, hw, hh6, NULL));
    double hsum = 0.0;
    for (int k = 0; k < 6 * q.ntheta; ++k) hsum += fabs(hh6[k]);
    printf("hyp_horizon_abs_sum %.17g\n", hsum);
    CHECK(teuk_destroy(hh));
    free(hw);
    free(hh6);
    free(wave);
    free(hor);
    free(u0);
    free(u1);
    free(u2);
    return 0;
}

int main(int argc, char** argv) {
    if (argc > 1 && strcmp(argv[1], "gpu") == 0) return gpu_mode();
    return host_mode();
}
