// Host side of the library: parameter validation, the Kerr coefficient
// generator, the time-step rule and error reporting. binary64 throughout.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "teuk_internal.h"

namespace teuk {

static thread_local std::string g_last_error;

teuk_status fail(teuk_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}
void clear_error() { g_last_error.clear(); }

// Tortoise coordinate (Sec. 2.2): dr*/dr = (r^2+a^2)/Delta. The unknown is
// y = ln(r - r_+), so the horizon region (r* -> -infinity) stays resolved and
// Delta = x (x + r_+ - r_-) is formed without cancellation (x = r - r_+).
// Integration constant: r* -> r + 2M ln(r/2M - 1) at a = 0.
namespace {
struct Tortoise {
    double M, a, rp, w, kp, km;
    bool extremal;
    Tortoise(double M_, double a_) : M(M_), a(std::fabs(a_)) {
        extremal = !(a < M);
        double d = extremal ? 0.0 : std::sqrt(M * M - a * a);
        rp = M + d;
        w = 2.0 * d;
        kp = extremal ? 0.0 : 2.0 * M * rp / w;
        km = extremal ? 0.0 : 2.0 * M * (M - d) / w;
    }
    // r*(y) - target and its y-derivative (x dr*/dr = varpi / (x + w) > 0).
    void eval(double y, double target, double* g, double* dg) const {
        double x = std::exp(y);
        double r = rp + x;
        double rs;
        if (extremal) {
            rs = r + 2.0 * M * (y - std::log(M)) - 2.0 * M * M / x;
        } else {
            rs = r + kp * (y - std::log(2.0 * M)) - km * std::log((x + w) / (2.0 * M));
        }
        *g = rs - target;
        *dg = (r * r + a * a) / (x + w);
    }
};
}  // namespace

double r_of_rstar(double rstar, double M, double a, double* x_out) {
    Tortoise T(M, a);
    // bracket y, then safeguarded Newton
    double ylo = -5.0, yhi = 5.0, g, dg;
    T.eval(ylo, rstar, &g, &dg);
    while (g > 0.0 && ylo > -740.0) { ylo -= 8.0; T.eval(ylo, rstar, &g, &dg); }
    T.eval(yhi, rstar, &g, &dg);
    while (g < 0.0 && yhi < 700.0) { yhi += 4.0; T.eval(yhi, rstar, &g, &dg); }
    double y = 0.5 * (ylo + yhi);
    for (int it = 0; it < 200; ++it) {
        T.eval(y, rstar, &g, &dg);
        if (g > 0.0) yhi = y; else ylo = y;
        double yn = y - g / dg;
        if (!(yn > ylo && yn < yhi)) yn = 0.5 * (ylo + yhi);
        if (std::fabs(yn - y) <= 1e-16 * std::fmax(1.0, std::fabs(y))) { y = yn; break; }
        y = yn;
    }
    double x = std::exp(y);
    if (x_out) *x_out = x;
    return T.rp + x;
}

// Continuum coefficients of the first-order form at (r*, theta). With
// Psi = exp(i m phi~) psi and pi = psi_t + b psi_* (Sec. 2.3):
//   psi_t = pi - b psi_*
//   pi_t  = b pi_* + K psi_* + Ath psi_thth + Bth psi_th + Bt pi + C psi
// where, from Eq. teuk0 divided by Sigma^2/Delta,
//   b = varpi/Sigma,  K = B* - b b_* - b Bt,  b_* = (Delta/varpi) db/dr,
//   B* = [2 r Delta + 2 s (r-M) varpi + 2 i m a varpi]/Sigma^2,
//   Bt = [-2 s (r Delta - M (r^2-a^2)) - i (4 M a m r + 2 s a Delta cos)]/Sigma^2,
//   C  = [Delta (s - (m + s cos)^2/sin^2) + 4 i s m a (r-M)]/Sigma^2,
//   Ath = Delta/Sigma^2, Bth = Delta cot/Sigma^2.
PointCoef point_coefficients(double rstar, double theta, const teuk_params& p) {
    double x;
    const double r = r_of_rstar(rstar, p.M, p.a, &x);
    return point_coefficients_rx(r, x, theta, p);
}

PointCoef point_coefficients_rx(double r, double x, double theta, const teuk_params& p) {
    const double M = p.M, a = p.a, s = p.s, m = p.m;
    Tortoise T(M, a);
    const double Delta = x * (x + T.w);
    const double varpi = r * r + a * a;
    const double sn = std::sin(theta), cs = std::cos(theta);
    const double S2 = varpi * varpi - a * a * Delta * sn * sn;
    const double inv = 1.0 / S2;
    const double b = varpi / std::sqrt(S2);
    // d ln b / dr = 2r/varpi - (dSigma^2/dr) / (2 Sigma^2)
    const double dS2 = 4.0 * r * varpi - 2.0 * a * a * (r - M) * sn * sn;
    const double bstar = (Delta / varpi) * b * (2.0 * r / varpi - 0.5 * dS2 * inv);
    PointCoef c;
    c.b = b;
    const double Bs_r = (2.0 * r * Delta + 2.0 * s * (r - M) * varpi) * inv;
    const double Bs_i = (2.0 * m * a * varpi) * inv;
    c.Btr = (-2.0 * s * (r * Delta - M * (r * r - a * a))) * inv;
    c.Bti = -(4.0 * M * a * m * r + 2.0 * s * a * Delta * cs) * inv;
    const double mc = m + s * cs;
    c.Cr = Delta * (s - mc * mc / (sn * sn)) * inv;
    c.Ci = 4.0 * s * m * a * (r - M) * inv;
    c.Kr = Bs_r - b * bstar - b * c.Btr;
    c.Ki = Bs_i - b * c.Bti;
    c.Ath = Delta * inv;
    c.Bth = Delta * (cs / sn) * inv;
    return c;
}

// Spin-weighted spherical harmonic sY_lm(theta, phi = 0), Goldberg et al.
// (1967): (-1)^m sqrt[(l+m)!(l-m)!(2l+1) / (4 pi (l+s)!(l-s)!)]
//   x sum_r C(l-s, r) C(l+s, r+s-m) (-1)^(l-r-s) sin^(2l-k)(th/2) cos^k(th/2),
// k = 2r + s - m (sin^2l(x) cot^k(x) written without negative powers).
double swsh(int s, int l, int m, double theta) {
    auto fact = [](int n) { double f = 1.0; for (int k = 2; k <= n; ++k) f *= k; return f; };
    auto binom = [&](int n, int k) { return (k < 0 || k > n) ? 0.0 : fact(n) / (fact(k) * fact(n - k)); };
    const double x = 0.5 * theta, sx = std::sin(x), cx = std::cos(x);
    const double norm = std::sqrt(fact(l + m) * fact(l - m) * (2 * l + 1) /
                                  (4.0 * M_PI * fact(l + s) * fact(l - s)));
    double sum = 0.0;
    for (int r = 0; r <= l - s; ++r) {
        const int k2 = r + s - m;
        if (k2 < 0 || k2 > l + s) continue;
        const int k = 2 * r + s - m;
        const double sign = ((l - r - s) % 2 == 0) ? 1.0 : -1.0;
        sum += binom(l - s, r) * binom(l + s, k2) * sign * std::pow(sx, 2 * l - k) * std::pow(cx, k);
    }
    return ((m % 2 == 0) ? 1.0 : -1.0) * norm * sum;
}

// SplitMix64 (Steele, Lea, Flood 2014): one 64-bit output per call.
uint64_t splitmix64(uint64_t& state) {
    uint64_t z = (state += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// r and r - r_+ at every r* node.
static void radial_nodes(const teuk_params& p, std::vector<double>& r, std::vector<double>& x) {
    const double h = (p.rstar_max - p.rstar_min) / (p.nr - 1);
    r.resize(p.nr);
    x.resize(p.nr);
    for (int i = 0; i < p.nr; ++i) r[i] = r_of_rstar(p.rstar_min + i * h, p.M, p.a, &x[i]);
}

// Runs body(j0, j1) over theta-row ranges on up to hardware_concurrency threads.
template <class F>
static void for_rows(int nth, long long work, F body) {
    unsigned nt = std::thread::hardware_concurrency();
    if (nt == 0) nt = 1;
    if (work < (1LL << 16)) nt = 1;
    nt = std::min<unsigned>(nt, (unsigned)nth);
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < nt; ++t) {
        const int j0 = (int)((long long)nth * t / nt), j1 = (int)((long long)nth * (t + 1) / nt);
        pool.emplace_back(body, j0, j1);
    }
    for (auto& th : pool) th.join();
}

}  // namespace teuk

using namespace teuk;

extern "C" {

const char* teuk_status_str(teuk_status st) {
    switch (st) {
    case TEUK_OK: return "ok";
    case TEUK_ERR_ARG: return "invalid argument";
    case TEUK_ERR_CUDA: return "CUDA error";
    case TEUK_ERR_NONFINITE: return "non-finite state";
    case TEUK_ERR_TIMEOUT: return "device wait timed out";
    case TEUK_ERR_STATE: return "call out of order";
    }
    return "unknown status";
}

const char* teuk_last_error(void) { return g_last_error.c_str(); }

teuk_status teuk_check_params(const teuk_params* p) {
    if (!p) return fail(TEUK_ERR_ARG, "params is NULL");
    if (p->nr < 7) return fail(TEUK_ERR_ARG, "nr must be >= 7 (WENO5 stencil)");
    if (p->ntheta < 5) return fail(TEUK_ERR_ARG, "ntheta must be >= 5");
    if ((double)p->nr * p->ntheta > 4.0e9)
        return fail(TEUK_ERR_ARG, "grid larger than 4e9 nodes");
    if (!(p->rstar_max > p->rstar_min) || !std::isfinite(p->rstar_min) ||
        !std::isfinite(p->rstar_max))
        return fail(TEUK_ERR_ARG, "need finite rstar_max > rstar_min");
    if (!(p->M > 0.0) || !std::isfinite(p->M)) return fail(TEUK_ERR_ARG, "need M > 0");
    if (!(std::fabs(p->a) <= p->M)) return fail(TEUK_ERR_ARG, "need |a| <= M");
    if (p->s < -2 || p->s > 2) return fail(TEUK_ERR_ARG, "spin weight s must be in -2..2");
    if (p->m < -64 || p->m > 64) return fail(TEUK_ERR_ARG, "|m| must be <= 64");
    if (!(p->eps >= 1e-60 && p->eps <= 1.0)) return fail(TEUK_ERR_ARG, "eps must be in [1e-60, 1]");
    if (p->wprec < TEUK_W_FP64 || p->wprec > TEUK_W_BF16)
        return fail(TEUK_ERR_ARG, "unknown weight precision");
    if (p->theta_mode != TEUK_THETA_CENTERED4 && p->theta_mode != TEUK_THETA_WENO5)
        return fail(TEUK_ERR_ARG, "unknown theta mode");
    if (p->rk != TEUK_RK_SSP33 && p->rk != TEUK_RK_SSP104)
        return fail(TEUK_ERR_ARG, "unknown time integrator");
    if (p->scheme != TEUK_SCHEME_WENO5 && p->scheme != TEUK_SCHEME_FD6_KO8)
        return fail(TEUK_ERR_ARG, "unknown r* scheme");
    if (p->scheme == TEUK_SCHEME_FD6_KO8 && p->theta_mode != TEUK_THETA_CENTERED4)
        return fail(TEUK_ERR_ARG, "the FD6+KO8 scheme uses centred theta differences");
    if (p->scheme == TEUK_SCHEME_FD6_KO8 && !(p->ko_sigma >= 0.0 && p->ko_sigma <= 1.0))
        return fail(TEUK_ERR_ARG, "ko_sigma must be in [0, 1]");
    if (p->dt < 0.0 || !std::isfinite(p->dt)) return fail(TEUK_ERR_ARG, "dt must be >= 0");
    if (p->dt == 0.0 && !(p->cfl > 0.0 && p->cfl <= 1.0))
        return fail(TEUK_ERR_ARG, "cfl must be in (0, 1] when dt == 0");
    return TEUK_OK;
}

teuk_status teuk_stable_dt(const teuk_params* p, double* dt_out) {
    teuk_status st = teuk_check_params(p);
    if (st != TEUK_OK) return st;
    if (!dt_out) return fail(TEUK_ERR_ARG, "dt_out is NULL");
    if (p->dt > 0.0) { *dt_out = p->dt; return TEUK_OK; }
    const double h = (p->rstar_max - p->rstar_min) / (p->nr - 1);
    const double dth = M_PI / p->ntheta;
    std::vector<double> r, x;
    radial_nodes(*p, r, x);
    std::vector<double> row_lam(p->ntheta, 0.0);
    for_rows(p->ntheta, (long long)p->nr * p->ntheta, [&](int j0, int j1) {
        for (int j = j0; j < j1; ++j) {
            double lam = 0.0;
            for (int i = 0; i < p->nr; ++i) {
                PointCoef c = point_coefficients_rx(r[i], x[i], (j + 0.5) * dth, *p);
                double kappa = c.Ath * (16.0 / 3.0) / (dth * dth) + std::fabs(c.Bth) * 1.5 / dth +
                               std::hypot(c.Cr, c.Ci);
                lam = std::fmax(lam, c.b / h + std::sqrt(kappa));
            }
            row_lam[j] = lam;
        }
    });
    double lam = 0.0;
    for (double v : row_lam) lam = std::fmax(lam, v);
    // SSP-RK(10,4): 2.8 = min(4.92 / sqrt(3), 13.9 / 2.51), its imaginary- and
    // real-axis stability extents relative to SSP-RK(3,3)
    *dt_out = (p->rk == TEUK_RK_SSP104 ? 2.8 : 1.0) * p->cfl / lam;
    return TEUK_OK;
}

size_t teuk_coeff_count(const teuk_params* p) {
    if (teuk_check_params(p) != TEUK_OK) return 0;
    return (size_t)coef_planes(p->theta_mode) * (size_t)p->nr * (size_t)p->ntheta;
}

teuk_status teuk_build_coefficients(const teuk_params* p, double dt, double* coef) {
    teuk_status st = teuk_check_params(p);
    if (st != TEUK_OK) return st;
    if (!coef) return fail(TEUK_ERR_ARG, "coef_host is NULL");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(TEUK_ERR_ARG, "dt must be > 0");
    const int nr = p->nr, nth = p->ntheta;
    const size_t plane = (size_t)nr * nth;
    const double h = (p->rstar_max - p->rstar_min) / (nr - 1);
    const double dth = M_PI / nth;
    const double sigma = ((p->m + p->s) % 2 == 0) ? 1.0 : -1.0;   // pole parity
    dt = stage_step(*p, dt);                 // forward-Euler step of one stage
    const double c6h = dt / (6.0 * h);
    std::vector<double> r, x;
    radial_nodes(*p, r, x);
    for_rows(nth, (long long)nr * nth, [&](int j0, int j1) {
    for (int j = j0; j < j1; ++j) {
        const double th = (j + 0.5) * dth;
        for (int i = 0; i < nr; ++i) {
            PointCoef c = point_coefficients_rx(r[i], x[i], th, *p);
            const size_t q = (size_t)j * nr + i;
            coef[kCb * plane + q] = c6h * c.b;
            coef[kCKr * plane + q] = c6h * c.Kr;
            coef[kCKi * plane + q] = c6h * c.Ki;
            coef[kCBr * plane + q] = dt * c.Btr;
            coef[kCBi * plane + q] = dt * c.Bti;
            coef[kCCi * plane + q] = dt * c.Ci;
            // fourth-order centred theta differences:
            //   12 dth^2 Psi_thth = -P(j+2) + 16 P(j+1) - 30 P(j) + 16 P(j-1) - P(j-2)
            //   12 dth   Psi_th   = -P(j+2) +  8 P(j+1)            -  8 P(j-1) + P(j-2)
            const bool weno_th = p->theta_mode == TEUK_THETA_WENO5;
            const double A = dt * c.Ath / (12.0 * dth * dth);
            const double B = weno_th ? 0.0 : dt * c.Bth / (12.0 * dth);
            if (weno_th) coef[kCBth * plane + q] = dt * c.Bth / (6.0 * dth);
            double w[5] = {-A + B, 16.0 * A - 8.0 * B, -30.0 * A + dt * c.Cr,
                           16.0 * A + 8.0 * B, -A - B};
            // Rows outside [0, nth) mirror across the pole with parity sigma:
            // row -1 -> 0, -2 -> 1, nth -> nth-1, nth+1 -> nth-2.
            for (int k = -2; k <= 2; ++k) {
                const int jj = j + k;
                int tgt;
                if (jj < 0) tgt = -1 - jj;
                else if (jj >= nth) tgt = 2 * nth - 1 - jj;
                else continue;
                w[tgt - j + 2] += sigma * w[k + 2];
                w[k + 2] = 0.0;
            }
            for (int k = 0; k < 5; ++k) coef[(kWm2 + k) * plane + q] = w[k];
        }
    }
    });
    return TEUK_OK;
}

}  // extern "C"
