// Host side of the library: parameter validation, the Kerr coefficient
// generator, the time-step rule and error reporting. binary64 throughout.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <system_error>
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

teuk_status fail_host(const char* what, const char* why) noexcept {
    try {
        g_last_error = std::string(what) + ": " + why;
    } catch (...) {
        g_last_error.clear();     // clear() never allocates
    }
    return TEUK_ERR_HOST;
}

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
// For the field Phi = r Delta^s Psi (TEUK_FIELD_PHI), Psi = Phi Delta^-s / r
// substituted into the same equation changes only B* and C:
//   Re B* = -[2 a^2 Delta / r + 2 s (r-M) varpi]/Sigma^2,
//   C    += [Delta (2a^2/r^2 - 2(1+s) M/r) - 2 i m a (2 s (r-M) + Delta/r)]/Sigma^2,
// so that Im C = -2 m a Delta / (r Sigma^2).
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
    double Bsr = Bs_r;
    if (p.field == TEUK_FIELD_PHI) {
        Bsr = -(2.0 * a * a * Delta / r + 2.0 * s * (r - M) * varpi) * inv;
        c.Cr += Delta * (2.0 * a * a / (r * r) - 2.0 * (1.0 + s) * M / r) * inv;
        c.Ci = -2.0 * m * a * Delta / r * inv;
    }
    c.Kr = Bsr - b * bstar - b * c.Btr;
    c.Ki = Bs_i - b * c.Bti;
    c.Ath = Delta * inv;
    c.Bth = Delta * (cs / sn) * inv;
    c.c = b;
    return c;
}

// Hyperboloidal slices (Sec. 2.2) for Phi = r Delta^s Psi: Eq. teuk0 under
// tau = t + T(r), T' = varpi/Delta - H', H' = 2 - W^2 + 4MW/S,
// rho = r/(1 + r/S), rho' = W^2, W = S/(r+S), and phi~ = phi + int a/Delta,
// divided by D = -A^tautau. Every quantity is written in rho, W = 1 - rho/S
// and x = 1/r = 1/rho - 1/S, finite from the horizon to scri:
//   delta = Delta x^2 = 1 - x (2M - a^2 x),  w = varpi x^2 = 1 + a^2 x^2,
//   sig = Sigma x^2 = sqrt(w^2 - a^2 x^2 delta sin^2),
//   G = (2 varpi - Delta H') = rho (rho + 4M + 8M^2/S - 2MW + a^2 x (W - 4M/S)),
//   E = Sigma + varpi - Delta H' = G - a^2 delta sin^2/(sig + w),
//   D = H' G - a^2 sin^2.
// The outgoing and ingoing speeds are b = rho^2 delta/E and c = W^2 E/D (the
// roots of the characteristic quadratic, whose discriminant is 4 W^4 Sigma^2);
// with pi = Phi_tau + b Phi_rho,
//   pi_tau = c pi_rho + K Phi_rho + Ath Phi_thth + Bth Phi_th + Bt pi + C Phi,
//   K = B^rho/D - b Bt - c db/drho,  Ath = 1/D,  Bth = cot/D,
//   D Bt = 2 s rho (4M/S - W) - 2(1+s) M H' + 2a^2 x (H' - 1)
//          - 2 delta rho^2 (W - 2M/S)/S + i (2 m a (1 - H') - 2 s a cos),
//   B^rho = 2 i m a W^2 - 2 W rho ((s+1) - W - rho x (2M - a^2 x)/S)
//           + 2 W^2 (M (1+s) - a^2 x),
//   D C = s - (m + s cos)^2/sin^2 - 2(s+1) M x + 2a^2 x^2 - 2 i m a x.
// db/drho is differentiated by hand from b = rho^2 delta / E.
PointCoef point_coefficients_hyp(double rho, double theta, const teuk_params& p) {
    const double M = p.M, a = p.a, s = p.s, m = p.m, S = p.hyp_S;
    const double a2 = a * a;
    const double sn = std::sin(theta), cs = std::cos(theta), sn2 = sn * sn;
    const double x = 1.0 / rho - 1.0 / S, x_r = -1.0 / (rho * rho);
    const double W = 1.0 - rho / S;
    const double delta = 1.0 - x * (2.0 * M - a2 * x), delta_r = (2.0 * a2 * x - 2.0 * M) * x_r;
    const double w = 1.0 + a2 * x * x, w_r = 2.0 * a2 * x * x_r;
    const double sig2 = w * w - a2 * x * x * delta * sn2;
    const double sig = std::sqrt(sig2);
    const double sig_r = (2.0 * w * w_r - a2 * sn2 * (2.0 * x * x_r * delta + x * x * delta_r)) /
                         (2.0 * sig);
    const double Hp = 2.0 - W * W + 4.0 * M * W / S;
    const double inner = rho + 4.0 * M + 8.0 * M * M / S - 2.0 * M * W + a2 * x * (W - 4.0 * M / S);
    const double G = rho * inner;
    const double G_r = inner + rho * (1.0 + 2.0 * M / S + a2 * x_r * (W - 4.0 * M / S) - a2 * x / S);
    const double den = sig + w;
    const double E = G - a2 * delta * sn2 / den;
    const double E_r = G_r - a2 * sn2 * (delta_r * den - delta * (sig_r + w_r)) / (den * den);
    const double D = Hp * G - a2 * sn2;
    const double invD = 1.0 / D;
    PointCoef c;
    c.b = rho * rho * delta / E;
    c.c = W * W * E * invD;
    const double b_r = (2.0 * rho * delta + rho * rho * delta_r) / E - c.b * E_r / E;
    c.Btr = (2.0 * s * rho * (4.0 * M / S - W) - 2.0 * (1.0 + s) * M * Hp + 2.0 * a2 * x * (Hp - 1.0)
             - 2.0 * delta * rho * rho * (W - 2.0 * M / S) / S) * invD;
    c.Bti = (2.0 * m * a * (1.0 - Hp) - 2.0 * s * a * cs) * invD;
    const double Brr = (-2.0 * W * rho * ((s + 1.0) - W - rho * x * (2.0 * M - a2 * x) / S)
                        + 2.0 * W * W * (M * (1.0 + s) - a2 * x)) * invD;
    const double Bri = 2.0 * m * a * W * W * invD;
    const double mc = m + s * cs;
    c.Cr = (s - mc * mc / sn2 - 2.0 * (s + 1.0) * M * x + 2.0 * a2 * x * x) * invD;
    c.Ci = -2.0 * m * a * x * invD;
    c.Kr = Brr - c.b * c.Btr - c.c * b_r;
    c.Ki = Bri - c.b * c.Bti;
    c.Ath = invD;
    c.Bth = (cs / sn) * invD;
    return c;
}

double horizon_rho(double M, double a, double S) {
    const double rp = M + std::sqrt(std::fmax(M * M - a * a, 0.0));
    return rp * S / (rp + S);
}

// On the hyperboloidal slices a range given as [0, 0] stands for the whole
// slice, from the outer horizon rho_+ to scri (rho = S).
teuk_params resolve_params(const teuk_params& p) {
    teuk_params q = p;
    if (q.coords == TEUK_COORDS_HYPERBOLOIDAL && q.rstar_min == 0.0 && q.rstar_max == 0.0 &&
        q.M > 0.0 && std::fabs(q.a) <= q.M && q.hyp_S > 0.0) {
        q.rstar_min = horizon_rho(q.M, q.a, q.hyp_S);
        q.rstar_max = q.hyp_S;
    }
    return q;
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

// Per radial node: r and r - r_+ at every r* node; rho itself on the
// hyperboloidal grid (kept in r, x unused).
static void radial_nodes(const teuk_params& p, std::vector<double>& r, std::vector<double>& x) {
    const double h = (p.rstar_max - p.rstar_min) / (p.nr - 1);
    r.resize(p.nr);
    x.resize(p.nr);
    for (int i = 0; i < p.nr; ++i) {
        if (p.coords == TEUK_COORDS_HYPERBOLOIDAL) {
            r[i] = p.rstar_min + i * h;
            x[i] = 0.0;
        } else {
            r[i] = r_of_rstar(p.rstar_min + i * h, p.M, p.a, &x[i]);
        }
    }
}

static PointCoef node_coefficients(double r, double x, double theta, const teuk_params& p) {
    return p.coords == TEUK_COORDS_HYPERBOLOIDAL ? point_coefficients_hyp(r, theta, p)
                                                 : point_coefficients_rx(r, x, theta, p);
}

// Runs body(j0, j1) over theta-row ranges on up to hardware_concurrency threads.
template <class F>
static void for_rows(int nth, long long work, F body) {
    unsigned nt = std::thread::hardware_concurrency();
    if (nt == 0) nt = 1;
    if (work < (1LL << 16)) nt = 1;
    nt = std::min<unsigned>(nt, (unsigned)nth);
    std::vector<std::thread> pool;
    pool.reserve(nt);
    for (unsigned t = 0; t < nt; ++t) {
        const int j0 = (int)((long long)nth * t / nt), j1 = (int)((long long)nth * (t + 1) / nt);
        bool started = false;
        try {
            pool.emplace_back(body, j0, j1);
            started = true;
        } catch (const std::system_error&) {
        }
        if (!started) body(j0, j1);     // no thread available: this range here
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
    case TEUK_ERR_HOST: return "host resource unavailable";
    }
    return "unknown status";
}

const char* teuk_last_error(void) { return g_last_error.c_str(); }

teuk_status teuk_horizon_rho(double M, double a, double S, double* rho_out) {
    if (!rho_out) return fail(TEUK_ERR_ARG, "rho_out is NULL");
    if (!(M > 0.0) || !std::isfinite(M)) return fail(TEUK_ERR_ARG, "need M > 0");
    if (!(std::fabs(a) <= M)) return fail(TEUK_ERR_ARG, "need |a| <= M");
    if (!(S >= M && S <= 1e6 * M)) return fail(TEUK_ERR_ARG, "S must be in [M, 1e6 M]");
    *rho_out = horizon_rho(M, a, S);
    return TEUK_OK;
}

teuk_status teuk_check_params(const teuk_params* p) {
    if (!p) return fail(TEUK_ERR_ARG, "params is NULL");
    const teuk_params q = resolve_params(*p);
    p = &q;
    if (p->nr < 7) return fail(TEUK_ERR_ARG, "nr must be >= 7 (WENO5 stencil)");
    if (p->ntheta < 5) return fail(TEUK_ERR_ARG, "ntheta must be >= 5");
    if (p->ntheta > 4 * 65535)      // four theta rows per CTA, grid y <= 65535
        return fail(TEUK_ERR_ARG, "ntheta must be <= 262140");
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
        return fail(TEUK_ERR_ARG, "unknown radial scheme");
    if (p->scheme == TEUK_SCHEME_FD6_KO8 && p->theta_mode != TEUK_THETA_CENTERED4)
        return fail(TEUK_ERR_ARG, "the FD6+KO8 scheme uses centred theta differences");
    if (p->scheme == TEUK_SCHEME_FD6_KO8 && !(p->ko_sigma >= 0.0 && p->ko_sigma <= 1.0))
        return fail(TEUK_ERR_ARG, "ko_sigma must be in [0, 1]");
    if (p->field != TEUK_FIELD_PSI && p->field != TEUK_FIELD_PHI)
        return fail(TEUK_ERR_ARG, "unknown field");
    if (p->coords == TEUK_COORDS_HYPERBOLOIDAL) {
        if (p->field != TEUK_FIELD_PHI)
            return fail(TEUK_ERR_ARG, "the hyperboloidal slices evolve Phi (TEUK_FIELD_PHI)");
        if (!(p->hyp_S >= p->M && p->hyp_S <= 1e6 * p->M))
            return fail(TEUK_ERR_ARG, "hyp_S must be in [M, 1e6 M]");
        const double rhop = horizon_rho(p->M, p->a, p->hyp_S);
        if (p->rstar_min < rhop * (1.0 - 1e-12))
            return fail(TEUK_ERR_ARG, "rho_min below the horizon rho_+");
        if (p->rstar_max > p->hyp_S * (1.0 + 1e-12))
            return fail(TEUK_ERR_ARG, "rho_max beyond scri (rho = S)");
    } else if (p->coords != TEUK_COORDS_RSTAR) {
        return fail(TEUK_ERR_ARG, "unknown coordinates");
    }
    if (p->dt < 0.0 || !std::isfinite(p->dt)) return fail(TEUK_ERR_ARG, "dt must be >= 0");
    if (p->dt == 0.0 && !(p->cfl > 0.0 && p->cfl <= 1.0))
        return fail(TEUK_ERR_ARG, "cfl must be in (0, 1] when dt == 0");
    return TEUK_OK;
}

teuk_status teuk_stable_dt(const teuk_params* p, double* dt_out) {
    return guarded("teuk_stable_dt", [&]() -> teuk_status {
        teuk_status st = teuk_check_params(p);
        if (st != TEUK_OK) return st;
        if (!dt_out) return fail(TEUK_ERR_ARG, "dt_out is NULL");
        const teuk_params q = resolve_params(*p);
        p = &q;
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
                    PointCoef c = node_coefficients(r[i], x[i], (j + 0.5) * dth, *p);
                    double kappa = c.Ath * (16.0 / 3.0) / (dth * dth) +
                                   std::fabs(c.Bth) * 1.5 / dth + std::hypot(c.Cr, c.Ci);
                    const double speed = std::fmax(std::fabs(c.b), std::fabs(c.c));
                    lam = std::fmax(lam, speed / h + std::sqrt(kappa));
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
    });
}

size_t teuk_coeff_count(const teuk_params* p) {
    if (teuk_check_params(p) != TEUK_OK) return 0;
    return (size_t)coef_planes(*p) * (size_t)p->nr * (size_t)p->ntheta;
}

teuk_status teuk_build_coefficients(const teuk_params* p, double dt, double* coef) {
    return guarded("teuk_build_coefficients", [&]() -> teuk_status {
        teuk_status st = teuk_check_params(p);
        if (st != TEUK_OK) return st;
        if (!coef) return fail(TEUK_ERR_ARG, "coef_host is NULL");
        const teuk_params q = resolve_params(*p);
        p = &q;
        if (!(dt > 0.0) || !std::isfinite(dt)) return fail(TEUK_ERR_ARG, "dt must be > 0");
        const int nr = p->nr, nth = p->ntheta;
        const size_t plane = (size_t)nr * nth;
        const double h = (p->rstar_max - p->rstar_min) / (nr - 1);
        const double dth = M_PI / nth;
        const double sigma = ((p->m + p->s) % 2 == 0) ? 1.0 : -1.0;   // pole parity
        dt = stage_step(*p, dt);                 // forward-Euler step of one stage
        // radial planes: the WENO5 kernel forms 6 h D, the FD6 + KO8 kernel
        // 60 h D (the sixth-order stencil's own normalisation)
        const double c6h = dt / ((p->scheme == TEUK_SCHEME_FD6_KO8 ? 60.0 : 6.0) * h);
        std::vector<double> r, x;
        radial_nodes(*p, r, x);
        for_rows(nth, (long long)nr * nth, [&](int j0, int j1) {
        for (int j = j0; j < j1; ++j) {
            const double th = (j + 0.5) * dth;
            for (int i = 0; i < nr; ++i) {
                PointCoef c = node_coefficients(r[i], x[i], th, *p);
                const size_t q = (size_t)j * nr + i;
                coef[kCb * plane + q] = c6h * c.b;
                if (p->coords == TEUK_COORDS_HYPERBOLOIDAL) coef[kCc * plane + q] = c6h * c.c;
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
                else if (p->coords == TEUK_COORDS_HYPERBOLOIDAL) coef[kCBth * plane + q] = 0.0;
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
    });
}

}  // extern "C"
