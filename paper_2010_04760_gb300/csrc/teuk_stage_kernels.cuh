#pragma once
// Fused WENO5 / Teukolsky right-hand side / Runge-Kutta stage kernel for
// sm_103a (SSP-RK(3,3) stages, or the forward-Euler stages of SSP-RK(10,4)):
// the device code, shared by teuk_stage.cu (r* kernels, batches, launch code),
// teuk_stage_hyp.cu (the hyperboloidal instantiations) and teuk_fused.cu /
// teuk_fused_hyp.cu (the fused persistent step), compiled in parallel.
//
// A work item is a segment of SEG consecutive radial nodes (r*, or rho on the
// hyperboloidal slices) of WARPS theta rows, one row per warp. The block's
// threads share phases 1-3 over the item's rows (process_item), and each warp
// then does phase 4 for its own row:
//   1. forms the binary64 first differences d_k = f_{k+1} - f_k of the four
//      components over the segment plus its halo (ghosts copy the edge value
//      in r*; on the hyperboloidal slices they extrapolate the quartic
//      through the five edge nodes),
//   2. forms s_k = d_{k-1} - 2 d_k + d_{k+1},
//   3. at every interface computes the nonlinear weights (Sec. 3.1.2) in the
//      requested precision (Sec. 3.1.3) and the binary64 flux term
//         F = x1 + 2 x2 - 2 w0 s(x0,x1,x2) - w2 s(x1,x2,x3),
//      which equals 6 (fhat_{i+1/2} - f_i) for the positive-direction flux
//      with x = (d_{i-2}, d_{i-1}, d_i, d_{i+1}); the negative-direction flux
//      is its mirror image (x = d_{i+2}, d_{i+1}, d_i, d_{i-1}, G = -F),
//   4. at every node forms 6 h D = 6 d + F_{i+1/2} - F_{i-1/2}, the theta
//      stencil, the right-hand side -(M du + L u + A u) (Sec. 2.3; the pi
//      rows move with their own speed c on the hyperboloidal slices) and the
//      Runge-Kutta combination (Sec. 3.2), and stores the new stage.
// Every binary64 quantity is formed once per node (no recomputation inside a
// segment); the weights run in their format's own arithmetic, off the FP64
// pipe. The only binary64 operations are the differences, the weighted flux
// combination, the right-hand side and the Runge-Kutta update.
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "teuk_internal.h"

namespace teuk {

#ifndef TEUK_WARPS
#define TEUK_WARPS 4
#endif
#ifndef TEUK_MINB
#define TEUK_MINB 8                // resident CTAs per SM the register budget targets
#endif
constexpr int WARPS = TEUK_WARPS;  // theta rows per CTA (one per warp)
#define TEUK_BOUNDS __launch_bounds__(TEUK_WARPS * 32, TEUK_MINB)

// Radial nodes per warp: 32 with reduced-precision weights, 64 with binary64
// weights (each the measured best on GB300 for the 2048 x 128 workload).
template <int W> struct Seg {
#ifdef TEUK_SEG
    static constexpr int value = TEUK_SEG;
#else
    static constexpr int value = W == TEUK_W_FP64 ? 64 : 32;
#endif
};
// Shared-memory layout of one warp's segment, per component: first
// differences d_k (k = i0-3 .. i0+S+1), then s_k (k = i0-2 .. i0+S), then
// flux terms of interfaces i+1/2 (i = i0-1 .. i0+S-1).
template <int S> struct Geo {
    static constexpr int SEG = S, ND = S + 5, NS = S + 3, NF = S + 1, NW = ND + NS + NF;
};
// The FD6 + KO8 comparison scheme needs only first differences, with a
// 4-node halo (k = i0-4 .. i0+S+3).
template <int S> struct GeoFD {
    static constexpr int SEG = S, ND = S + 8, NS = 0, NF = 0, NW = ND;
};

struct StageArgs {
    const double* coef;   // coef_planes(p) planes of nth*nr
    const double* un;     // u^n (stages 2, 3)
    const double* up;     // u^{(s-1)}, the operator's argument
    double* out;          // may alias un (read only at the same node)
    int nr, nth;
    long long plane;
    double dt;            // step (the Psi rows need dt * pi)
    double alpha, beta;   // u_out = alpha u^n + beta (u_prev + dt F)
    double eps4;          // 4 eps (binary64 weights)
    int eps_exp;          // floor(log2 eps)
    int eps_pow2;         // eps is a power of two
    unsigned eps_mant;    // binary32 bits of eps 2^-eps_exp rounded to the
                          // weight format (a value in [1, 2])
    unsigned pole_flip;   // 0x80000000 when the pole parity (-1)^(m+s) is odd
    double ko;            // FD6+KO8 scheme: h_stage sigma / (256 h), else 0
};

// The SSP-RK(3,3) step of the WENO5 scheme keeps its second stage scaled by
// four (Sec. 3.2): v = 4 u^(2) = 3 u^n + (u^(1) + dt F(u^(1))), one
// multiply-add per row fewer than 3/4 u^n + 1/4 (...) (the kStageScaled form
// of the stage kernels, alpha = 3). The third stage then needs F(v/4). The
// smoothness indicators are quadratic in the data, so data scaled by 4 and
// epsilon scaled by 16 give every (eps + IS_k) times 16 and the same weights
// (Sec. 3.1.2), while the rest of F is linear: F_eps(v/4) = F_16eps(v)/4, and
// u^{n+1} = 1/3 u^n + 1/6 (v + dt F_16eps(v)). Scaling by powers of two is
// exact in binary floating point and commutes with every rounding, so this
// third stage rounds exactly like 1/3 u^n + 2/3 (u^(2) + dt F(u^(2))) on
// u^(2) = v/4; only the second stage's own roundings differ (one fewer).
constexpr double kScaledAlpha = 3.0;
constexpr double kThirdBetaScaled = 1.0 / 6.0;
constexpr int kScaledEpsLog2 = 4;      // the third stage's eps: 16 eps
__host__ __device__ inline void eps_times_16(StageArgs& A) {
    A.eps4 *= 16.0;
    A.eps_exp += kScaledEpsLog2;
}

// ---------------------------------------------------------------------------
// Exact bit-level helpers (integer pipes only).
// ---------------------------------------------------------------------------

// 2^q as a binary32, q in [-149, 127].
__device__ __forceinline__ float pow2f(int q) {
    return q >= -126 ? __int_as_float((q + 127) << 23) : __int_as_float(1 << (q + 149));
}

// |x| 2^-e rounded to P significant bits (ties to even), with the subnormal
// spacing of a format whose smallest normal exponent is EMIN; returned as the
// binary32 holding that value exactly (requires |x| 2^-e < 2^128).
template <int P, int EMIN>
__device__ __forceinline__ float round_scaled(double x, int e) {
    // bit pattern from the 32-bit halves (see max_exponent)
    const unsigned long long bits = ((unsigned long long)(unsigned)__double2hiint(x) << 32) |
                                    (unsigned)__double2loint(x);
    const bool neg = (bits >> 63) != 0;
    const int E = (int)((bits >> 52) & 0x7ff);
    unsigned long long m = bits & 0xfffffffffffffULL;
    int ex;
    if (E == 0) {
        if (m == 0) return neg ? -0.0f : 0.0f;
        ex = -1074;
    } else {
        m |= (1ULL << 52);
        ex = E - 1075;
    }
    const int L = 64 - __clzll((long long)m);
    const int lead = ex - e + L - 1;             // floor(log2(|x| 2^-e))
    const int leff = lead < EMIN ? EMIN : lead;
    const int q = leff - (P - 1);                // unit of the last place
    const int sh = q - (ex - e);
    unsigned long long n;
    if (sh <= 0) {
        n = m << (-sh);
    } else if (sh >= 64) {
        n = 0;
    } else {
        n = m >> sh;
        const unsigned long long rem = m & ((1ULL << sh) - 1);
        const unsigned long long half = 1ULL << (sh - 1);
        if (rem > half || (rem == half && (n & 1ULL))) n += 1;
    }
    if (n == 0) return neg ? -0.0f : 0.0f;
    // n <= 2^P <= 2^24: a 32-bit conversion is exact (a 64-bit one would run
    // on the FP64 pipe)
    const float v = __fmul_rn(__uint2float_rn((unsigned)n), pow2f(q < -149 ? -149 : q));
    return neg ? -v : v;
}

// Same result as round_scaled for a normal x whose scaled value is normal in
// the format, with 32-bit integer operations only; other inputs take the
// general path.
template <int P, int EMIN>
__device__ __forceinline__ float round_scaled_fast(double x, int e) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int E = (int)((hi >> 20) & 0x7ffu);
    const int t = E - 1023 - e;                      // floor(log2(|x| 2^-e))
    if (E == 0 || t < EMIN) return round_scaled<P, EMIN>(x, e);
    constexpr int D = 53 - P;                        // dropped significand bits
    unsigned kept, rup;
    if constexpr (D < 32) {
        kept = ((hi & 0xfffffu) << (32 - D)) | (lo >> D);
        const unsigned dropped = lo & ((1u << D) - 1u);
        const unsigned half = 1u << (D - 1);
        rup = (dropped > half || (dropped == half && (kept & 1u))) ? 1u : 0u;
    } else {
        constexpr int DH = D - 32;
        kept = (hi & 0xfffffu) >> DH;
        const unsigned dh = hi & ((1u << DH) - 1u);
        const unsigned half = 1u << (DH - 1);
        rup = (dh > half || (dh == half && (lo != 0u || (kept & 1u)))) ? 1u : 0u;
    }
    // a carry out of the significand increments the exponent field
    const unsigned mag = ((unsigned)(t + 127) << 23) + ((kept + rup) << (24 - P));
    return __uint_as_float((hi & 0x80000000u) | mag);
}

// binary32 -> binary64, exact, on the integer pipes (finite input).
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned sign = u & 0x80000000u;
    const unsigned E = (u >> 23) & 0xffu;
    const unsigned mnt = u & 0x7fffffu;
    if (E == 0) {
        if (mnt == 0) return __hiloint2double((int)sign, 0);
        const int p = 31 - __clz((int)mnt);                      // 0..22
        const unsigned long long frac =
            ((unsigned long long)(mnt ^ (1u << p))) << (52 - p);
        const unsigned long long b = ((unsigned long long)(p - 149 + 1023) << 52) | frac;
        return __hiloint2double((int)(sign | (unsigned)(b >> 32)), (int)(unsigned)b);
    }
    return __hiloint2double((int)(sign | ((E + 896u) << 20) | (mnt >> 3)), (int)(mnt << 29));
}

// ---------------------------------------------------------------------------
// Weight formats: significand bits P, smallest normal exponent EMIN, and the
// clamp range [2^LOG2TINY, 2^LOG2HUGE] of the scaled epsilon; the arithmetic
// of each format is Ops<W> below.
// ---------------------------------------------------------------------------
template <int W> struct Fmt;
template <> struct Fmt<TEUK_W_FP32> {
    static constexpr int P = 24, EMIN = -126, LOG2TINY = -126, LOG2HUGE = 100;
};
template <> struct Fmt<TEUK_W_FP16> {
    static constexpr int P = 11, EMIN = -14, LOG2TINY = -14, LOG2HUGE = 15;
};
template <> struct Fmt<TEUK_W_BF16> {
    static constexpr int P = 8, EMIN = -126, LOG2TINY = -126, LOG2HUGE = 100;
};

// floor(log2 max_k |x_k|) from the bit patterns (0 if all are zero).
__device__ __forceinline__ int max_exponent(double x0, double x1, double x2, double x3) {
    unsigned ex = (unsigned)__double2hiint(x0) & 0x7ff00000u;
    ex = max(ex, (unsigned)__double2hiint(x1) & 0x7ff00000u);
    ex = max(ex, (unsigned)__double2hiint(x2) & 0x7ff00000u);
    ex = max(ex, (unsigned)__double2hiint(x3) & 0x7ff00000u);
    if (ex != 0u) return (int)(ex >> 20) - 1023;
    // all zero or subnormal: the largest significand decides. The significand
    // is assembled from the 32-bit halves (masking a reinterpreted double's
    // sign bit would be turned into an absolute-value instruction on the
    // FP64 pipe).
    unsigned long long a = 0;
    const double xs[4] = {x0, x1, x2, x3};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const unsigned long long mk =
            ((unsigned long long)((unsigned)__double2hiint(xs[k]) & 0xfffffu) << 32) |
            (unsigned)__double2loint(xs[k]);
        a = max(a, mk);
    }
    if (a == 0) return 0;
    return (63 - __clzll((long long)a)) - 1074;
}

// Arithmetic of a weight format: values held in the format's own type, each
// operation correctly rounded to nearest even in the format (the half and
// bfloat16 instructions without contraction; a quotient taken in binary32 and
// rounded once more is the correctly rounded quotient, 24 >= 2p + 2).
template <int W> struct Ops;
template <> struct Ops<TEUK_W_FP32> {
    using T = float;
    __device__ static T in(float x) { return x; }
    __device__ static float out(T x) { return x; }
    __device__ static T add(T a, T b) { return __fadd_rn(a, b); }
    __device__ static T sub(T a, T b) { return __fsub_rn(a, b); }
    __device__ static T mul(T a, T b) { return __fmul_rn(a, b); }
    __device__ static T div(T a, T b) { return __fdiv_rn(a, b); }
    __device__ static T min(T a, T b) { return fminf(a, b); }
};
template <> struct Ops<TEUK_W_FP16> {
    using T = __half;
    __device__ static T in(float x) { return __float2half_rn(x); }
    __device__ static float out(T x) { return __half2float(x); }
    __device__ static T add(T a, T b) { return __hadd_rn(a, b); }
    __device__ static T sub(T a, T b) { return __hsub_rn(a, b); }
    __device__ static T mul(T a, T b) { return __hmul_rn(a, b); }
    __device__ static T div(T a, T b) { return in(__fdiv_rn(out(a), out(b))); }
    __device__ static T min(T a, T b) { return __hmin(a, b); }
};
template <> struct Ops<TEUK_W_BF16> {
    using T = __nv_bfloat16;
    __device__ static T in(float x) { return __float2bfloat16_rn(x); }
    __device__ static float out(T x) { return __bfloat162float(x); }
    __device__ static T add(T a, T b) { return __hadd_rn(a, b); }
    __device__ static T sub(T a, T b) { return __hsub_rn(a, b); }
    __device__ static T mul(T a, T b) { return __hmul_rn(a, b); }
    __device__ static T div(T a, T b) { return in(__fdiv_rn(out(a), out(b))); }
    __device__ static T min(T a, T b) { return __hmin(a, b); }
};

// Reduced-precision Jiang-Shu weights omega_0, omega_2 (Sec. 3.1.2-3.1.3) of
// the stencil with first differences x0..x3 (positive-direction order).
// Smoothness indicators in first differences:
//   IS0 = 13/12 (x1-x0)^2 + 1/4 (3x1-x0)^2
//   IS1 = 13/12 (x2-x1)^2 + 1/4 (x1+x2)^2
//   IS2 = 13/12 (x3-x2)^2 + 1/4 (3x2-x3)^2
// The differences are scaled by 2^-e (e = floor(log2 max|x|)) before rounding
// to the format, epsilon by 2^-2e (clamped to [tiny, huge]), and alpha_k is
// normalised by the smallest eps + IS: alpha_k = d_k (t_min/t_k)^2. The
// operation sequence is fixed (no contraction) so that every rounding is
// determined; each operation is one of Ops<W>, in the format itself.
template <int W>
__device__ __forceinline__ void reduced_weights(double x0, double x1, double x2, double x3,
                                                const StageArgs& A, float& w0, float& w2) {
    using F = Fmt<W>;
    using O = Ops<W>;
    using T = typename O::T;
    const int e = max_exponent(x0, x1, x2, x3);
    const T y0 = O::in(round_scaled_fast<F::P, F::EMIN>(x0, e));
    const T y1 = O::in(round_scaled_fast<F::P, F::EMIN>(x1, e));
    const T y2 = O::in(round_scaled_fast<F::P, F::EMIN>(x2, e));
    const T y3 = O::in(round_scaled_fast<F::P, F::EMIN>(x3, e));
    // eps 2^-2e clamped to [tiny, huge], rounded to the format. Inside the
    // clamp range the value is normal in the format, so rounding it is
    // rounding eps's significand (precomputed) and shifting the exponent.
    float ehf;
    {
        const int lead = A.eps_exp - 2 * e;
        if (lead < F::LOG2TINY) ehf = pow2f(F::LOG2TINY);
        else if (lead > F::LOG2HUGE || (lead == F::LOG2HUGE && !A.eps_pow2))
            ehf = pow2f(F::LOG2HUGE);
        else ehf = __uint_as_float(A.eps_mant + ((unsigned)lead << 23));
    }
    const T eh = O::in(ehf);
    const T c13 = O::in((float)(13.0 / 12.0)), three = O::in(3.0f), quarter = O::in(0.25f);
    const T d0 = O::in(0.1f), d1 = O::in(0.6f), d2 = O::in(0.3f);
    T a, b, IS0, IS1, IS2;
    a = O::sub(y1, y0);
    b = O::sub(O::mul(three, y1), y0);
    IS0 = O::add(O::mul(c13, O::mul(a, a)), O::mul(quarter, O::mul(b, b)));
    a = O::sub(y2, y1);
    b = O::add(y1, y2);
    IS1 = O::add(O::mul(c13, O::mul(a, a)), O::mul(quarter, O::mul(b, b)));
    a = O::sub(y3, y2);
    b = O::sub(O::mul(three, y2), y3);
    IS2 = O::add(O::mul(c13, O::mul(a, a)), O::mul(quarter, O::mul(b, b)));
    const T t0 = O::add(eh, IS0), t1 = O::add(eh, IS1), t2 = O::add(eh, IS2);
    const T tm = O::min(t0, O::min(t1, t2));
    const T r0 = O::div(tm, t0), r1 = O::div(tm, t1), r2 = O::div(tm, t2);
    const T a0 = O::mul(d0, O::mul(r0, r0));
    const T a1 = O::mul(d1, O::mul(r1, r1));
    const T a2 = O::mul(d2, O::mul(r2, r2));
    const T sum = O::add(O::add(a0, a1), a2);
    w0 = O::out(O::div(a0, sum));
    w2 = O::out(O::div(a2, sum));
}

// 6 (fhat_{i+1/2} - f_i) for first differences x0..x3 (positive-direction
// order) and s1 = x0 - 2x1 + x2, s2 = x1 - 2x2 + x3:
//   q0 - q1 = -s1/3, q2 - q1 = -s2/6, q1 - f_i = (x1 + 2 x2)/6,
//   6 (fhat - f_i) = x1 + 2 x2 - 2 omega_0 s1 - omega_2 s2.
// NEG returns the negated value (the negative-direction flux term), with the
// sign folded into the multiply-adds.
template <int W, bool NEG>
__device__ __forceinline__ double flux6(double x0, double x1, double x2, double x3,
                                        double s1, double s2, const StageArgs& A) {
    const double base = NEG ? fma(-2.0, x2, -x1) : fma(2.0, x2, x1);
    if constexpr (W == TEUK_W_FP64) {
        // 4 (eps + IS_k) = (13/3) a^2 + b^2 + 4 eps; omega from one reciprocal:
        //   omega_0 = d0 t1^2 t2^2 / S, omega_2 = d2 t0^2 t1^2 / S,
        //   S = d0 t1^2 t2^2 + d1 t0^2 t2^2 + d2 t0^2 t1^2.
        const double c133 = 13.0 / 3.0;
        const double a0 = x1 - x0, b0 = fma(3.0, x1, -x0);
        const double a1 = x2 - x1, b1 = x1 + x2;
        const double a2 = x3 - x2, b2 = fma(3.0, x2, -x3);
        const double t0 = fma(c133 * a0, a0, fma(b0, b0, A.eps4));
        const double t1 = fma(c133 * a1, a1, fma(b1, b1, A.eps4));
        const double t2 = fma(c133 * a2, a2, fma(b2, b2, A.eps4));
        const double q0 = t0 * t0, q1 = t1 * t1, q2 = t2 * t2;
        const double p12 = q1 * q2, p02 = q0 * q2, p01 = q0 * q1;
        const double S = fma(0.1, p12, fma(0.6, p02, 0.3 * p01));
        const double rS = __drcp_rn(S);
        const double c1 = (NEG ? 0.2 : -0.2) * p12 * rS;   // -+ 2 omega_0
        const double c2 = (NEG ? 0.3 : -0.3) * p01 * rS;   // -+ omega_2
        return fma(c2, s2, fma(c1, s1, base));
    } else {
        float w0, w2;
        reduced_weights<W>(x0, x1, x2, x3, A, w0, w2);
        const double c1 = f2d_exact(NEG ? 2.0f * w0 : -2.0f * w0);   // exact
        const double c2 = f2d_exact(NEG ? w2 : -w2);
        return fma(c2, s2, fma(c1, s1, base));
    }
}

// Flux term of interface number idx (component idx / NF) of a warp's segment;
// sw is the warp's shared-memory block (first differences, then s, then flux).
// Psi components take the positive-direction flux, x = d_{i-2..i+1}; pi
// components the negative-direction one, whose stencil is the mirror image
// (x = d_{i+2..i-1}) and whose flux term is the negated positive form. The
// stencil is chosen by integer index and the sign applied to the bit pattern,
// so that no binary64 instruction is spent on either.
template <int W, class G>
__device__ __forceinline__ double interface_flux(const double* sw, int idx, const StageArgs& A) {
    const int c = idx / G::NF, k = idx - c * G::NF;
    const double* dl = sw + c * G::NW;
    const double* sd = dl + G::ND;
    const bool neg = c >= 2;
    const double F = flux6<W, false>(dl[neg ? k + 4 : k], dl[neg ? k + 3 : k + 1], dl[k + 2],
                                     dl[neg ? k + 1 : k + 3], sd[neg ? k + 2 : k], sd[k + 1], A);
    const int hi = __double2hiint(F) ^ (neg ? (int)0x80000000 : 0);
    return __hiloint2double(hi, __double2loint(F));
}

// x with its sign bit XORed with mask (integer pipe).
__device__ __forceinline__ double flip_sign(double x, unsigned mask) {
    return __hiloint2double(__double2hiint(x) ^ (int)mask, __double2loint(x));
}

// 6 dtheta times the positive-direction WENO5 derivative at v[3] of the six
// values v[0..5] (rows -3..+2 of the oriented theta line): the interfaces
// +1/2 and -1/2 use the same first/third-difference flux form as in r*.
template <int W>
__device__ __forceinline__ double theta_weno_6hd(const double v[6], const StageArgs& A) {
    const double d0 = v[1] - v[0], d1 = v[2] - v[1], d2 = v[3] - v[2];
    const double d3 = v[4] - v[3], d4 = v[5] - v[4];
    const double sa = fma(-2.0, d1, d0 + d2);
    const double sb = fma(-2.0, d2, d1 + d3);
    const double sc = fma(-2.0, d3, d2 + d4);
    const double fp = flux6<W, false>(d1, d2, d3, d4, sb, sc, A);
    const double fm = flux6<W, false>(d0, d1, d2, d3, sa, sb, A);
    return fma(6.0, d2, fp) - fm;
}

// Right-hand side and Runge-Kutta combination at node i0 + p of row j
// (Sec. 2.3, Sec. 3.2). sw holds the segment's first differences and flux
// terms. Loads use a clamped node index; the caller stores only real nodes.
// 60h times the sixth-order centred derivative and the eighth difference
// delta^8 u at a node, from the first differences d[-4..3] around it
// (d[m] = u_{j+m+1} - u_{j+m}):
//   60 h u' = (d-3 + d2) - 8 (d-2 + d1) + 37 (d-1 + d0)     (Sec. 3.1.1 stencil)
//   delta^8 u = (d3 - d-4) + 7 (d-3 - d2) + 21 (d1 - d-2) + 35 (d-1 - d0).
// The radial coefficient planes of this scheme carry 1/(60h).
__device__ __forceinline__ void fd6_ko8(const double* d, double& D60h, double& e8) {
    const double t = fma(-8.0, d[2] + d[5], d[1] + d[6]);
    D60h = fma(37.0, d[3] + d[4], t);
    const double u = fma(7.0, d[1] - d[6], d[7] - d[0]);
    e8 = fma(35.0, d[3] - d[4], fma(21.0, d[5] - d[2], u));
}

// Load of a state value. The stage kernels read states that no thread writes
// during the launch (read-only data path); the fused step kernel reads states
// that other blocks of the same launch wrote, so it loads them from L2 (after
// the acquire that orders those writes before the load).
template <bool FUSED>
__device__ __forceinline__ double ld_state(const double* p) {
    if constexpr (FUSED) return __ldcg(p);
    else return __ldg(p);
}

// Node k of a radial line f[0..nr) extended past either end (k in
// [-4, nr+3]) by the quartic through the five edge nodes: the fifth
// difference of the extended line vanishes, so each ghost follows from the
// five values before it, u = 5 v0 - 10 v1 + 10 v2 - 5 v3 + v4 (v0 nearest).
template <bool FUSED = false>
static __device__ __noinline__ double ghost_value(const double* f, int nr, int k) {
    if (k >= 0 && k < nr) return ld_state<FUSED>(f + k);
    const bool left = k < 0;
    const int step = left ? 1 : -1;
    const int e = left ? 0 : nr - 1;
    double v0 = ld_state<FUSED>(f + e), v1 = ld_state<FUSED>(f + e + step);
    double v2 = ld_state<FUSED>(f + e + 2 * step);
    double v3 = ld_state<FUSED>(f + e + 3 * step), v4 = ld_state<FUSED>(f + e + 4 * step);
    const int n = left ? -k : k - (nr - 1);
    for (int t = 0; t < n; ++t) {
        const double u = fma(5.0, v0 - v3, fma(10.0, v2 - v1, v4));
        v4 = v3; v3 = v2; v2 = v1; v1 = v0; v0 = u;
    }
    return v0;
}

// HYP: the hyperboloidal slices, whose pi rows have their own speed (plane
// kCc); in r* they share the Psi rows' b.
template <int W, int STAGE, int THETA, class G, int SCHEME = 0, bool HYP = false,
          bool FUSED = false>
__device__ __forceinline__ void node_update(const StageArgs& A, const double* sw, int j,
                                            int i0, int p, double out[4]) {
    constexpr int NW = G::NW, FO = G::ND + G::NS;   // flux terms start at FO
    const int nr = A.nr;
    const int i = min(i0 + p, nr - 1);
    const long long P = A.plane;
    const long long q = (long long)j * nr + i;
    const double* cf = A.coef + q;
    // 6 h D for each component (60 h D and the eighth differences for the
    // FD6+KO8 scheme)
    double D0, D1, D2, D3, E0 = 0.0, E1 = 0.0, E2 = 0.0, E3 = 0.0;
    if constexpr (SCHEME == 1) {
        fd6_ko8(sw + 0 * NW + p, D0, E0);
        fd6_ko8(sw + 1 * NW + p, D1, E1);
        fd6_ko8(sw + 2 * NW + p, D2, E2);
        fd6_ko8(sw + 3 * NW + p, D3, E3);
    } else {
        D0 = fma(6.0, sw[0 * NW + p + 2], sw[0 * NW + FO + p + 1]) - sw[0 * NW + FO + p];
        D1 = fma(6.0, sw[1 * NW + p + 2], sw[1 * NW + FO + p + 1]) - sw[1 * NW + FO + p];
        D2 = fma(6.0, sw[2 * NW + p + 3], sw[2 * NW + FO + p + 1]) - sw[2 * NW + FO + p];
        D3 = fma(6.0, sw[3 * NW + p + 3], sw[3 * NW + FO + p + 1]) - sw[3 * NW + FO + p];
    }
    const double psr = ld_state<FUSED>(A.up + q), psi = ld_state<FUSED>(A.up + P + q);
    const double pir = ld_state<FUSED>(A.up + 2 * P + q), pii = ld_state<FUSED>(A.up + 3 * P + q);
    const double cb = __ldg(cf + kCb * P);
    const double cc = HYP ? __ldg(cf + kCc * P) : cb;
    const double cKr = __ldg(cf + kCKr * P);
    const double cKi = __ldg(cf + kCKi * P), cBr = __ldg(cf + kCBr * P);
    const double cBi = __ldg(cf + kCBi * P), cCi = __ldg(cf + kCCi * P);
    double acc0, acc1, acc2, acc3;
    if (STAGE == 0) {
        acc0 = A.dt * pir; acc1 = A.dt * pii; acc2 = 0.0; acc3 = 0.0;
    } else if (STAGE == kStageScaled) {
        // alpha u^n + u_prev + dt F(u_prev): u^n enters through the first
        // multiply-add of each row, and no combination is left for the end
        const double* un = A.un + q;
        const double n0 = FUSED ? __ldcg(un) : un[0], n1 = FUSED ? __ldcg(un + P) : un[P];
        const double n2 = FUSED ? __ldcg(un + 2 * P) : un[2 * P];
        const double n3 = FUSED ? __ldcg(un + 3 * P) : un[3 * P];
        acc0 = fma(A.dt, pir, fma(A.alpha, n0, psr));
        acc1 = fma(A.dt, pii, fma(A.alpha, n1, psi));
        acc2 = fma(A.alpha, n2, pir);
        acc3 = fma(A.alpha, n3, pii);
    } else {
        acc0 = fma(A.dt, pir, psr); acc1 = fma(A.dt, pii, psi); acc2 = pir; acc3 = pii;
    }
    // Psi rows: dt (pi - b D_Psi)
    acc0 = fma(-cb, D0, acc0);
    acc1 = fma(-cb, D1, acc1);
    // pi rows: dt (c D_pi + K D_Psi + Bt pi + i Im(C) Psi + theta terms)
    acc2 = fma(cc, D2, acc2);
    acc2 = fma(cKr, D0, acc2);
    acc2 = fma(-cKi, D1, acc2);
    acc2 = fma(cBr, pir, acc2);
    acc2 = fma(-cBi, pii, acc2);
    acc2 = fma(-cCi, psi, acc2);
    acc3 = fma(cc, D3, acc3);
    acc3 = fma(cKi, D0, acc3);
    acc3 = fma(cKr, D1, acc3);
    acc3 = fma(cBi, pir, acc3);
    acc3 = fma(cBr, pii, acc3);
    acc3 = fma(cCi, psr, acc3);
#pragma unroll
    for (int k = -2; k <= 2; ++k) {
        const int jj = min(max(j + k, 0), A.nth - 1);   // weight is 0 off-grid
        const double w = __ldg(cf + (kW0 + k) * P);
        const long long qq = (long long)jj * nr + i;
        acc2 = fma(w, ld_state<FUSED>(A.up + qq), acc2);
        acc3 = fma(w, ld_state<FUSED>(A.up + P + qq), acc3);
    }
    if constexpr (THETA == TEUK_THETA_WENO5) {
        // Bth dPsi/dtheta with the WENO5 theta derivative, upwinded by the
        // sign of -Bth; the negative direction is the positive one on the
        // mirrored line, negated. Rows beyond a pole reflect with parity.
        const double cBt = __ldg(cf + kCBth * P);
        const bool pos = !(cBt > 0.0);
        double v0[6], v1[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            int jj = pos ? j + k - 3 : j + 3 - k;
            unsigned flip = 0u;
            if (jj < 0) { jj = -1 - jj; flip = A.pole_flip; }
            if (jj >= A.nth) { jj = 2 * A.nth - 1 - jj; flip = A.pole_flip; }
            const long long qq = (long long)jj * nr + i;
            v0[k] = flip_sign(ld_state<FUSED>(A.up + qq), flip);
            v1[k] = flip_sign(ld_state<FUSED>(A.up + P + qq), flip);
        }
        const double c = flip_sign(cBt, pos ? 0u : 0x80000000u);
        acc2 = fma(c, theta_weno_6hd<W>(v0, A), acc2);
        acc3 = fma(c, theta_weno_6hd<W>(v1, A), acc3);
    }
    if constexpr (SCHEME == 1) {    // Kreiss-Oliger dissipation, subtracted
        acc0 = fma(-A.ko, E0, acc0);
        acc1 = fma(-A.ko, E1, acc1);
        acc2 = fma(-A.ko, E2, acc2);
        acc3 = fma(-A.ko, E3, acc3);
    }
    if (STAGE == 2 || STAGE == 3) {
        const double* un = A.un + q;
        const double n0 = FUSED ? __ldcg(un) : un[0], n1 = FUSED ? __ldcg(un + P) : un[P];
        const double n2 = FUSED ? __ldcg(un + 2 * P) : un[2 * P];
        const double n3 = FUSED ? __ldcg(un + 3 * P) : un[3 * P];
        acc0 = fma(A.beta, acc0, A.alpha * n0);
        acc1 = fma(A.beta, acc1, A.alpha * n1);
        acc2 = fma(A.beta, acc2, A.alpha * n2);
        acc3 = fma(A.beta, acc3, A.alpha * n3);
    }
    out[0] = acc0; out[1] = acc1; out[2] = acc2; out[3] = acc3;
}

// Phase 1 at one flat index of a warp's segment: the first difference
// d_k (component c, k = i0-HALO ..) of row `row` into the warp's block sw
// (ghosts: edge copies, d = 0; on the hyperboloidal slices the quartic
// through the five edge nodes).
template <int HALO, int ND, int NW, bool HYP, bool FUSED>
__device__ __forceinline__ void first_difference(const StageArgs& A, double* sw, long long row,
                                                 int i0, int c, int k) {
    const int nr = A.nr;
    const int g = i0 - HALO + k;
    const double* f = A.up + c * A.plane + row;
    double v;
    if (HYP && (g < 0 || g >= nr - 1)) {
        // nodes beyond nr-1+HALO feed no stored node
        v = g + 1 <= nr - 1 + HALO
                ? ghost_value<FUSED>(f, nr, g + 1) - ghost_value<FUSED>(f, nr, g)
                : 0.0;
    } else {
        const int ia = min(max(g, 0), nr - 1), ib = min(max(g + 1, 0), nr - 1);
        v = ld_state<FUSED>(f + ib) - ld_state<FUSED>(f + ia);
    }
    sw[c * NW + k] = v;
}

// Phase 4: nodes i = i0 .. i0+SEG-1 of row j (two per lane and iteration
// when SEG = 64, computed side by side; the second node's loads use a clamped
// index and its store is predicated).
template <int W, int STAGE, int THETA, class G, int SCHEME, bool HYP, bool FUSED>
__device__ __forceinline__ void node_phase(const StageArgs& A, const double* sw, int lane, int j,
                                           int i0) {
    constexpr int SEG = G::SEG;
    const int nr = A.nr;
    const long long row = (long long)j * nr;
    for (int p = lane; p < SEG; p += 64) {
        double ua[4], ub[4];
        node_update<W, STAGE, THETA, G, SCHEME, HYP, FUSED>(A, sw, j, i0, p, ua);
        const bool has_b = p + 32 < SEG;
        if (has_b) node_update<W, STAGE, THETA, G, SCHEME, HYP, FUSED>(A, sw, j, i0, p + 32, ub);
        const long long P = A.plane;
        if (i0 + p < nr) {
            const long long q = row + i0 + p;
            A.out[q] = ua[0]; A.out[P + q] = ua[1]; A.out[2 * P + q] = ua[2]; A.out[3 * P + q] = ua[3];
        }
        if (has_b && i0 + p + 32 < nr) {
            const long long q = row + i0 + p + 32;
            A.out[q] = ub[0]; A.out[P + q] = ub[1]; A.out[2 * P + q] = ub[2]; A.out[3 * P + q] = ub[3];
        }
    }
}

// One warp's work (the FD6 + KO8 scheme): segment seg_blk (nodes
// seg_blk*SEG ..) of theta row j; sw is the warp's shared-memory block. The
// scheme needs only the first differences (4 x (SEG + 8) of them, whole
// 32-lane iterations).
template <int STAGE, int SEGV, bool HYP>
__device__ __forceinline__ void process_segment_fd6(const StageArgs& A, double* sw, int lane, int j,
                                                    int seg_blk) {
    using G = GeoFD<SEGV>;
    constexpr int ND = G::ND, NW = G::NW;
    const int i0 = seg_blk * G::SEG;
    const long long row = (long long)j * A.nr;
    for (int idx = lane; idx < 4 * ND; idx += 32) {
        const int c = idx / ND;
        first_difference<4, ND, NW, HYP, false>(A, sw, row, i0, c, idx - c * ND);
    }
    __syncwarp();
    node_phase<TEUK_W_FP64, STAGE, TEUK_THETA_CENTERED4, G, 1, HYP, false>(A, sw, lane, j, i0);
}

// One work item of the WENO5 scheme: radial segment seg_blk of the rows
// j0 .. j0+nrows-1 (nrows <= WARPS; warp w owns row j0 + w and the block
// sm + w * 4 NW of shared memory). The three halo phases (first differences,
// third differences s_k = d_{k-1} - 2 d_k + d_{k+1}, interface flux terms)
// are shared by all threads of the block as one flat list per phase over
// the item's rows, so that only the block's last 32-lane iteration of a
// phase can leave lanes idle (a warp doing its own row alone idles 12, 20
// and 28 lanes of its last iterations on 32-node segments). Every thread of
// the block must call this (it contains block barriers); the node phase is
// the warp's own.
template <int W, int STAGE, int THETA, int SEGV, bool HYP = false, bool FUSED = false>
__device__ __forceinline__ void process_item(const StageArgs& A, double* sm, int j0, int nrows,
                                             int seg_blk) {
    using G = Geo<SEGV>;
    constexpr int ND = G::ND, NS = G::NS, NF = G::NF, NW = G::NW;
    const int i0 = seg_blk * G::SEG;
    const int t = threadIdx.x;
    const int warp = t >> 5, lane = t & 31;
    for (int idx = t; idx < nrows * 4 * ND; idx += WARPS * 32) {
        const int r = idx / (4 * ND), e = idx - r * (4 * ND);
        const int c = e / ND;
        first_difference<3, ND, NW, HYP, FUSED>(A, sm + r * (4 * NW), (long long)(j0 + r) * A.nr,
                                                i0, c, e - c * ND);
    }
    __syncthreads();
    for (int idx = t; idx < nrows * 4 * NS; idx += WARPS * 32) {
        const int r = idx / (4 * NS), e = idx - r * (4 * NS);
        const int c = e / NS, k = e - c * NS;
        const double* dl = sm + r * (4 * NW) + c * NW;
        sm[r * (4 * NW) + c * NW + ND + k] = fma(-2.0, dl[k + 1], dl[k] + dl[k + 2]);
    }
    __syncthreads();
    for (int idx = t; idx < nrows * 4 * NF; idx += WARPS * 32) {
        const int r = idx / (4 * NF), e = idx - r * (4 * NF);
        const int c = e / NF;
        double* sw = sm + r * (4 * NW);
        sw[c * NW + ND + NS + (e - c * NF)] = interface_flux<W, G>(sw, e, A);
    }
    __syncthreads();
    if (warp < nrows)
        node_phase<W, STAGE, THETA, G, 0, HYP, FUSED>(A, sm + warp * (4 * NW), lane, j0 + warp, i0);
}

// Programmatic dependent launch (PTX griddepcontrol, sm_90 and later): the
// block first waits until the previous kernel of the stream has completed and
// its writes are visible (a no-op when the launch did not ask for early
// scheduling), then lets the next kernel's blocks be scheduled onto SMs this
// grid no longer fills; they in turn wait here for this grid to complete.
__device__ __forceinline__ void dependent_launch_gate() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Single evolution: blockIdx.x = segment, blockIdx.y = block of WARPS rows.
template <int W, int STAGE, int THETA, bool HYP = false>
__global__ void TEUK_BOUNDS stage_kernel(const StageArgs A) {
    constexpr int SEGV = Seg<W>::value;
    __shared__ double sm[WARPS][4 * Geo<SEGV>::NW];
    dependent_launch_gate();
    const int j0 = blockIdx.y * WARPS;
    process_item<W, STAGE, THETA, SEGV, HYP>(A, &sm[0][0], j0, min(WARPS, A.nth - j0), blockIdx.x);
}

// FD6 + KO8 comparison scheme (Sec. 3.1.1), single evolution, centred theta;
// HYP as for stage_kernel.
template <int STAGE, bool HYP = false>
__global__ void TEUK_BOUNDS fd6_stage_kernel(const StageArgs A) {
    constexpr int SEGV = 32;
    __shared__ double sm[WARPS][4 * GeoFD<SEGV>::NW];
    dependent_launch_gate();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.y * WARPS + warp;
    if (j >= A.nth) return;
    process_segment_fd6<STAGE, SEGV, HYP>(A, sm[warp], lane, j, blockIdx.x);
}

// Batched evolutions: one work item is a block of WARPS rows x one segment of
// one evolution; items of all evolutions are numbered consecutively
// (item0[k] = first item of evolution k) and a persistent grid walks them.
// All evolutions advance the same Runge-Kutta stage in one launch; the launch
// boundary is the stage barrier.
struct BatchDesc {
    const double* coef;
    double* u;            // state
    double* w;            // two stage buffers (4 planes each)
    int nr, nth, nseg;
    long long plane;
    long long item0;      // first work item of this evolution
    double dt, eps4;
    int eps_exp, eps_pow2;
    unsigned eps_mant, pole_flip;
};

template <int W, int STAGE, int THETA, int SEGV, bool HYP = false>
__global__ void TEUK_BOUNDS batch_stage_kernel(const BatchDesc* __restrict__ D, int n,
                                               long long items) {
    __shared__ double sm[WARPS][4 * Geo<SEGV>::NW];
    // The member of item `it` is the last k with item0 <= it. A block's items
    // rise, so its member index only moves forward: usually zero or one load
    // per item instead of a binary search (measured: 2% faster on 64 members).
    int lo = 0;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        while (lo + 1 < n && D[lo + 1].item0 <= it) ++lo;
        const BatchDesc& d = D[lo];
        const long long local = it - d.item0;
        const int seg_blk = (int)(local % d.nseg);
        const int j0 = (int)(local / d.nseg) * WARPS;
        {
            StageArgs A;
            A.coef = d.coef;
            A.nr = d.nr; A.nth = d.nth; A.plane = d.plane;
            A.dt = d.dt; A.eps4 = d.eps4;
            A.eps_exp = d.eps_exp; A.eps_pow2 = d.eps_pow2; A.eps_mant = d.eps_mant;
            A.pole_flip = d.pole_flip;
            A.ko = 0.0;
            double* w1 = d.w;
            double* w2 = d.w + 4 * d.plane;
            // the step's second stage in its scaled form (kStageScaled)
            if (STAGE == 1) { A.un = nullptr; A.up = d.u; A.out = w1; A.alpha = 0.0; A.beta = 1.0; }
            if (STAGE == 2) { A.un = d.u; A.up = w1; A.out = w2; A.alpha = kScaledAlpha; A.beta = 1.0; }
            if (STAGE == 3) {
                A.un = d.u; A.up = w2; A.out = d.u; A.alpha = 1.0 / 3.0; A.beta = kThirdBetaScaled;
                eps_times_16(A);
            }
            process_item<W, STAGE == 2 ? kStageScaled : STAGE, THETA, SEGV, HYP>(
                A, &sm[0][0], j0, min(WARPS, d.nth - j0), seg_blk);
        }
        __syncthreads();            // the next item's halo phases overwrite sm
    }
}

// Launch with programmatic stream serialisation when the grid fills at least
// one wave of resident blocks: the kernel may then be scheduled onto the SMs
// its predecessor's last wave leaves free, before that predecessor completes;
// its dependent_launch_gate keeps every memory access after the completion.
// A grid smaller than one wave is launched plainly: every block of such a
// predecessor starts at once and releases its dependents immediately, so they
// would crowd onto the few free slots unevenly (measured: 8% slower on the
// binary64-weight kernel at 2048 x 128, against 3% faster at 1.7 waves).
inline cudaError_t launch_early(void (*kernel)(StageArgs), dim3 grid, dim3 block,
                                const StageArgs& A, cudaStream_t st) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel,
                                                          (int)(block.x * block.y * block.z), 0);
    if (e != cudaSuccess) return e;
    if ((long long)grid.x * grid.y * grid.z < (long long)sms * per_sm) {
        kernel<<<grid, block, 0, st>>>(A);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, A);
}

template <int W, int THETA, bool HYP = false>
cudaError_t launch_stage_wt(const StageArgs& A, int stage, cudaStream_t st) {
    constexpr int SEG = Seg<W>::value;
    dim3 grid((A.nr + SEG - 1) / SEG, (A.nth + WARPS - 1) / WARPS);
    dim3 block(WARPS * 32);
    switch (stage) {
    case 0: return launch_early(stage_kernel<W, 0, THETA, HYP>, grid, block, A, st);
    case 1: return launch_early(stage_kernel<W, 1, THETA, HYP>, grid, block, A, st);
    case kStageScaled:
        return launch_early(stage_kernel<W, kStageScaled, THETA, HYP>, grid, block, A, st);
    default: return launch_early(stage_kernel<W, 2, THETA, HYP>, grid, block, A, st);
    }
}


template <int W, int THETA, int SEGV, bool HYP>
cudaError_t launch_batch_wts(int stage, const BatchDesc* d, int n, long long items, int grid,
                             cudaStream_t st) {
    const dim3 block(WARPS * 32);
    switch (stage) {
    case 1: batch_stage_kernel<W, 1, THETA, SEGV, HYP><<<grid, block, 0, st>>>(d, n, items); break;
    case 2: batch_stage_kernel<W, 2, THETA, SEGV, HYP><<<grid, block, 0, st>>>(d, n, items); break;
    default: batch_stage_kernel<W, 3, THETA, SEGV, HYP><<<grid, block, 0, st>>>(d, n, items); break;
    }
    return cudaGetLastError();
}

template <int W, bool HYP>
cudaError_t launch_batch_w(int stage, int segv, int theta, const BatchDesc* d, int n,
                           long long items, int grid, cudaStream_t st) {
    if (theta == TEUK_THETA_WENO5)
        return segv == 64
                   ? launch_batch_wts<W, TEUK_THETA_WENO5, 64, HYP>(stage, d, n, items, grid, st)
                   : launch_batch_wts<W, TEUK_THETA_WENO5, 32, HYP>(stage, d, n, items, grid, st);
    return segv == 64
               ? launch_batch_wts<W, TEUK_THETA_CENTERED4, 64, HYP>(stage, d, n, items, grid, st)
               : launch_batch_wts<W, TEUK_THETA_CENTERED4, 32, HYP>(stage, d, n, items, grid, st);
}

// ---------------------------------------------------------------------------
// Fused persistent step kernel: all SSP-RK(3,3) stages of `steps` steps of one
// evolution in a single launch.
//
// A work item is a block of WARPS theta rows x one radial segment (the tile of
// one stage_kernel block); epoch e = 3 (step) + (stage - 1). Tickets
// t = e * items + item are handed out in increasing order: block b starts with
// ticket b and takes each later one from an atomic counter (plus the grid
// size) as soon as it reads its current one. An item of epoch e reads, through its radial (+-3 nodes) and theta
// (+-2 rows, +-3 with theta-WENO, reflected at the poles) stencils, only
// nodes of its own and the eight neighbouring items, so it may start as soon
// as those nine have completed epoch e - 1. That also orders every overwrite
// after the reads of the old value: the stage buffer w1 (written in stage 1)
// was last read by stage 2 of the previous step at the neighbours, w2 by
// stage 3 at the neighbours, and u (written in stage 3) by stage 1 at the
// neighbours and stage 2 at the item itself, all of which precede epoch e - 1
// of the neighbours in the dependency chain. No block waits for a ticket above
// its own, and every ticket below it is held by a running block, so the
// smallest unfinished ticket can always proceed: the launch needs no
// co-residency guarantee.
//
// Completion of epoch e at an item is published as flags[item] = base + e + 1
// (a block barrier, then a release store at gpu scope by one thread); a block
// waits for flags[neighbour] >= base + e with acquire loads, then a block
// barrier. The host advances `base` by
// the launch's epochs after every launch, so flags left by earlier launches
// never satisfy a wait and nothing is cleared between launches. Each wait is
// bounded by wait_ns of %globaltimer; when it runs out the block records the
// item and epoch in host-mapped memory, raises `abort`, and every block stops
// at its next spin, so the launch ends and the host reports TEUK_ERR_TIMEOUT.
// The ticket counter and the abort word come in two copies used by alternate
// launches (`parity`, kept by the host): block 0 of a launch zeroes the other
// copy, which the previous launch has finished with and the next one will
// use, so no block has to meet the others at the end of a launch.
// ---------------------------------------------------------------------------
struct FusedCtl {
    unsigned long long ticket[2];   // next ticket, one per launch parity
    int abort[2];                   // a wait ran out: every block stops
};

struct FusedArgs {
    StageArgs A;                 // grid, coefficients, weights' epsilon, pole parity, dt
    double* u;                   // state u^n (updated in place by stage 3)
    double* w1;                  // stage buffers
    double* w2;
    int nseg, nrb;               // radial segments, theta-row blocks
    int items;                   // nseg * nrb
    int epochs;                  // 3 x steps
    unsigned* flags;             // [items]
    FusedCtl* ctl;
    unsigned base;               // epoch base of this launch
    int parity;                  // which ticket counter and abort word it uses
    int* err_host;               // host-mapped {code, epoch, item}; code 1 = timeout
    unsigned long long wait_ns;  // bound of one dependency wait
    int withhold;                // test hook: item 0 does not publish epoch 0
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Lanes 0..8 of warp 0: wait until neighbour (rb + lane/3 - 1, sg + lane%3 - 1)
// has completed epoch e - 1. The first acquire load usually finds it done;
// only a wait that has to spin also watches the abort word and the time
// bound. Returns false (warp-uniform) if a wait ran out or another block
// raised abort. (A block whose neighbourhoods keep being ready after an abort
// runs on to the end of its tickets: every other block stops at its next
// spin, so the launch still ends.)
__device__ __forceinline__ bool wait_neighbours(const FusedArgs& F, unsigned base, int e, int rb,
                                                int sg, int item, int lane) {
    int ok = 1;
    if (e > 0 && lane < 9) {
        const int r = rb + lane / 3 - 1, g = sg + lane % 3 - 1;
        if (r >= 0 && r < F.nrb && g >= 0 && g < F.nseg) {
            const unsigned* f = F.flags + (long long)r * F.nseg + g;
            const unsigned need = base + (unsigned)e;
            if ((int)(ld_acquire_u32(f) - need) < 0) {
                int* abort = &F.ctl->abort[F.parity];
                const unsigned long long t0 = global_ns();
                for (;;) {
                    if (*(volatile int*)abort) { ok = 0; break; }
                    if (global_ns() - t0 > F.wait_ns) {
                        ok = 0;
                        if (atomicCAS(abort, 0, 1) == 0) {
                            volatile int* eh = F.err_host;
                            eh[1] = e;
                            eh[2] = item;
                            __threadfence_system();
                            eh[0] = 1;
                        }
                        break;
                    }
                    __nanosleep(100);
                    if ((int)(ld_acquire_u32(f) - need) >= 0) break;
                }
            }
        }
    }
    return __all_sync(0xffffffffu, ok) != 0;
}

template <int W, int THETA, bool HYP, int SEGV>
__global__ void TEUK_BOUNDS fused_step_kernel(const FusedArgs F) {
    __shared__ double sm[WARPS][4 * Geo<SEGV>::NW];
    __shared__ long long s_ticket;
    __shared__ int s_go;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned base = F.base;
    const long long total = (long long)F.items * F.epochs;
    unsigned long long* counter = &F.ctl->ticket[F.parity];
    if (blockIdx.x == 0 && threadIdx.x == 0) {     // ready the other copy for the next launch
        F.ctl->ticket[1 - F.parity] = 0ULL;
        F.ctl->abort[1 - F.parity] = 0;
    }
    // first ticket: the block's own index (no atomic traffic while the whole
    // grid starts); later ones from the counter, offset by the grid size
    // first ticket: the block's own index (no atomic traffic while the whole
    // grid starts); later ones from the counter, offset by the grid size
    unsigned long long next = blockIdx.x;
    // Warp 0 takes the ticket (lane 0 also asks the counter for the one after
    // it) and waits for the item's neighbourhood; one block barrier then hands
    // the ticket and the outcome of the wait to the other warps.
    for (;;) {
        if (warp == 0) {
            long long tk = 0;
            if (lane == 0) {
                tk = (long long)next;
                if (tk < total) next = gridDim.x + atomicAdd(counter, 1ULL);
            }
            tk = __shfl_sync(0xffffffffu, tk, 0);
            bool go = false;
            if (tk < total) {
                const int e0 = (int)(tk / F.items);
                const int it0 = (int)(tk - (long long)e0 * F.items);
                const int rb0 = it0 / F.nseg;
                go = wait_neighbours(F, base, e0, rb0, it0 - rb0 * F.nseg, it0, lane);
            }
            if (lane == 0) { s_ticket = tk; s_go = go; }
        }
        __syncthreads();
        const long long t = s_ticket;
        if (t >= total || !s_go) break;
        const int e = (int)(t / F.items);
        const int item = (int)(t - (long long)e * F.items);
        const int rb = item / F.nseg, sg = item - rb * F.nseg;
        const int stage = e % 3 + 1;
        StageArgs A = F.A;
        // the second stage in its scaled form (kStageScaled), as in the stage launches
        if (stage == 1) { A.un = nullptr; A.up = F.u; A.out = F.w1; A.alpha = 0.0; A.beta = 1.0; }
        if (stage == 2) { A.un = F.u; A.up = F.w1; A.out = F.w2; A.alpha = kScaledAlpha; A.beta = 1.0; }
        if (stage == 3) {
            A.un = F.u; A.up = F.w2; A.out = F.u; A.alpha = 1.0 / 3.0; A.beta = kThirdBetaScaled;
            eps_times_16(A);
        }
        const int j0 = rb * WARPS, nrows = min(WARPS, A.nth - j0);
        if (stage == 1)
            process_item<W, 1, THETA, SEGV, HYP, true>(A, &sm[0][0], j0, nrows, sg);
        else if (stage == 2)
            process_item<W, kStageScaled, THETA, SEGV, HYP, true>(A, &sm[0][0], j0, nrows, sg);
        else
            process_item<W, 2, THETA, SEGV, HYP, true>(A, &sm[0][0], j0, nrows, sg);
        // Every thread's stores of this item precede the barrier; thread 0's
        // release store at gpu scope after it makes them visible to any block
        // that acquires the flag (a release is cumulative over what the
        // barrier ordered before it).
        __syncthreads();
        if (threadIdx.x == 0 && !(F.withhold && e == 0 && item == 0))
            st_release_u32(F.flags + item, base + (unsigned)e + 1u);
    }
}

// Radial segment of the fused kernel: 64 nodes with binary64 weights; with
// reduced-precision weights 32, or 64 on grids with at least kSeg64Items
// 64-node work items per stage (three waves of resident blocks and more: the
// halo phases idle fewer lanes per node, measured 6% faster on the
// 8192 x 256 and 16384 x 64 grids, while the 2048 x 128 grid needs the 32-node
// items to fill the device).
constexpr long long kSeg64Items = 3 * 8 * 152;
inline int fused_seg(int wprec, int nr, int ntheta) {
    if (wprec == TEUK_W_FP64) return 64;
    const long long items64 = (long long)((nr + 63) / 64) * ((ntheta + WARPS - 1) / WARPS);
    return items64 >= kSeg64Items ? 64 : 32;
}

template <int W, int THETA, bool HYP, int SEGV>
cudaError_t launch_fused_wts(const FusedArgs& F, int blocks_per_sm_cap, cudaStream_t st) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, fused_step_kernel<W, THETA, HYP, SEGV>, WARPS * 32, 0);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm_cap > 0) per_sm = std::min(per_sm, blocks_per_sm_cap);
    const int grid = (int)std::max(1LL, std::min<long long>((long long)sms * per_sm, F.items));
    fused_step_kernel<W, THETA, HYP, SEGV><<<grid, WARPS * 32, 0, st>>>(F);
    return cudaGetLastError();
}

template <int W, int THETA, bool HYP>
cudaError_t launch_fused_wt(const FusedArgs& F, int seg, int cap, cudaStream_t st) {
    if constexpr (W == TEUK_W_FP64) {
        return launch_fused_wts<W, THETA, HYP, 64>(F, cap, st);
    } else {
        return seg == 64 ? launch_fused_wts<W, THETA, HYP, 64>(F, cap, st)
                         : launch_fused_wts<W, THETA, HYP, 32>(F, cap, st);
    }
}

// Resident blocks per SM of the fused kernel (the same for both segment
// lengths: 64 registers and at most 26 KB of shared memory per block).
template <bool HYP>
cudaError_t fused_occupancy_h(int wprec, int theta, int* per_sm) {
    const bool tw = theta == TEUK_THETA_WENO5;
    const int nt = WARPS * 32;
    switch (wprec) {
    case TEUK_W_FP64:
        return tw ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                        per_sm, fused_step_kernel<TEUK_W_FP64, TEUK_THETA_WENO5, HYP, 64>, nt, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                        per_sm, fused_step_kernel<TEUK_W_FP64, TEUK_THETA_CENTERED4, HYP, 64>,
                        nt, 0);
    default:
        return tw ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                        per_sm, fused_step_kernel<TEUK_W_FP32, TEUK_THETA_WENO5, HYP, 64>, nt, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                        per_sm, fused_step_kernel<TEUK_W_FP32, TEUK_THETA_CENTERED4, HYP, 64>,
                        nt, 0);
    }
}

template <bool HYP>
cudaError_t launch_fused_h(const FusedArgs& F, int wprec, int theta, int seg, int cap,
                           cudaStream_t st) {
    const bool tw = theta == TEUK_THETA_WENO5;
    switch (wprec) {
    case TEUK_W_FP64:
        return tw ? launch_fused_wt<TEUK_W_FP64, TEUK_THETA_WENO5, HYP>(F, seg, cap, st)
                  : launch_fused_wt<TEUK_W_FP64, TEUK_THETA_CENTERED4, HYP>(F, seg, cap, st);
    case TEUK_W_FP32:
        return tw ? launch_fused_wt<TEUK_W_FP32, TEUK_THETA_WENO5, HYP>(F, seg, cap, st)
                  : launch_fused_wt<TEUK_W_FP32, TEUK_THETA_CENTERED4, HYP>(F, seg, cap, st);
    case TEUK_W_FP16:
        return tw ? launch_fused_wt<TEUK_W_FP16, TEUK_THETA_WENO5, HYP>(F, seg, cap, st)
                  : launch_fused_wt<TEUK_W_FP16, TEUK_THETA_CENTERED4, HYP>(F, seg, cap, st);
    default:
        return tw ? launch_fused_wt<TEUK_W_BF16, TEUK_THETA_WENO5, HYP>(F, seg, cap, st)
                  : launch_fused_wt<TEUK_W_BF16, TEUK_THETA_CENTERED4, HYP>(F, seg, cap, st);
    }
}

// teuk_stage.cu: the StageArgs fields that depend on p alone, and the work
// items of the fused step kernel (radial segments x theta-row blocks).
void stage_args_common(StageArgs& A, const teuk_params& p);
void fused_layout(const teuk_params& p, int* nseg, int* nrb);
// teuk_fused.cu / teuk_fused_hyp.cu: fused step launches per coordinate system.
cudaError_t launch_fused_rstar(const FusedArgs& F, int wprec, int theta, int seg, int cap,
                               cudaStream_t st);
cudaError_t launch_fused_hyp(const FusedArgs& F, int wprec, int theta, int seg, int cap,
                             cudaStream_t st);
cudaError_t fused_occupancy_rstar(int wprec, int theta, int* per_sm);
cudaError_t fused_occupancy_hyp(int wprec, int theta, int* per_sm);

// Hyperboloidal-slice kernels, single evolution and batches (teuk_stage_hyp.cu).
cudaError_t launch_stage_hyp(const StageArgs& A, int wprec, int theta, int stage,
                             cudaStream_t st);
cudaError_t launch_batch_stage_hyp(int wprec, int theta, int stage, int segv,
                                   const BatchDesc* d, int n, long long items, int grid,
                                   cudaStream_t st);

}  // namespace teuk
