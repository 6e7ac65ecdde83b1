// Internal declarations shared by the host (.cpp) and device (.cu) parts of
// the library. Not part of the public ABI.
#pragma once
#include <cstdint>
#include <exception>
#include <new>
#include <string>
#include "../../include/teuk.h"

namespace teuk {

// Number of coefficient planes per grid node: 11; 12 with the theta-WENO
// option (dt Bth / (6 dtheta)); 13 on the hyperboloidal slices (the pi rows'
// speed, plane 12; plane 11 is then unused and holds zeros).
constexpr int kCoefPlanes = 11;
inline int coef_planes(const teuk_params& p) {
    if (p.coords == TEUK_COORDS_HYPERBOLOIDAL) return 13;
    return p.theta_mode == TEUK_THETA_WENO5 ? 12 : kCoefPlanes;
}
// Plane order (all pre-multiplied by dt; 60h in place of 6h for the FD6 + KO8
// scheme):
//   0 cb   = b/(6h)          1 cKr = Re K/(6h)     2 cKi = Im K/(6h)
//   3 cBr  = Re Bt           4 cBi = Im Bt         5 cCi = Im C
//   6..10  theta stencil weights on Psi rows j-2, j-1, j, j+1, j+2
//          (Ath and Bth centred differences, Re C on the centre, pole parity
//          folded in).
//   11     (theta-WENO option) dt Bth / (6 dtheta); the five stencil planes
//          then hold only the second derivative and Re C.
//   12     (hyperboloidal slices) cc = c/(6h), the pi rows' speed; in r* the
//          pi rows use cb (c = b).
enum CoefPlane { kCb = 0, kCKr, kCKi, kCBr, kCBi, kCCi, kWm2, kWm1, kW0, kWp1, kWp2, kCBth, kCc };

// Forward-Euler step of one stage of p's integrator: dt for SSP-RK(3,3),
// dt/6 for SSP-RK(10,4).
inline double stage_step(const teuk_params& p, double dt) {
    return p.rk == TEUK_RK_SSP104 ? dt / 6.0 : dt;
}

teuk_status fail(teuk_status st, const std::string& msg);
void clear_error();
// TEUK_ERR_HOST with "what: why"; allocates nothing that can throw out of it.
teuk_status fail_host(const char* what, const char* why) noexcept;

// Runs body() (returning teuk_status) and turns a C++ exception escaping it
// (a failed host allocation, a thread that could not start) into
// TEUK_ERR_HOST, so that no exception crosses the C ABI.
template <class F>
teuk_status guarded(const char* what, F&& body) noexcept {
    try {
        return body();
    } catch (const std::bad_alloc&) {
        return fail_host(what, "host memory exhausted");
    } catch (const std::exception& ex) {
        return fail_host(what, ex.what());
    } catch (...) {
        return fail_host(what, "unknown host exception");
    }
}

// r(r*) and the continuum coefficients at one node, real arithmetic.
struct PointCoef {
    double b, Kr, Ki, Btr, Bti, Cr, Ci, Ath, Bth;
    double c;   // the pi rows' speed (c = b in r*)
};
double r_of_rstar(double rstar, double M, double a, double* x_out);
PointCoef point_coefficients(double rstar, double theta, const teuk_params& p);
PointCoef point_coefficients_rx(double r, double x, double theta, const teuk_params& p);
PointCoef point_coefficients_hyp(double rho, double theta, const teuk_params& p);
double horizon_rho(double M, double a, double S);
// p with a hyperboloidal range given as [0, 0] replaced by [rho_+, S].
teuk_params resolve_params(const teuk_params& p);

double swsh(int s, int l, int m, double theta);
uint64_t splitmix64(uint64_t& state);

// Batched evolutions: pointers and step of one member.
struct BatchEvo {
    teuk_params p;
    const double* coef;
    double* u;
    double* w;
    double dt;
};
long long batch_items(const teuk_params& p, int segv);
size_t batch_desc_bytes(int n);

}  // namespace teuk

#ifdef __CUDACC__
#include <cuda_runtime.h>
namespace teuk {
// kind 4 (kStageScaled): u_out = alpha u_n + u_prev + h F(u_prev), the scaled
// second stage of the WENO5 SSP-RK(3,3) step; eps_log2 scales the WENO
// epsilon by 2^eps_log2 (4 for the stage after it).
constexpr int kStageScaled = 4;
cudaError_t launch_stage_ab(const teuk_params& p, const double* coef, const double* un,
                            const double* up, double* out, int kind, double h, double alpha,
                            double beta, cudaStream_t st, int eps_log2 = 0);
cudaError_t launch_rk104_combine(const double* u, const double* v, double* q, double* u5,
                                 long long n, cudaStream_t st);
cudaError_t upload_batch_desc(const BatchEvo* evos, int n, int segv, void* d_desc,
                              long long* items_out, cudaStream_t st);
cudaError_t launch_batch_stage(int wprec, int theta, bool hyp, int stage, int segv,
                               const void* d_desc, int n, long long items, int grid,
                               cudaStream_t st);
// Scheduling state of the fused step kernel held by a handle.
struct FusedRun {
    unsigned* flags;             // fused_items(p) completion flags (device, zeroed once)
    void* ctl;                   // fused_ctl_bytes() control block (device, zeroed once)
    int* err_dev;                // device address of 3 host-mapped error words
    unsigned long long wait_ns;  // bound of one device-side wait
    int withhold;                // test hook: the first item withholds its first flag
    int blocks_per_sm;           // 0: as many as fit
    unsigned base;               // epochs completed by earlier launches (mod 2^32)
    int parity;                  // launches so far, mod 2
};
cudaError_t launch_fused_step(const teuk_params& p, const double* coef, double dt, double* u,
                              double* w, int steps, const FusedRun& run, cudaStream_t st);
size_t fused_items(const teuk_params& p);
size_t fused_ctl_bytes();
// Blocks of the fused kernel of p that fit on the device at once.
cudaError_t fused_resident_blocks(const teuk_params& p, long long* blocks);
}  // namespace teuk
#endif
