// Launch code of the fused stage kernel (teuk_stage_kernels.cuh) for r*
// grids and batches, the FD6 + KO8 comparison scheme, and the SSP-RK(10,4)
// combination kernel; the hyperboloidal instantiations live in
// teuk_stage_hyp.cu.
#include "teuk_stage_kernels.cuh"

#include <cmath>

namespace teuk {

// eps = m 2^E with m in [1, 2): E, whether m == 1, and the binary32 bits of m
// rounded (to nearest, ties to even) to the weight format's significand.
static void eps_parts(double eps, int wprec, int* E, int* pow2, unsigned* mant_bits) {
    uint64_t b;
    std::memcpy(&b, &eps, sizeof b);
    *E = (int)((b >> 52) & 0x7ff) - 1023;
    const uint64_t m = b & 0xfffffffffffffULL;
    *pow2 = m == 0;
    const int P = wprec == TEUK_W_FP16 ? 11 : (wprec == TEUK_W_BF16 ? 8 : 24);
    const int D = 53 - P;
    uint64_t kept = m >> D;
    const uint64_t dropped = m & ((1ULL << D) - 1), half = 1ULL << (D - 1);
    if (dropped > half || (dropped == half && (kept & 1))) kept += 1;
    // exponent field 127 (value in [1, 2)); a carry makes it exactly 2
    *mant_bits = (127u << 23) + (unsigned)(kept << (24 - P));
}

template <int W>
static cudaError_t launch_stage_w(const StageArgs& A, int stage, int theta, cudaStream_t st) {
    return theta == TEUK_THETA_WENO5 ? launch_stage_wt<W, TEUK_THETA_WENO5>(A, stage, st)
                                     : launch_stage_wt<W, TEUK_THETA_CENTERED4>(A, stage, st);
}

static unsigned pole_flip_of(const teuk_params& p) {
    return ((p.m + p.s) % 2 == 0) ? 0u : 0x80000000u;
}

// The fields of StageArgs that come from p alone (grid, epsilon, pole parity);
// the pointers, step and stage weights are the caller's.
void stage_args_common(StageArgs& A, const teuk_params& p) {
    A.nr = p.nr;
    A.nth = p.ntheta;
    A.plane = (long long)p.nr * p.ntheta;
    A.eps4 = 4.0 * p.eps;
    eps_parts(p.eps, p.wprec, &A.eps_exp, &A.eps_pow2, &A.eps_mant);
    A.pole_flip = pole_flip_of(p);
    A.ko = 0.0;
}

void fused_layout(const teuk_params& p, int* nseg, int* nrb) {
    const int seg = fused_seg(p.wprec, p.nr, p.ntheta);
    *nseg = (p.nr + seg - 1) / seg;
    *nrb = (p.ntheta + WARPS - 1) / WARPS;
}

cudaError_t launch_stage(const teuk_params& p, const double* coef, const double* un,
                         const double* up, double* out, int stage, double dt,
                         cudaStream_t st) {
    const double alpha = stage == 2 ? 0.75 : (stage == 3 ? 1.0 / 3.0 : 0.0);
    const double beta = stage == 2 ? 0.25 : (stage == 3 ? 2.0 / 3.0 : 1.0);
    return launch_stage_ab(p, coef, un, up, out, stage, stage_step(p, dt), alpha, beta, st);
}

// kind 0: u_out = h F(u_prev); kind 1: u_out = u_prev + h F(u_prev);
// kind 2, 3: u_out = alpha u_n + beta (u_prev + h F(u_prev));
// kind kStageScaled (WENO5 only): u_out = alpha u_n + u_prev + h F(u_prev).
// eps_log2: the WENO epsilon times 2^eps_log2.
cudaError_t launch_stage_ab(const teuk_params& p, const double* coef, const double* un,
                            const double* up, double* out, int kind, double h, double alpha,
                            double beta, cudaStream_t st, int eps_log2) {
    const int stage = kind == kStageScaled ? kStageScaled : (kind > 2 ? 2 : kind);
    StageArgs A;
    stage_args_common(A, p);
    A.coef = coef; A.un = un; A.up = up; A.out = out;
    A.dt = h;
    A.alpha = alpha;
    A.beta = beta;
    A.eps4 = std::ldexp(A.eps4, eps_log2);
    A.eps_exp += eps_log2;
    if (p.scheme == TEUK_SCHEME_FD6_KO8) {
        if (stage == kStageScaled) return cudaErrorInvalidValue;
        A.ko = h * p.ko_sigma / (256.0 * ((p.rstar_max - p.rstar_min) / (p.nr - 1)));
        dim3 grid((A.nr + 31) / 32, (A.nth + WARPS - 1) / WARPS), block(WARPS * 32);
        if (p.coords == TEUK_COORDS_HYPERBOLOIDAL) {
            switch (stage) {
            case 0: return launch_early(fd6_stage_kernel<0, true>, grid, block, A, st);
            case 1: return launch_early(fd6_stage_kernel<1, true>, grid, block, A, st);
            default: return launch_early(fd6_stage_kernel<2, true>, grid, block, A, st);
            }
        }
        switch (stage) {
        case 0: return launch_early(fd6_stage_kernel<0>, grid, block, A, st);
        case 1: return launch_early(fd6_stage_kernel<1>, grid, block, A, st);
        default: return launch_early(fd6_stage_kernel<2>, grid, block, A, st);
        }
    }
    const int th = p.theta_mode;
    if (p.coords == TEUK_COORDS_HYPERBOLOIDAL) return launch_stage_hyp(A, p.wprec, th, stage, st);
    switch (p.wprec) {
    case TEUK_W_FP64: return launch_stage_w<TEUK_W_FP64>(A, stage, th, st);
    case TEUK_W_FP32: return launch_stage_w<TEUK_W_FP32>(A, stage, th, st);
    case TEUK_W_FP16: return launch_stage_w<TEUK_W_FP16>(A, stage, th, st);
    default: return launch_stage_w<TEUK_W_BF16>(A, stage, th, st);
    }
}

// `steps` SSP-RK(3,3) steps of p in one launch of the fused step kernel
// (WENO5 radial scheme). w holds the two stage buffers (8 planes); flags,
// ctl and err_dev are the handle's scheduling state (fused_items(p) flags, a
// zeroed FusedCtl, host-mapped error words).
cudaError_t launch_fused_step(const teuk_params& p, const double* coef, double dt, double* u,
                              double* w, int steps, const FusedRun& run, cudaStream_t st) {
    FusedArgs F;
    stage_args_common(F.A, p);
    F.A.coef = coef;
    F.A.un = nullptr; F.A.up = nullptr; F.A.out = nullptr;
    F.A.dt = stage_step(p, dt);
    F.A.alpha = 0.0; F.A.beta = 1.0;
    const size_t n = 4 * (size_t)p.nr * p.ntheta;
    F.u = u; F.w1 = w; F.w2 = w + n;
    fused_layout(p, &F.nseg, &F.nrb);
    F.items = F.nseg * F.nrb;
    F.epochs = 3 * steps;
    F.flags = run.flags;
    F.ctl = static_cast<FusedCtl*>(run.ctl);
    F.base = run.base;
    F.parity = run.parity;
    F.err_host = run.err_dev;
    F.wait_ns = run.wait_ns;
    F.withhold = run.withhold;
    const int seg = fused_seg(p.wprec, p.nr, p.ntheta);
    if (p.coords == TEUK_COORDS_HYPERBOLOIDAL)
        return launch_fused_hyp(F, p.wprec, p.theta_mode, seg, run.blocks_per_sm, st);
    return launch_fused_rstar(F, p.wprec, p.theta_mode, seg, run.blocks_per_sm, st);
}

size_t fused_items(const teuk_params& p) {
    int nseg = 0, nrb = 0;
    fused_layout(p, &nseg, &nrb);
    return (size_t)nseg * nrb;
}

size_t fused_ctl_bytes() { return sizeof(FusedCtl); }

cudaError_t fused_resident_blocks(const teuk_params& p, long long* blocks) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = p.coords == TEUK_COORDS_HYPERBOLOIDAL
                ? fused_occupancy_hyp(p.wprec, p.theta_mode, &per_sm)
                : fused_occupancy_rstar(p.wprec, p.theta_mode, &per_sm);
    *blocks = (long long)sms * per_sm;
    return e;
}

// SSP-RK(10,4) after its fifth stage (v = u4 + dt/6 F(u4)), in the two-register
// form: q = u/25 + 9/25 v (kept to the end of the step), u5 = 3/5 u + 2/5 v.
__global__ void rk104_combine_kernel(const double* __restrict__ u, const double* __restrict__ v,
                                     double* __restrict__ q, double* __restrict__ u5,
                                     long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const double uk = u[k], vk = v[k];
        q[k] = fma(9.0 / 25.0, vk, uk / 25.0);
        u5[k] = fma(2.0 / 5.0, vk, 3.0 / 5.0 * uk);
    }
}

cudaError_t launch_rk104_combine(const double* u, const double* v, double* q, double* u5,
                                 long long n, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long blocks = std::min<long long>((n + 255) / 256, (long long)sms * 8);
    rk104_combine_kernel<<<(int)std::max<long long>(blocks, 1), 256, 0, st>>>(u, v, q, u5, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched evolutions (host side).
// ---------------------------------------------------------------------------

long long batch_items(const teuk_params& p, int segv) {
    return (long long)((p.nr + segv - 1) / segv) * ((p.ntheta + WARPS - 1) / WARPS);
}

cudaError_t upload_batch_desc(const BatchEvo* evos, int n, int segv, void* d_desc,
                              long long* items_out, cudaStream_t st) {
    std::vector<BatchDesc> h(n);
    long long item = 0;
    for (int k = 0; k < n; ++k) {
        const teuk_params& p = evos[k].p;
        BatchDesc& d = h[k];
        d.coef = evos[k].coef; d.u = evos[k].u; d.w = evos[k].w;
        d.nr = p.nr; d.nth = p.ntheta; d.nseg = (p.nr + segv - 1) / segv;
        d.plane = (long long)p.nr * p.ntheta;
        d.item0 = item;
        d.dt = evos[k].dt; d.eps4 = 4.0 * p.eps;
        eps_parts(p.eps, p.wprec, &d.eps_exp, &d.eps_pow2, &d.eps_mant);
        d.pole_flip = pole_flip_of(p);
        item += batch_items(p, segv);
    }
    *items_out = item;
    cudaError_t e = cudaMemcpyAsync(d_desc, h.data(), sizeof(BatchDesc) * n,
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

size_t batch_desc_bytes(int n) { return sizeof(BatchDesc) * (size_t)n; }

cudaError_t launch_batch_stage(int wprec, int theta, bool hyp, int stage, int segv,
                               const void* d_desc, int n, long long items, int grid,
                               cudaStream_t st) {
    const BatchDesc* d = static_cast<const BatchDesc*>(d_desc);
    if (hyp) return launch_batch_stage_hyp(wprec, theta, stage, segv, d, n, items, grid, st);
    switch (wprec) {
    case TEUK_W_FP64:
        return launch_batch_w<TEUK_W_FP64, false>(stage, segv, theta, d, n, items, grid, st);
    case TEUK_W_FP32:
        return launch_batch_w<TEUK_W_FP32, false>(stage, segv, theta, d, n, items, grid, st);
    case TEUK_W_FP16:
        return launch_batch_w<TEUK_W_FP16, false>(stage, segv, theta, d, n, items, grid, st);
    default:
        return launch_batch_w<TEUK_W_BF16, false>(stage, segv, theta, d, n, items, grid, st);
    }
}

}  // namespace teuk
