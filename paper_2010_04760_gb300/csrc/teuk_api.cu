// C ABI: stateless device entry points, the handle (library-owned memory,
// CUDA-graph stepping), observation and the non-finite check.
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "teuk_internal.h"

namespace teuk {

cudaError_t launch_stage(const teuk_params& p, const double* coef, const double* un,
                         const double* up, double* out, int stage, double dt,
                         cudaStream_t st);
// launch_stage_ab, launch_rk104_combine: teuk_internal.h

static teuk_status cuda_fail(cudaError_t e, const char* what) {
    return fail(TEUK_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define TEUK_CUDA(call)                                         \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
    } while (0)

// NVTX range for the lifetime of a scope (host-side tracing of the public
// calls; a no-op unless a profiler collects NVTX).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// State-sized scratch arrays one step of p's integrator needs.
static int scratch_states(const teuk_params& p) { return p.rk == TEUK_RK_SSP104 ? 3 : 2; }

// One step of p's integrator (Sec. 3.2) in place on u; w holds
// scratch_states(p) arrays of 4 planes.
//   SSP-RK(3,3): u -> w1 -> w2 -> u (with WENO5, w2 = 4 u^(2): the scaled
//   second stage of teuk_stage_kernels.cuh).
//   SSP-RK(10,4): stages 1-5 are forward-Euler steps of dt/6 from u (A/B
//   ping-pong), then q = u/25 + 9/25 u5' and u5 = 3/5 u + 2/5 u5' (u5' the fifth
//   forward-Euler result), stages 6-9 forward Euler from u5, and
//   u^{n+1} = q + 3/5 (u9 + dt/6 F(u9)): the printed Shu-Osher form rearranged
//   into two registers plus q.
static cudaError_t launch_step(const teuk_params& p, const double* coef, double dt,
                               double* u, double* w, cudaStream_t st) {
    const size_t n = 4 * (size_t)p.nr * p.ntheta;
    cudaError_t e = cudaSuccess;
    if (p.rk == TEUK_RK_SSP104) {
        const double h = dt / 6.0;
        double* A = w;
        double* B = w + n;
        double* Q = w + 2 * n;
        const double* src = u;
        double* dst = A;
        for (int i = 1; i <= 5 && e == cudaSuccess; ++i) {    // u1..u4, then u4 + h F(u4)
            e = launch_stage_ab(p, coef, nullptr, src, dst, 1, h, 0.0, 1.0, st);
            src = dst;
            dst = (dst == A) ? B : A;
        }
        if (e == cudaSuccess) e = launch_rk104_combine(u, A, Q, B, (long long)n, st);  // B = u5
        src = B;
        dst = A;
        for (int i = 6; i <= 9 && e == cudaSuccess; ++i) {    // u6..u9 (u9 in B)
            e = launch_stage_ab(p, coef, nullptr, src, dst, 1, h, 0.0, 1.0, st);
            src = dst;
            dst = (dst == A) ? B : A;
        }
        if (e == cudaSuccess) e = launch_stage_ab(p, coef, Q, B, u, 2, h, 1.0, 3.0 / 5.0, st);
        return e;
    }
    e = launch_stage(p, coef, nullptr, u, w, 1, dt, st);
    if (p.scheme == TEUK_SCHEME_FD6_KO8) {
        if (e == cudaSuccess) e = launch_stage(p, coef, u, w, w + n, 2, dt, st);
        if (e == cudaSuccess) e = launch_stage(p, coef, u, w + n, u, 3, dt, st);
        return e;
    }
    // WENO5: w2 holds 4 u^(2), and the third stage runs on it with 16 eps
    // (teuk_stage_kernels.cuh, kStageScaled)
    if (e == cudaSuccess)
        e = launch_stage_ab(p, coef, u, w, w + n, kStageScaled, dt, 3.0, 1.0, st);
    if (e == cudaSuccess)
        e = launch_stage_ab(p, coef, u, w + n, u, 3, dt, 1.0 / 3.0, 1.0 / 6.0, st, 4);
    return e;
}

// Sets *flag when any of n values is NaN or infinite.
__global__ void nonfinite_kernel(const double* __restrict__ u, long long n, int* flag) {
    int bad = 0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        bad |= !isfinite(u[k]);
    bad = __syncthreads_or(bad);
    if (bad && threadIdx.x == 0) atomicOr(flag, 1);
}

// obs[2j..] = Psi at (ie, j); obs[2 nth + 6j ..] = Psi, pi, dPsi/dx at i = 0
// (x = r* or rho).
__global__ void observe_kernel(const double* __restrict__ u, int nr, int nth, long long plane,
                               int ie, double inv2h, double* obs) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nth) return;
    const long long row = (long long)j * nr;
    obs[2 * j] = u[row + ie];
    obs[2 * j + 1] = u[plane + row + ie];
    double* hz = obs + 2 * nth + 6 * j;
    for (int c = 0; c < 4; ++c) hz[c] = u[c * plane + row];
    for (int c = 0; c < 2; ++c) {
        const double* f = u + c * plane + row;
        hz[4 + c] = (-3.0 * f[0] + 4.0 * f[1] - f[2]) * inv2h;
    }
}

// Eight independent FMA chains per thread; one result per thread.
constexpr int kRateIters = 4096;
__global__ void fp64_rate_kernel(double* out, double a, double b) {
    double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
    double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < kRateIters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

// A smooth, non-zero synthetic state (used only to time tile shapes).
__global__ void synth_state_kernel(double* u, long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        u[k] = sin(1e-3 * (double)(k % 100003)) + 0.25;
}

}  // namespace teuk

using namespace teuk;

struct teuk_batch {
    int n = 0, wprec = 0;
    std::vector<teuk_params> p;
    std::vector<double> dt, t;
    std::vector<size_t> off;      // member k: u at off[k], w at off[k] + 4 plane, coef after
    double* pool = nullptr;
    void* desc = nullptr;
    long long items = 0;
    int seg = 32, ctas = 8, sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraphExec_t exec = nullptr;
    int chunk = 0;
    size_t plane(int k) const { return (size_t)p[k].nr * p[k].ntheta; }
    double* u(int k) const { return pool + off[k]; }
    double* w(int k) const { return pool + off[k] + 4 * plane(k); }
    double* coef(int k) const { return pool + off[k] + 12 * plane(k); }
};

struct teuk_handle {
    teuk_params p;
    double dt = 0.0, t = 0.0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    double* u = nullptr;
    double* w = nullptr;      // two stage buffers
    double* coef = nullptr;
    double* obs = nullptr;
    int* flag = nullptr;
    cudaGraphExec_t exec = nullptr;
    int chunk = 0;
    // fused step kernel (SSP-RK(3,3) with WENO5): completion flags per work
    // item, control block, host-mapped error words {code, epoch, item}
    unsigned* fflags = nullptr;
    void* fctl = nullptr;
    int* err_host = nullptr;
    int* err_dev = nullptr;
    int launch = TEUK_LAUNCH_AUTO;
    double wait_s = 2.0;
    int withhold = 0;
    long long fused_items = 0, fused_blocks = 0;   // work items per stage, resident blocks
    unsigned fused_base = 0;                       // epochs of the fused launches so far
    int fused_parity = 0;                          // fused launches so far, mod 2
    size_t plane() const { return (size_t)p.nr * p.ntheta; }
    bool fused_ok() const { return p.rk == TEUK_RK_SSP33 && p.scheme == TEUK_SCHEME_WENO5; }
    // The schedule of teuk_step. AUTO: the fused step on grids with at least
    // as many work items per stage as resident blocks (measured faster than
    // stage launches from one step per call up); otherwise stage launches
    // (on a smaller grid the blocks of consecutive stages wait on each other).
    int launch_used() const {
        if (launch == TEUK_LAUNCH_STAGES || !fused_ok()) return TEUK_LAUNCH_STAGES;
        if (launch == TEUK_LAUNCH_FUSED) return TEUK_LAUNCH_FUSED;
        return fused_items >= fused_blocks ? TEUK_LAUNCH_FUSED : TEUK_LAUNCH_STAGES;
    }
};

// TEUK_ERR_TIMEOUT if a fused launch of h ran out of a device-side wait (read
// after the stream has passed it); clears the record.
static teuk_status wait_status(teuk_handle* h) {
    volatile int* eh = h->err_host;
    if (!eh || eh[0] == 0) return TEUK_OK;
    const int epoch = eh[1], item = eh[2];
    eh[0] = 0;
    return fail(TEUK_ERR_TIMEOUT, "a device-side wait of the fused step ran out (stage " +
                                      std::to_string(epoch % 3 + 1) + " of step " +
                                      std::to_string(epoch / 3) + " of the launch, work item " +
                                      std::to_string(item) + "); the state is undefined");
}

extern "C" {

teuk_status teuk_stage_dev(const teuk_params* p, double dt, const double* coef_dev,
                           const double* u_n, const double* u_prev, double* u_out,
                           int stage, void* stream) {
    return guarded("teuk_stage_dev", [&]() -> teuk_status {
        teuk_status st = teuk_check_params(p);
        if (st != TEUK_OK) return st;
        const teuk_params q = resolve_params(*p);
        p = &q;
        if (!(dt > 0.0) || !std::isfinite(dt)) return fail(TEUK_ERR_ARG, "dt must be > 0");
        if (stage < 0 || stage > 3) return fail(TEUK_ERR_ARG, "stage must be 0..3");
        if (!coef_dev || !u_prev || !u_out) return fail(TEUK_ERR_ARG, "NULL device pointer");
        if (stage >= 2 && p->rk != TEUK_RK_SSP33)
            return fail(TEUK_ERR_ARG, "stages 2 and 3 are SSP-RK(3,3) stages");
        if (stage >= 2 && !u_n) return fail(TEUK_ERR_ARG, "u_n is NULL for stage 2/3");
        if (u_out == u_prev) return fail(TEUK_ERR_ARG, "u_out aliases u_prev");
        TEUK_CUDA(launch_stage(*p, coef_dev, u_n, u_prev, u_out, stage, dt, (cudaStream_t)stream));
        clear_error();
        return TEUK_OK;
    });
}

teuk_status teuk_step_dev(const teuk_params* p, double dt, const double* coef_dev,
                          double* u_dev, double* work_dev, int64_t nsteps, void* stream) {
    return guarded("teuk_step_dev", [&]() -> teuk_status {
        NvtxRange trace("teuk_step_dev");
        teuk_status st = teuk_check_params(p);
        if (st != TEUK_OK) return st;
        const teuk_params q = resolve_params(*p);
        p = &q;
        if (!(dt > 0.0) || !std::isfinite(dt)) return fail(TEUK_ERR_ARG, "dt must be > 0");
        if (!coef_dev || !u_dev || !work_dev) return fail(TEUK_ERR_ARG, "NULL device pointer");
        if (nsteps < 0) return fail(TEUK_ERR_ARG, "nsteps < 0");
        const size_t n = 4 * (size_t)p->nr * p->ntheta;
        if (work_dev < u_dev + n && u_dev < work_dev + scratch_states(*p) * n)
            return fail(TEUK_ERR_ARG, "work_dev overlaps u_dev");
        for (int64_t k = 0; k < nsteps; ++k)
            TEUK_CUDA(launch_step(*p, coef_dev, dt, u_dev, work_dev, (cudaStream_t)stream));
        clear_error();
        return TEUK_OK;
    });
}

// Stage buffers of teuk_step_dev_static: a fixed device array, so that the
// call allocates nothing. In host code `g_static_stages` is only a host-side
// stand-in for the array; its device address comes from cudaGetSymbolAddress,
// looked up once per device (with that device current) and cached.
constexpr size_t kStaticStageDoubles = 8 * (size_t)TEUK_STATIC_MAX_NODES;  // 2 stages x 4 planes
static __device__ __align__(256) double g_static_stages[kStaticStageDoubles];
static std::mutex g_static_mutex;
static double* g_static_ptr[256] = {nullptr};

teuk_status teuk_step_dev_static(const teuk_params* p, double dt, const double* coef_dev,
                                 double* u_dev, int64_t nsteps, void* stream) {
    return guarded("teuk_step_dev_static", [&]() -> teuk_status {
        teuk_status st = teuk_check_params(p);
        if (st != TEUK_OK) return st;
        const teuk_params q = resolve_params(*p);
        p = &q;
        const size_t nodes = (size_t)p->nr * p->ntheta;
        if (nodes > (size_t)TEUK_STATIC_MAX_NODES)
            return fail(TEUK_ERR_ARG, "grid has " + std::to_string(nodes) +
                                          " nodes; teuk_step_dev_static holds at most " +
                                          std::to_string(TEUK_STATIC_MAX_NODES));
        if (!(dt > 0.0) || !std::isfinite(dt)) return fail(TEUK_ERR_ARG, "dt must be > 0");
        if (!coef_dev || !u_dev) return fail(TEUK_ERR_ARG, "NULL device pointer");
        if (nsteps < 0) return fail(TEUK_ERR_ARG, "nsteps < 0");
        if (p->rk != TEUK_RK_SSP33)
            return fail(TEUK_ERR_ARG, "teuk_step_dev_static supports SSP-RK(3,3) only");
        int dev = 0;
        TEUK_CUDA(cudaGetDevice(&dev));
        if (dev < 0 || dev >= 256) return fail(TEUK_ERR_ARG, "device ordinal out of range");
        double* stages = nullptr;
        {
            std::lock_guard<std::mutex> lock(g_static_mutex);
            if (!g_static_ptr[dev]) {
                void* ptr = nullptr;
                TEUK_CUDA(cudaGetSymbolAddress(&ptr, g_static_stages));
                g_static_ptr[dev] = static_cast<double*>(ptr);
            }
            stages = g_static_ptr[dev];
        }
        for (int64_t k = 0; k < nsteps; ++k)
            TEUK_CUDA(launch_step(*p, coef_dev, dt, u_dev, stages, (cudaStream_t)stream));
        clear_error();
        return TEUK_OK;
    });
}

teuk_status teuk_fp64_fma_rate(void* stream, double* fma_per_s) {
    return guarded("teuk_fp64_fma_rate", [&]() -> teuk_status {
        if (!fma_per_s) return fail(TEUK_ERR_ARG, "fma_per_s is NULL");
        int dev = 0, sms = 0;
        TEUK_CUDA(cudaGetDevice(&dev));
        TEUK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int threads = 256, blocks = sms * 8;
        cudaStream_t st = (cudaStream_t)stream;
        double* out = nullptr;
        TEUK_CUDA(cudaMalloc(&out, sizeof(double) * (size_t)threads * blocks));
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaError_t e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        float best = 0.0f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
            e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) {
                fp64_rate_kernel<<<blocks, threads, 0, st>>>(out, 0.999999, 1e-7);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(out);
        if (e != cudaSuccess) return cuda_fail(e, "teuk_fp64_fma_rate");
        *fma_per_s = 8.0 * kRateIters * (double)threads * blocks / (best * 1e-3);
        clear_error();
        return TEUK_OK;
    });
}

static cudaError_t batch_upload(teuk_batch* b, int seg) {
    std::vector<BatchEvo> ev(b->n);
    for (int k = 0; k < b->n; ++k) ev[k] = BatchEvo{b->p[k], b->coef(k), b->u(k), b->w(k), b->dt[k]};
    return upload_batch_desc(ev.data(), b->n, seg, b->desc, &b->items, b->stream);
}

static cudaError_t batch_launch_step(teuk_batch* b) {
    const int grid = b->sms * b->ctas;
    cudaError_t e = cudaSuccess;
    for (int stage = 1; stage <= 3 && e == cudaSuccess; ++stage)
        e = launch_batch_stage(b->wprec, b->p[0].theta_mode,
                               b->p[0].coords == TEUK_COORDS_HYPERBOLOIDAL, stage, b->seg,
                               b->desc, b->n, b->items, grid, b->stream);
    return e;
}

teuk_status teuk_batch_destroy(teuk_batch* b) {
    if (!b) return TEUK_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    cudaFree(b->pool);
    cudaFree(b->desc);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return TEUK_OK;
}

teuk_status teuk_batch_create(const teuk_params* ps, int n, void* stream, int autotune,
                              teuk_batch** out) {
    return guarded("teuk_batch_create", [&]() -> teuk_status {
        NvtxRange trace("teuk_batch_create");
        if (!out) return fail(TEUK_ERR_ARG, "out is NULL");
        *out = nullptr;
        if (!ps || n < 1) return fail(TEUK_ERR_ARG, "need n >= 1 parameter sets");
        for (int k = 0; k < n; ++k) {
            teuk_status st = teuk_check_params(&ps[k]);
            if (st != TEUK_OK)
                return fail(st, "member " + std::to_string(k) + ": " + teuk_last_error());
            if (ps[k].wprec != ps[0].wprec || ps[k].theta_mode != ps[0].theta_mode ||
                ps[k].coords != ps[0].coords)
                return fail(TEUK_ERR_ARG, "all members need the same wprec, theta_mode and coords");
            if (ps[k].rk != TEUK_RK_SSP33 || ps[k].scheme != TEUK_SCHEME_WENO5)
                return fail(TEUK_ERR_ARG, "batched evolutions use WENO5 and SSP-RK(3,3)");
        }
        struct Owner {             // destroys a half-built batch on any early return or throw
            teuk_batch* b;
            ~Owner() { if (b) teuk_batch_destroy(b); }
        } own{new teuk_batch()};
        teuk_batch* b = own.b;
        b->n = n;
        b->wprec = ps[0].wprec;
        b->p.resize(n);
        for (int k = 0; k < n; ++k) b->p[k] = resolve_params(ps[k]);
        b->dt.resize(n);
        b->t.assign(n, 0.0);
        b->off.resize(n);
        size_t total = 0, max_plane = 0;
        for (int k = 0; k < n; ++k) {
            teuk_status st = teuk_stable_dt(&ps[k], &b->dt[k]);
            if (st != TEUK_OK) return st;
            b->off[k] = total;
            total += (((12 + coef_planes(ps[k])) * b->plane(k) + 31) / 32) * 32;  // aligned
            max_plane = std::max(max_plane, b->plane(k));
        }
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) {
            if (stream) {
                b->stream = (cudaStream_t)stream;
            } else {
                e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
                b->own_stream = (e == cudaSuccess);
            }
        }
        if (e == cudaSuccess) e = cudaMalloc(&b->pool, total * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&b->desc, batch_desc_bytes(n));
        int max_planes = 0;
        for (int k = 0; k < n; ++k) max_planes = std::max(max_planes, coef_planes(ps[k]));
        std::vector<double> host((size_t)max_planes * max_plane);
        for (int k = 0; k < n && e == cudaSuccess; ++k) {
            teuk_status st = teuk_build_coefficients(&ps[k], b->dt[k], host.data());
            if (st != TEUK_OK) return st;
            e = cudaMemcpyAsync(b->coef(k), host.data(),
                                coef_planes(ps[k]) * b->plane(k) * sizeof(double),
                                cudaMemcpyHostToDevice, b->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);   // host buffer is reused
        }
        b->seg = b->wprec == TEUK_W_FP64 ? 64 : 32;
        b->ctas = 8;
        if (e == cudaSuccess && autotune) {
            // time every (segment, CTAs per SM) candidate on a synthetic state
            for (int k = 0; k < n && e == cudaSuccess; ++k) {
                synth_state_kernel<<<b->sms * 4, 256, 0, b->stream>>>(b->u(k),
                                                                      4 * (long long)b->plane(k));
                e = cudaGetLastError();
            }
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (e == cudaSuccess) e = cudaEventCreate(&e0);
            if (e == cudaSuccess) e = cudaEventCreate(&e1);
            float best = -1.0f;
            int best_seg = b->seg, best_ctas = b->ctas;
            const int segs[2] = {32, 64}, ctas[2] = {4, 8};
            for (int a = 0; a < 2 && e == cudaSuccess; ++a) {
                e = batch_upload(b, segs[a]);
                for (int c = 0; c < 2 && e == cudaSuccess; ++c) {
                    b->seg = segs[a];
                    b->ctas = ctas[c];
                    e = batch_launch_step(b);                                  // warm-up
                    if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
                    for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = batch_launch_step(b);
                    if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                    float ms = 0.0f;
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                    if (e == cudaSuccess && (best < 0.0f || ms < best)) {
                        best = ms; best_seg = segs[a]; best_ctas = ctas[c];
                    }
                }
            }
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
            b->seg = best_seg;
            b->ctas = best_ctas;
        }
        for (int k = 0; k < n && e == cudaSuccess; ++k)
            e = cudaMemsetAsync(b->u(k), 0, 4 * b->plane(k) * sizeof(double), b->stream);
        if (e == cudaSuccess) e = batch_upload(b, b->seg);
        if (e != cudaSuccess) return cuda_fail(e, "teuk_batch_create");
        *out = b;
        own.b = nullptr;
        clear_error();
        return TEUK_OK;
    });
}

teuk_status teuk_batch_set_state(teuk_batch* b, int k, const double* u_host, double t) {
    return guarded("teuk_batch_set_state", [&]() -> teuk_status {
        if (!b || !u_host || k < 0 || k >= b->n) return fail(TEUK_ERR_ARG, "bad argument");
        TEUK_CUDA(cudaMemcpyAsync(b->u(k), u_host, 4 * b->plane(k) * sizeof(double),
                                  cudaMemcpyHostToDevice, b->stream));
        TEUK_CUDA(cudaStreamSynchronize(b->stream));
        b->t[k] = t;
        clear_error();
        return TEUK_OK;
    });
}

teuk_status teuk_batch_get_state(teuk_batch* b, int k, double* u_host, double* t_out) {
    return guarded("teuk_batch_get_state", [&]() -> teuk_status {
        if (!b || !u_host || k < 0 || k >= b->n) return fail(TEUK_ERR_ARG, "bad argument");
        TEUK_CUDA(cudaMemcpyAsync(u_host, b->u(k), 4 * b->plane(k) * sizeof(double),
                                  cudaMemcpyDeviceToHost, b->stream));
        TEUK_CUDA(cudaStreamSynchronize(b->stream));
        if (t_out) *t_out = b->t[k];
        clear_error();
        return TEUK_OK;
    });
}

teuk_status teuk_batch_step(teuk_batch* b, int64_t nsteps) {
    return guarded("teuk_batch_step", [&]() -> teuk_status {
        NvtxRange trace("teuk_batch_step");
        if (!b) return fail(TEUK_ERR_ARG, "batch is NULL");
        if (nsteps < 0) return fail(TEUK_ERR_ARG, "nsteps < 0");
        const int kChunk = 16;
        if (nsteps >= kChunk && !b->exec) {
            cudaGraph_t g = nullptr;
            TEUK_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            for (int k = 0; k < kChunk && e == cudaSuccess; ++k) e = batch_launch_step(b);
            cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
            if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(e, "capture"); }
            if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&b->exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                b->exec = nullptr;
                return cuda_fail(e, "cudaGraphInstantiate");
            }
            b->chunk = kChunk;
        }
        int64_t left = nsteps;
        while (b->exec && left >= b->chunk) {
            TEUK_CUDA(cudaGraphLaunch(b->exec, b->stream));
            left -= b->chunk;
        }
        for (; left > 0; --left) TEUK_CUDA(batch_launch_step(b));
        for (int k = 0; k < b->n; ++k) b->t[k] += (double)nsteps * b->dt[k];
        clear_error();
        return TEUK_OK;
    });
}

teuk_status teuk_batch_get_info(const teuk_batch* b, int k, double* dt_out, double* t_out,
                                int* seg_out, int* ctas_per_sm_out) {
    return guarded("teuk_batch_get_info", [&]() -> teuk_status {
        if (!b || k < 0 || k >= b->n) return fail(TEUK_ERR_ARG, "bad argument");
        if (dt_out) *dt_out = b->dt[k];
        if (t_out) *t_out = b->t[k];
        if (seg_out) *seg_out = b->seg;
        if (ctas_per_sm_out) *ctas_per_sm_out = b->ctas;
        return TEUK_OK;
    });
}

teuk_status teuk_destroy(teuk_handle* h) {
    if (!h) return TEUK_OK;
    if (h->exec) cudaGraphExecDestroy(h->exec);
    cudaFree(h->u);
    cudaFree(h->w);
    cudaFree(h->coef);
    cudaFree(h->obs);
    cudaFree(h->flag);
    cudaFree(h->fflags);
    cudaFree(h->fctl);
    if (h->err_host) cudaFreeHost(h->err_host);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return TEUK_OK;
}

teuk_status teuk_create(const teuk_params* p, void* stream, teuk_handle** out) {
    return guarded("teuk_create", [&]() -> teuk_status {
        NvtxRange trace("teuk_create");
        if (!out) return fail(TEUK_ERR_ARG, "out is NULL");
        *out = nullptr;
        teuk_status st = teuk_check_params(p);
        if (st != TEUK_OK) return st;
        double dt = 0.0;
        st = teuk_stable_dt(p, &dt);
        if (st != TEUK_OK) return st;
        const size_t n = (size_t)p->nr * p->ntheta;
        std::vector<double> coef((size_t)coef_planes(*p) * n);       // may throw: nothing held yet
        st = teuk_build_coefficients(p, dt, coef.data());
        if (st != TEUK_OK) return st;
        teuk_handle* h = new teuk_handle();
        h->p = resolve_params(*p);
        h->dt = dt;
        cudaError_t e = cudaSuccess;
        if (stream) {
            h->stream = (cudaStream_t)stream;
        } else {
            e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
            h->own_stream = (e == cudaSuccess);
        }
        if (e == cudaSuccess) e = cudaMalloc(&h->u, 4 * n * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&h->w, 4 * scratch_states(*p) * n * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&h->coef, coef.size() * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&h->obs, 8 * (size_t)p->ntheta * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&h->flag, sizeof(int));
        if (e == cudaSuccess && h->fused_ok()) {
            h->fused_items = (long long)fused_items(h->p);
            e = fused_resident_blocks(h->p, &h->fused_blocks);
        }
        if (e == cudaSuccess && h->fused_ok()) {
            const size_t nf = fused_items(h->p) * sizeof(unsigned);
            e = cudaMalloc(&h->fflags, nf);
            if (e == cudaSuccess) e = cudaMalloc(&h->fctl, fused_ctl_bytes());
            if (e == cudaSuccess) e = cudaMemsetAsync(h->fflags, 0, nf, h->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(h->fctl, 0, fused_ctl_bytes(), h->stream);
            if (e == cudaSuccess)
                e = cudaHostAlloc(reinterpret_cast<void**>(&h->err_host), 3 * sizeof(int),
                                  cudaHostAllocMapped);
            if (e == cudaSuccess) {
                h->err_host[0] = h->err_host[1] = h->err_host[2] = 0;
                e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&h->err_dev), h->err_host, 0);
            }
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(h->u, 0, 4 * n * sizeof(double), h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->coef, coef.data(), coef.size() * sizeof(double),
                                cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) {
            teuk_destroy(h);
            return cuda_fail(e, "teuk_create");
        }
        *out = h;
        clear_error();
        return TEUK_OK;
    });
}

teuk_status teuk_get_info(const teuk_handle* h, teuk_params* p_out, double* dt_out,
                          double* t_out) {
    return guarded("teuk_get_info", [&]() -> teuk_status {
        if (!h) return fail(TEUK_ERR_ARG, "handle is NULL");
        if (p_out) *p_out = h->p;
        if (dt_out) *dt_out = h->dt;
        if (t_out) *t_out = h->t;
        return TEUK_OK;
    });
}

teuk_status teuk_set_state(teuk_handle* h, const double* u_host, double t) {
    return guarded("teuk_set_state", [&]() -> teuk_status {
        if (!h || !u_host) return fail(TEUK_ERR_ARG, "NULL argument");
        TEUK_CUDA(cudaMemcpyAsync(h->u, u_host, 4 * h->plane() * sizeof(double),
                                  cudaMemcpyHostToDevice, h->stream));
        TEUK_CUDA(cudaStreamSynchronize(h->stream));
        h->t = t;
        teuk_status ws = wait_status(h);
        if (ws != TEUK_OK) return ws;
        clear_error();
        return TEUK_OK;
    });
}

teuk_status teuk_get_state(teuk_handle* h, double* u_host, double* t_out) {
    return guarded("teuk_get_state", [&]() -> teuk_status {
        if (!h || !u_host) return fail(TEUK_ERR_ARG, "NULL argument");
        TEUK_CUDA(cudaMemcpyAsync(u_host, h->u, 4 * h->plane() * sizeof(double),
                                  cudaMemcpyDeviceToHost, h->stream));
        TEUK_CUDA(cudaStreamSynchronize(h->stream));
        if (t_out) *t_out = h->t;
        teuk_status ws = wait_status(h);
        if (ws != TEUK_OK) return ws;
        clear_error();
        return TEUK_OK;
    });
}

teuk_status teuk_set_state_async(teuk_handle* h, const double* u_host, double t) {
    return guarded("teuk_set_state_async", [&]() -> teuk_status {
        if (!h || !u_host) return fail(TEUK_ERR_ARG, "NULL argument");
        TEUK_CUDA(cudaMemcpyAsync(h->u, u_host, 4 * h->plane() * sizeof(double),
                                  cudaMemcpyHostToDevice, h->stream));
        h->t = t;
        clear_error();
        return TEUK_OK;
    });
}

teuk_status teuk_get_state_async(teuk_handle* h, double* u_host) {
    return guarded("teuk_get_state_async", [&]() -> teuk_status {
        if (!h || !u_host) return fail(TEUK_ERR_ARG, "NULL argument");
        TEUK_CUDA(cudaMemcpyAsync(u_host, h->u, 4 * h->plane() * sizeof(double),
                                  cudaMemcpyDeviceToHost, h->stream));
        clear_error();
        return TEUK_OK;
    });
}

teuk_status teuk_synchronize(teuk_handle* h) {
    return guarded("teuk_synchronize", [&]() -> teuk_status {
        if (!h) return fail(TEUK_ERR_ARG, "handle is NULL");
        TEUK_CUDA(cudaStreamSynchronize(h->stream));
        teuk_status ws = wait_status(h);
        if (ws != TEUK_OK) return ws;
        clear_error();
        return TEUK_OK;
    });
}

teuk_status teuk_set_initial(teuk_handle* h, const double* psi, const double* pi) {
    return guarded("teuk_set_initial", [&]() -> teuk_status {
        if (!h || !psi || !pi) return fail(TEUK_ERR_ARG, "NULL argument");
        const size_t n = h->plane();
        std::vector<double> u(4 * n);
        for (size_t k = 0; k < n; ++k) {
            u[k] = psi[2 * k];
            u[n + k] = psi[2 * k + 1];
            u[2 * n + k] = pi[2 * k];
            u[3 * n + k] = pi[2 * k + 1];
        }
        return teuk_set_state(h, u.data(), 0.0);
    });
}

teuk_status teuk_set_gaussian(teuk_handle* h, double rc, double width, const double* coeffs,
                              int nl, uint64_t seed) {
    return guarded("teuk_set_gaussian", [&]() -> teuk_status {
        if (!h) return fail(TEUK_ERR_ARG, "handle is NULL");
        if (nl < 1 || nl > 16) return fail(TEUK_ERR_ARG, "nl must be in 1..16");
        if (!(width > 0.0) || !std::isfinite(width) || !std::isfinite(rc))
            return fail(TEUK_ERR_ARG, "need finite rc and width > 0");
        const teuk_params& p = h->p;
        const int nr = p.nr, nth = p.ntheta;
        const size_t n = h->plane();
        std::vector<double> cre(nl), cim(nl);
        uint64_t state = seed;
        for (int k = 0; k < nl; ++k) {
            if (coeffs) {
                cre[k] = coeffs[2 * k];
                cim[k] = coeffs[2 * k + 1];
            } else {
                const double amp = 0.5 + (double)(splitmix64(state) >> 11) * 0x1.0p-53;
                const double ph = 2.0 * M_PI * (double)(splitmix64(state) >> 11) * 0x1.0p-53;
                cre[k] = amp * std::cos(ph);
                cim[k] = amp * std::sin(ph);
            }
        }
        const int l0 = std::max(std::abs(p.s), std::abs(p.m));
        const double hs = (p.rstar_max - p.rstar_min) / (nr - 1);
        std::vector<double> radial(nr), ang((size_t)nl * nth);
        for (int i = 0; i < nr; ++i) {
            const double z = (p.rstar_min + i * hs - rc) / width;
            radial[i] = std::exp(-0.5 * z * z);
        }
        for (int k = 0; k < nl; ++k)
            for (int j = 0; j < nth; ++j)
                ang[(size_t)k * nth + j] = swsh(p.s, l0 + k, p.m, (j + 0.5) * M_PI / nth);
        std::vector<double> u(4 * n, 0.0);
        for (int j = 0; j < nth; ++j) {
            double are = 0.0, aim = 0.0;
            for (int k = 0; k < nl; ++k) {
                are += cre[k] * ang[(size_t)k * nth + j];
                aim += cim[k] * ang[(size_t)k * nth + j];
            }
            for (int i = 0; i < nr; ++i) {
                u[(size_t)j * nr + i] = are * radial[i];
                u[n + (size_t)j * nr + i] = aim * radial[i];
            }
        }
        return teuk_set_state(h, u.data(), 0.0);
    });
}

teuk_status teuk_step(teuk_handle* h, int64_t nsteps) {
    return guarded("teuk_step", [&]() -> teuk_status {
        NvtxRange trace("teuk_step");
        if (!h) return fail(TEUK_ERR_ARG, "handle is NULL");
        if (nsteps < 0) return fail(TEUK_ERR_ARG, "nsteps < 0");
        teuk_status ws = wait_status(h);          // an earlier launch that already ran out
        if (ws != TEUK_OK) return ws;
        if (h->launch_used() == TEUK_LAUNCH_FUSED) {
            // one launch per 1024 steps (bounds a launch's duration)
            FusedRun run{h->fflags, h->fctl, h->err_dev,
                         (unsigned long long)(h->wait_s * 1e9), h->withhold, 0, 0u, 0};
            for (int64_t left = nsteps; left > 0;) {
                const int k = (int)std::min<int64_t>(left, 1024);
                run.base = h->fused_base;
                run.parity = h->fused_parity;
                TEUK_CUDA(launch_fused_step(h->p, h->coef, h->dt, h->u, h->w, k, run, h->stream));
                h->fused_base += 3u * (unsigned)k;
                h->fused_parity ^= 1;
                run.withhold = 0;
                h->withhold = 0;
                left -= k;
            }
            h->t += (double)nsteps * h->dt;
            clear_error();
            return TEUK_OK;
        }
        const int kChunk = 16;
        if (nsteps >= kChunk && !h->exec) {
            cudaGraph_t g = nullptr;
            TEUK_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            for (int k = 0; k < kChunk && e == cudaSuccess; ++k)
                e = launch_step(h->p, h->coef, h->dt, h->u, h->w, h->stream);
            cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
            if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(e, "capture"); }
            if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&h->exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                h->exec = nullptr;
                return cuda_fail(e, "cudaGraphInstantiate");
            }
            h->chunk = kChunk;
        }
        int64_t left = nsteps;
        while (h->exec && left >= h->chunk) {
            TEUK_CUDA(cudaGraphLaunch(h->exec, h->stream));
            left -= h->chunk;
        }
        for (; left > 0; --left)
            TEUK_CUDA(launch_step(h->p, h->coef, h->dt, h->u, h->w, h->stream));
        h->t += (double)nsteps * h->dt;
        clear_error();
        return TEUK_OK;
    });
}

teuk_status teuk_observe(teuk_handle* h, double rstar_ext, double* wave, double* horizon,
                         double* t_out) {
    return guarded("teuk_observe", [&]() -> teuk_status {
        NvtxRange trace("teuk_observe");
        if (!h) return fail(TEUK_ERR_ARG, "handle is NULL");
        if (!std::isfinite(rstar_ext)) return fail(TEUK_ERR_ARG, "rstar_ext not finite");
        const int nr = h->p.nr, nth = h->p.ntheta;
        const double hstep = (h->p.rstar_max - h->p.rstar_min) / (nr - 1);
        long ie = std::lround((rstar_ext - h->p.rstar_min) / hstep);
        ie = ie < 0 ? 0 : (ie > nr - 1 ? nr - 1 : ie);
        observe_kernel<<<(nth + 127) / 128, 128, 0, h->stream>>>(
            h->u, nr, nth, (long long)h->plane(), (int)ie, 0.5 / hstep, h->obs);
        TEUK_CUDA(cudaGetLastError());
        std::vector<double> o(8 * (size_t)nth);
        TEUK_CUDA(cudaMemcpyAsync(o.data(), h->obs, o.size() * sizeof(double),
                                  cudaMemcpyDeviceToHost, h->stream));
        TEUK_CUDA(cudaStreamSynchronize(h->stream));
        teuk_status ws = wait_status(h);
        if (ws != TEUK_OK) return ws;
        for (double v : o)
            if (!std::isfinite(v)) return fail(TEUK_ERR_NONFINITE, "observed value is not finite");
        if (wave) std::memcpy(wave, o.data(), 2 * (size_t)nth * sizeof(double));
        if (horizon) std::memcpy(horizon, o.data() + 2 * nth, 6 * (size_t)nth * sizeof(double));
        if (t_out) *t_out = h->t;
        clear_error();
        return TEUK_OK;
    });
}

teuk_status teuk_check_finite(teuk_handle* h) {
    return guarded("teuk_check_finite", [&]() -> teuk_status {
        if (!h) return fail(TEUK_ERR_ARG, "handle is NULL");
        TEUK_CUDA(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
        nonfinite_kernel<<<304, 256, 0, h->stream>>>(h->u, 4 * (long long)h->plane(), h->flag);
        TEUK_CUDA(cudaGetLastError());
        int flag = 0;
        TEUK_CUDA(cudaMemcpyAsync(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        TEUK_CUDA(cudaStreamSynchronize(h->stream));
        teuk_status ws = wait_status(h);
        if (ws != TEUK_OK) return ws;
        if (flag) return fail(TEUK_ERR_NONFINITE, "state holds NaN or infinity");
        clear_error();
        return TEUK_OK;
    });
}

teuk_status teuk_set_launch(teuk_handle* h, int mode, double wait_seconds) {
    return guarded("teuk_set_launch", [&]() -> teuk_status {
        if (!h) return fail(TEUK_ERR_ARG, "handle is NULL");
        if (mode != TEUK_LAUNCH_AUTO && mode != TEUK_LAUNCH_STAGES && mode != TEUK_LAUNCH_FUSED)
            return fail(TEUK_ERR_ARG, "unknown launch mode");
        if (mode == TEUK_LAUNCH_FUSED && !h->fused_ok())
            return fail(TEUK_ERR_ARG, "the fused step needs SSP-RK(3,3) and the WENO5 scheme");
        if (!(wait_seconds >= 1e-6 && wait_seconds <= 3600.0))
            return fail(TEUK_ERR_ARG, "wait_seconds must be in [1e-6, 3600]");
        h->launch = mode;
        h->wait_s = wait_seconds;
        clear_error();
        return TEUK_OK;
    });
}

teuk_status teuk_get_launch(const teuk_handle* h, int* mode_out, double* wait_seconds_out,
                            int* fused_out) {
    return guarded("teuk_get_launch", [&]() -> teuk_status {
        if (!h) return fail(TEUK_ERR_ARG, "handle is NULL");
        if (mode_out) *mode_out = h->launch;
        if (wait_seconds_out) *wait_seconds_out = h->wait_s;
        if (fused_out) *fused_out = h->launch_used() == TEUK_LAUNCH_FUSED;
        return TEUK_OK;
    });
}

teuk_status teuk_test_withhold(teuk_handle* h) {
    return guarded("teuk_test_withhold", [&]() -> teuk_status {
        if (!h) return fail(TEUK_ERR_ARG, "handle is NULL");
        if (h->launch != TEUK_LAUNCH_FUSED)
            return fail(TEUK_ERR_ARG, "set TEUK_LAUNCH_FUSED first (teuk_set_launch)");
        h->withhold = 1;
        clear_error();
        return TEUK_OK;
    });
}

teuk_status teuk_state_dev(teuk_handle* h, double** u_dev) {
    return guarded("teuk_state_dev", [&]() -> teuk_status {
        if (!h || !u_dev) return fail(TEUK_ERR_ARG, "NULL argument");
        *u_dev = h->u;
        return TEUK_OK;
    });
}

}  // extern "C"
