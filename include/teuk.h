/*
 * teuk.h -- C ABI of the GB300 (sm_103a) mixed-precision WENO5 Teukolsky solver.
 *
 * The library advances one azimuthal m-mode of the Teukolsky master equation
 * (arXiv 2010.04760, Eq. teuk0) on a 2+1-D (x, theta) grid, x the tortoise
 * r* or the hyperboloidal rho of Sec. 2.2. Each Runge-Kutta stage evaluates
 * the first-order system du/dt = -(M du/dx + L u + A u) (Sec. 2.3, Eq. evln)
 * with the WENO5 (Jiang-Shu) derivative in x (Sec. 3.1.2), the nonlinear
 * weights computed in a reduced precision (Sec. 3.1.3), fourth-order centred
 * differences in theta (Sec. 3.1 asks for centred differences), and the
 * SSP-RK(3,3) update (Sec. 3.2).
 *
 * Conventions shared by every call
 *  - State vector u = {Psi_R, Psi_I, pi_R, pi_I} (Sec. 2.3), Psi standing for
 *    the evolved field (Psi, or Phi = r Delta^s Psi, see teuk_field). In
 *    memory it is four planes, component-major: u[c][j][i], c = 0..3,
 *    j = theta row 0..ntheta-1, i = radial node 0..nr-1 (fastest).
 *    4*ntheta*nr doubles.
 *  - Grid: x_i = rstar_min + i h, h = (rstar_max - rstar_min)/(nr - 1), the
 *    two bounds holding the range of r* or of rho (teuk_coords);
 *    theta_j = (j + 1/2) pi / ntheta (cell centred, never on a pole).
 *  - In r*, time is Boyer-Lindquist t; on the hyperboloidal slices it is tau.
 *    The azimuth is the ingoing phi~ (Sec. 2.2) either way,
 *    Psi = exp(i m phi~) psi(t, x, theta); pi = psi_t + b psi_x.
 *  - Host pointers are read or written synchronously and stay owned by the
 *    caller. Device pointers ("_dev") are caller-owned device memory on the
 *    current CUDA device. Handles own their device memory.
 *  - Every call returns a teuk_status; nothing throws across the ABI (a
 *    failed host allocation returns TEUK_ERR_HOST and frees what the call
 *    had taken).
 *    A failing call leaves its outputs unspecified and the handle usable
 *    unless the status is TEUK_ERR_CUDA.
 *  - "stream" arguments are cudaStream_t values passed as void* (NULL = the
 *    legacy default stream, except in teuk_create and teuk_batch_create,
 *    where NULL gives the handle a non-blocking stream of its own).
 *  - Host threads: calls on different handles (or batches) may run at the
 *    same time on different threads; one handle must not be used by two
 *    threads at once. teuk_last_error is per thread.
 */
#ifndef TEUK_H
#define TEUK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TEUK_OK = 0,
    TEUK_ERR_ARG = 1,        /* invalid argument (message via teuk_last_error) */
    TEUK_ERR_CUDA = 2,       /* a CUDA call failed                               */
    TEUK_ERR_NONFINITE = 3,  /* the state holds a NaN or an infinity             */
    TEUK_ERR_TIMEOUT = 4,    /* a device-side wait of the fused step ran out     */
    TEUK_ERR_STATE = 5,      /* reserved: no call depends on an earlier one      */
    TEUK_ERR_HOST = 6        /* host memory or a host thread was not available   */
} teuk_status;

/* Precision of the WENO smoothness indicators and nonlinear weights
 * (Sec. 3.1.3). The derivative assembly, right-hand side and Runge-Kutta
 * update are always binary64. */
typedef enum {
    TEUK_W_FP64 = 0,   /* Jiang-Shu weights in binary64 (the plain baseline)  */
    TEUK_W_FP32 = 1,   /* weights in binary32                                 */
    TEUK_W_FP16 = 2,   /* weights in binary16, indicators scaled into range   */
    TEUK_W_BF16 = 3    /* weights in bfloat16, indicators scaled into range   */
} teuk_wprec;

/* Discretisation of the theta derivatives (Sec. 3.1). */
typedef enum {
    TEUK_THETA_CENTERED4 = 0,  /* fourth-order centred, the paper's choice      */
    TEUK_THETA_WENO5 = 1       /* option: the first theta derivative by WENO5,
                                  upwinded by the sign of -Bth (its speed when
                                  the term is read as -(-Bth) dPsi/dtheta), with
                                  the r* weight precision; the second derivative
                                  stays fourth-order centred */
} teuk_theta_mode;

/* Discretisation of the radial derivative (Sec. 3.1). */
typedef enum {
    TEUK_SCHEME_WENO5 = 0,    /* fifth-order WENO (Jiang-Shu), the method       */
    TEUK_SCHEME_FD6_KO8 = 1   /* the paper's comparison scheme (Sec. 3.1.1):
                                 sixth-order centred differences with the
                                 Kreiss-Oliger term sigma h^7 D+^4 D-^4 / 256
                                 subtracted from every component (the damping
                                 sign); centred theta only, no weights; the
                                 ghosts are those of the coordinates         */
} teuk_scheme;

/* Time integrator (Sec. 3.2). */
typedef enum {
    TEUK_RK_SSP33 = 0,    /* SSP-RK(3,3), Shu-Osher form (the paper's choice)   */
    TEUK_RK_SSP104 = 1    /* SSP-RK(10,4), ten forward-Euler stages of dt/6,
                             low-storage (two-register) evaluation            */
} teuk_rk;

/* Radial coordinate and slicing (Sec. 2.2). */
typedef enum {
    TEUK_COORDS_RSTAR = 0,         /* Boyer-Lindquist t, tortoise r*; the
                                      radial ghosts copy the edge value       */
    TEUK_COORDS_HYPERBOLOIDAL = 1  /* the paper's horizon-penetrating,
                                      compactified slices:
                                      tau = t~ - r^2/(r+S) + 4M ln(S/(r+S)),
                                      rho = r/(1 + r/S), t~ the ingoing Kerr
                                      time; the grid lies between the outer
                                      horizon rho_+ and scri (rho = S), both
                                      outflow boundaries, and the radial
                                      ghosts extrapolate the quartic through
                                      the five edge nodes. The pi rows move
                                      with their own speed -c (M33 = -c,
                                      c = Atr + b). Requires TEUK_FIELD_PHI.
                                      Both radial schemes and both theta
                                      modes; batches too.                     */
} teuk_coords;

/* How teuk_step launches a step (see teuk_set_launch). */
typedef enum {
    TEUK_LAUNCH_AUTO = 0,     /* the fused step on grids with at least as many
                                 work items per stage as the device holds
                                 blocks (SSP-RK(3,3) with WENO5), else stages  */
    TEUK_LAUNCH_STAGES = 1,   /* one launch per Runge-Kutta stage (CUDA graph)  */
    TEUK_LAUNCH_FUSED = 2     /* one persistent launch for all stages of up to
                                 1024 steps (SSP-RK(3,3) with WENO5 only)       */
} teuk_launch;

/* Evolved field. */
typedef enum {
    TEUK_FIELD_PSI = 0,   /* the Teukolsky function Psi of Eq. teuk0            */
    TEUK_FIELD_PHI = 1    /* Phi = r Delta^s Psi (Sec. 4's Phi = (r/Delta^2) Psi
                             at s = -2): finite on the horizon and at scri, and
                             O(1) at large r in r* as well                      */
} teuk_field;

/* Problem statement (Sec. 2.1-2.3, Sec. 4): grid, domain, black hole, mode.
 * Valid ranges: nr >= 7, 5 <= ntheta <= 262140 (four theta rows per CTA,
 * at most 65535 CTAs along theta), nr*ntheta <= 4e9, rstar_max > rstar_min,
 * M > 0, 0 <= |a| <= M, s in {-2..2}, |m| <= 64, eps in [1e-60, 1],
 * dt > 0, or dt == 0 with cfl in (0, 1] (dt from the stability rule below).
 * TEUK_COORDS_HYPERBOLOIDAL: hyp_S in [M, 1e6 M], and
 * rho_+ <= rstar_min < rstar_max <= S (rho_+ = r_+ S/(r_+ + S), r_+ = M +
 * sqrt(M^2 - a^2); a bound within 1e-12 relative of rho_+ or S counts as it),
 * or rstar_min == rstar_max == 0, which every call reads as the whole slice
 * [rho_+, S] (teuk_get_info returns the filled-in range).
 * Anything else returns TEUK_ERR_ARG. */
typedef struct {
    int nr, ntheta;                 /* grid nodes in x and theta             */
    double rstar_min, rstar_max;    /* x domain (r* or rho) in units of M    */
    double M, a;                    /* mass and spin                         */
    int s, m;                       /* spin weight, azimuthal number         */
    double cfl;                     /* Courant factor when dt == 0           */
    double dt;                      /* fixed time step, or 0                 */
    double eps;                     /* WENO epsilon (Jiang-Shu use 1e-6)     */
    int wprec;                      /* teuk_wprec                            */
    int theta_mode;                 /* teuk_theta_mode                       */
    int rk;                         /* teuk_rk                               */
    int scheme;                     /* teuk_scheme                           */
    double ko_sigma;                /* Kreiss-Oliger sigma (paper: 0.01)     */
    int coords;                     /* teuk_coords                           */
    int field;                      /* teuk_field                            */
    double hyp_S;                   /* slice parameter S (paper: ~20 M)      */
} teuk_params;

typedef struct teuk_handle teuk_handle;
typedef struct teuk_batch teuk_batch;

/* ---- diagnostics ------------------------------------------------------- */

/* Static description of a status code. Never NULL. */
const char* teuk_status_str(teuk_status st);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* teuk_last_error(void);

/* ---- host-side helpers ------------------------------------------------- */

/* Validate p (see teuk_params). Returns TEUK_OK or TEUK_ERR_ARG. */
teuk_status teuk_check_params(const teuk_params* p);

/* rho of the outer horizon on the hyperboloidal slices of Sec. 2.2:
 * rho_+ = r_+ S/(r_+ + S), r_+ = M + sqrt(M^2 - a^2) (the slice's rho =
 * r/(1 + r/S) at the horizon radius). Needs M > 0, |a| <= M, S in
 * [M, 1e6 M]; TEUK_ERR_ARG otherwise. */
teuk_status teuk_horizon_rho(double M, double a, double S, double* rho_out);

/* Time step of the stability rule used when p->dt == 0:
 *   dt = cfl / max_ij [ max(|b|, |c|)/h + sqrt(kappa) ],
 *   kappa = Ath (16/3)/dtheta^2 + |Bth| (3/2)/dtheta + |C|,
 * a bound of the largest frequency of the radial upwind part (the larger of
 * the two characteristic speeds over h, Sec. 3.2 forward-Euler limit; c = b
 * in r*) plus the theta part of the second-order operator; times 2.8 for
 * TEUK_RK_SSP104 (the smaller of its real- and imaginary-axis stability
 * extents relative to SSP-RK(3,3)). If p->dt > 0 it is returned unchanged. */
teuk_status teuk_stable_dt(const teuk_params* p, double* dt_out);

/* Number of doubles in the kernel coefficient array of p (11 planes of
 * ntheta*nr, 12 with TEUK_THETA_WENO5, 13 with TEUK_COORDS_HYPERBOLOIDAL).
 * 0 if p is invalid. */
size_t teuk_coeff_count(const teuk_params* p);

/* Kernel coefficient array for time step dt, written to host memory
 * coef_host[teuk_coeff_count(p)]. The planes are the first-order matrices
 * M, A, L of Sec. 2.3 pre-multiplied by the forward-Euler stage step of p's
 * integrator (dt for SSP-RK(3,3), dt/6 for SSP-RK(10,4)) and by 1/(6h)
 * (1/(60h) with TEUK_SCHEME_FD6_KO8), 1/(12 dtheta^k) for the stencil
 * normalisations, with the theta pole parity
 * folded into the theta-stencil planes. Built on the host in binary64; r(r*)
 * from the tortoise relation of Sec. 2.2; on the hyperboloidal slices the
 * coefficients of Eq. near_final for Phi, derived from Eq. teuk0 (they are
 * not printed in the paper). */
teuk_status teuk_build_coefficients(const teuk_params* p, double dt,
                                    double* coef_host);

/* Sustained binary64 FMA throughput of the current device, measured with a
 * short kernel of independent FMA chains (about 10 ms): *fma_per_s receives
 * lane-FMAs per second (2 flops each). The paper has no counterpart; this is
 * the denominator of the binary64 roofline that bounds the stage kernel.
 * Allocates and frees a small result buffer; synchronises the stream. */
teuk_status teuk_fp64_fma_rate(void* stream, double* fma_per_s);

/* ---- stateless device entry points (caller-owned device memory) --------- */

/* One fused Runge-Kutta stage (Sec. 3.2) on device arrays. With h the stage
 * step of p's integrator (dt for SSP-RK(3,3), dt/6 for SSP-RK(10,4)):
 *   stage 1: u_out = u_prev + h F(u_prev)
 *   stage 2: u_out = 3/4 u_n + 1/4 (u_prev + h F(u_prev))   (SSP-RK(3,3) only)
 *   stage 3: u_out = 1/3 u_n + 2/3 (u_prev + h F(u_prev))   (SSP-RK(3,3) only)
 *   stage 0: u_out = h F(u_prev)    (the operator alone, for checks)
 * F is the right-hand side of Eq. evln with the WENO5 radial derivative.
 * dt must be the step coef_dev was built for (teuk_build_coefficients).
 * coef_dev: teuk_coeff_count(p) doubles. u_n (read for stages 2, 3; may be
 * NULL otherwise), u_prev, u_out: 4*ntheta*nr doubles. u_out must not alias
 * u_prev; it may alias u_n (each node reads u_n only at itself).
 * Asynchronous on stream. Returns TEUK_ERR_ARG for bad p, dt, stage or
 * pointers, TEUK_ERR_CUDA if the launch fails. */
teuk_status teuk_stage_dev(const teuk_params* p, double dt, const double* coef_dev,
                           const double* u_n, const double* u_prev,
                           double* u_out, int stage, void* stream);

/* nsteps full steps of p's integrator (Sec. 3.2) in place on u_dev, using
 * caller scratch work_dev of 8*ntheta*nr doubles for SSP-RK(3,3) (the two
 * intermediate stages) or 12*ntheta*nr for SSP-RK(10,4) (two stage registers
 * and the retained combination). dt, coef_dev as for teuk_stage_dev.
 * Asynchronous on stream; u_dev holds the state after the last step.
 * work_dev must not overlap u_dev. With SSP-RK(3,3) and the WENO5 scheme the
 * last step leaves u^(1) in the first 4 planes of work_dev and 4 u^(2) in the
 * next 4: the second stage is kept scaled by four and the third runs on it
 * with 16 eps, which gives the same weights and the printed third stage's
 * roundings (Sec. 3.1.2, Sec. 3.2). */
teuk_status teuk_step_dev(const teuk_params* p, double dt, const double* coef_dev,
                          double* u_dev, double* work_dev, int64_t nsteps,
                          void* stream);

/* Same computation as teuk_step_dev, for callers that cannot allocate device
 * memory: code whose device memory is all owned by another allocator (for
 * example a framework's caching pool that has reserved the GPU, where a
 * direct cudaMalloc can fail or fragment the pool), and latency-critical loops
 * where cudaMalloc or cudaFree would synchronise the device. The paper has no
 * counterpart; this is a deployment convenience.
 * SSP-RK(3,3) only (TEUK_ERR_ARG otherwise).
 * The two intermediate stage buffers live in a fixed array inside the library
 * (8 MiB, held by every GPU that loads the library until the process exits),
 * so ntheta*nr must be <= TEUK_STATIC_MAX_NODES; larger grids return
 * TEUK_ERR_ARG. The caller still passes inputs and outputs (coef_dev, u_dev).
 * Nothing is allocated: no cudaMalloc, no cudaFree, no allocating library call.
 * The first call on a device looks up the array's device address on that
 * device (cudaGetSymbolAddress); make that first call before any stream
 * capture. The array keeps the last call's contents; each step writes every
 * element of both stage buffers before reading it, so nothing needs to start
 * at zero. All calls on a device share the one array: calls whose work
 * overlaps on the GPU (different streams without ordering between them) race
 * and give wrong results. */
#define TEUK_STATIC_MAX_NODES 131072
teuk_status teuk_step_dev_static(const teuk_params* p, double dt, const double* coef_dev,
                                 double* u_dev, int64_t nsteps, void* stream);

/* ---- handle API (library-owned device memory) --------------------------- */

/* One evolution of the paper's problem: the Teukolsky equation of spin
 * weight s for the azimuthal mode m on a Kerr black hole of mass M and spin a
 * (Eq. teuk0, Sec. 2), in first-order form (Eq. evln, Sec. 2.3), on the
 * (x, theta) grid of p (Sec. 3). Allocate the state, stage buffers and
 * coefficient array on the current device and build the coefficients
 * (teuk_stable_dt when p->dt == 0).
 * stream: the CUDA stream every later call of this handle runs on; NULL
 * creates a non-blocking stream that teuk_destroy destroys.
 * The state starts at zero, t = 0. */
teuk_status teuk_create(const teuk_params* p, void* stream, teuk_handle** out);

/* Free everything the handle owns. NULL is accepted. */
teuk_status teuk_destroy(teuk_handle* h);

/* Parameters and the time step actually used. */
teuk_status teuk_get_info(const teuk_handle* h, teuk_params* p_out,
                          double* dt_out, double* t_out);

/* Initial data from host arrays (Sec. 4: the field and its momentum):
 * psi, pi: [ntheta][nr] complex values as interleaved (re, im) doubles,
 * 2*ntheta*nr each. Sets t = 0. Synchronous. */
teuk_status teuk_set_initial(teuk_handle* h, const double* psi,
                             const double* pi);

/* Initial data of the paper's kind (Sec. 4: a Gaussian wave packet times
 * spin-weighted harmonics), built on the host and copied in:
 *   Psi(x, theta) = sum_{k<nl} c_k exp(-(x - rc)^2 / (2 width^2)) sY_{l_k m}(theta),
 * x the radial coordinate (r* or rho),
 *   l_k = max(|s|, |m|) + k,  pi = 0,  t = 0,
 * sY_lm by the Goldberg et al. (1967) sum formula at phi = 0. coeffs: 2*nl
 * doubles (re, im) per term; if coeffs is NULL, c_k = A_k exp(i phi_k) with
 * A_k = 0.5 + U, phi_k = 2 pi U', U, U' successive uniforms in [0, 1) from
 * SplitMix64 seeded with `seed` (u = (x >> 11) * 2^-53 per 64-bit output x).
 * nl in 1..16, width > 0. Synchronous. */
teuk_status teuk_set_gaussian(teuk_handle* h, double rc, double width, const double* coeffs,
                              int nl, uint64_t seed);

/* Checkpoint: copy the planar state u[4][ntheta][nr] and time t in or out
 * (host memory, synchronous). Restoring a saved state and stepping gives
 * bitwise the same result as never having stopped. */
teuk_status teuk_set_state(teuk_handle* h, const double* u_host, double t);
teuk_status teuk_get_state(teuk_handle* h, double* u_host, double* t_out);

/* Asynchronous forms: the copy is only enqueued on the handle's stream, in
 * order with teuk_step, and the call returns at once. The host buffer
 * (4*ntheta*nr doubles) must stay valid and, for set, unchanged until the
 * stream has passed the copy; for get, its contents are defined only after
 * teuk_synchronize. Use page-locked (pinned) host memory: with pageable
 * memory the copy may complete before the call returns. teuk_set_state_async
 * sets the handle's time to t at once. Several handles, each on its own
 * stream, overlap one evolution's copies with another's stepping. */
teuk_status teuk_set_state_async(teuk_handle* h, const double* u_host, double t);
teuk_status teuk_get_state_async(teuk_handle* h, double* u_host);

/* Wait until everything enqueued on the handle's stream has completed. */
teuk_status teuk_synchronize(teuk_handle* h);

/* Advance nsteps steps of p's integrator (Sec. 3.2: SSP-RK(3,3) or
 * SSP-RK(10,4); every stage the WENO5 operator of Sec. 3.1, or the FD6 + KO8
 * scheme of Sec. 3.1.1, and the right-hand side of Eq. evln). With the fused step (by default
 * for SSP-RK(3,3) with WENO5 when the grid has at least as many work items
 * per stage as resident blocks; see teuk_set_launch) one persistent launch
 * runs
 * every stage of up to 1024 steps: work items (4 theta rows x one radial
 * segment) are taken in stage order, and an item starts as soon as the eight
 * items around it have finished the previous stage, so stages overlap
 * instead of ending at a launch boundary. Otherwise 3 fused stage launches
 * per step for SSP-RK(3,3), 11 for SSP-RK(10,4), replayed from a captured CUDA
 * graph. Both give bitwise the same state. Asynchronous on the handle's
 * stream. Returns TEUK_ERR_TIMEOUT, without launching, if an earlier fused
 * launch of h ran out of a device-side wait. */
teuk_status teuk_step(teuk_handle* h, int64_t nsteps);

/* Launch mode of teuk_step (teuk_launch) and the bound of each device-side
 * wait of the fused step in seconds, wait_seconds in [1e-6, 3600] (default 2:
 * a wait lasts about one work item, tens of microseconds, when all is well).
 * A wait that runs out makes the launch end (every block stops at its next
 * wait that cannot be met at once); the next call
 * that synchronises the handle's stream (teuk_synchronize, teuk_observe,
 * teuk_get_state, teuk_set_state, teuk_check_finite) or the next teuk_step
 * returns TEUK_ERR_TIMEOUT, and the state is then undefined (restore it with
 * teuk_set_state). TEUK_LAUNCH_FUSED needs SSP-RK(3,3) with the WENO5 scheme
 * (TEUK_ERR_ARG otherwise). The paper has no counterpart: this is how the
 * library schedules its kernels. */
teuk_status teuk_set_launch(teuk_handle* h, int mode, double wait_seconds);

/* The launch mode set by teuk_set_launch (TEUK_LAUNCH_AUTO unless changed),
 * the wait bound, and whether teuk_step uses the fused step (1) or stage
 * launches (0). Any output may be NULL. */
teuk_status teuk_get_launch(const teuk_handle* h, int* mode_out, double* wait_seconds_out,
                            int* fused_out);

/* Test hook for the timeout path (no counterpart in the paper): the next
 * fused launch of h does not publish the completion of its first work item's
 * first stage, a flag nothing else sets, so the waits that depend on it run
 * out after the wait bound and the launch ends early with the state
 * undefined; the next synchronising call returns TEUK_ERR_TIMEOUT.
 * TEUK_ERR_ARG unless the handle's launch mode is TEUK_LAUNCH_FUSED. */
teuk_status teuk_test_withhold(teuk_handle* h);

/* Observation (Sec. 4): wave[2*ntheta] = Psi (re, im) along theta at the
 * radial node nearest rstar_ext (an r* or a rho: rho = S reads the field at
 * scri); horizon[6*ntheta] = for each theta row, Psi, pi and dPsi/dx
 * (one-sided, second order) at the innermost node i = 0, each as (re, im).
 * On the hyperboloidal slices with rstar_min = rho_+, node 0 is the horizon,
 * and these are Phi, pi and the radial derivative whose late-time behaviour
 * Sec. 4 compares with Aretakis' laws. Either output may be NULL. t_out (may
 * be NULL) = current t (tau on the hyperboloidal slices).
 * Synchronises the handle's stream. Returns TEUK_ERR_NONFINITE if a gathered
 * value is not finite. */
teuk_status teuk_observe(teuk_handle* h, double rstar_ext, double* wave,
                         double* horizon, double* t_out);

/* Device reduction over the whole state; TEUK_ERR_NONFINITE if any entry is
 * NaN or infinite. Synchronises the handle's stream. */
teuk_status teuk_check_finite(teuk_handle* h);

/* Device pointer of the state planes (valid until teuk_destroy). */
teuk_status teuk_state_dev(teuk_handle* h, double** u_dev);

/* ---- batched evolutions ---------------------------------------------------
 * Many independent evolutions (uneven grids, spins, modes, time steps) advanced
 * together: each Runge-Kutta stage of all members is one persistent launch over
 * a device work list of (member, 4-row block, radial segment) tiles, and the steps
 * are replayed from a captured CUDA graph. The launch boundary orders the
 * stages (no device-side waits). Every member runs the stage operator of
 * teuk_stage_dev (Sec. 2.3, 3.1, 3.2) with its own coefficients and dt. */

/* n members with parameters ps[0..n-1] (all with the same wprec, theta_mode
 * and coords, SSP-RK(3,3), WENO5; dt == 0 takes each member's own stability
 * rule). State starts at
 * zero, t = 0. autotune != 0 times the tile shapes (32- or 64-node segments)
 * and grid sizes (4 or 8 CTAs per SM) on a synthetic state and keeps the
 * fastest; otherwise the single-evolution defaults are used. stream as for
 * teuk_create. Allocates one device pool for all members. */
teuk_status teuk_batch_create(const teuk_params* ps, int n, void* stream, int autotune,
                              teuk_batch** out);
teuk_status teuk_batch_destroy(teuk_batch* b);

/* Member k's planar state u[4][ntheta_k][nr_k] and time (host, synchronous). */
teuk_status teuk_batch_set_state(teuk_batch* b, int k, const double* u_host, double t);
teuk_status teuk_batch_get_state(teuk_batch* b, int k, double* u_host, double* t_out);

/* Advance every member by nsteps of its own dt (asynchronous). */
teuk_status teuk_batch_step(teuk_batch* b, int64_t nsteps);

/* Member k's dt and t; the chosen segment length and CTAs per SM (either
 * output pointer may be NULL). */
teuk_status teuk_batch_get_info(const teuk_batch* b, int k, double* dt_out, double* t_out,
                                int* seg_out, int* ctas_per_sm_out);

#ifdef __cplusplus
}
#endif

#endif /* TEUK_H */
