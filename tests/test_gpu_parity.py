"""GPU parity: the CUDA path against the CPU oracle, element by element, on
seeded inputs, through the C ABI. Weights of every precision are computed on
both sides with the same rounding sequence, so the tolerance is binary64
round-off of the (differently arranged) stencil arithmetic for every weight
format, taken node by node: |gpu - oracle| <= 1e-12 x the size of the terms
entering that node (``_local_scale``), so that rows scaled down to 1e-40 and a
1e-200 tail are checked at their own scale, where the scaling of the
reduced-precision weights into range acts (Sec. 3.1.3)."""
import numpy as np
import pytest

import oracle as o
import paper_2010_04760_gb300 as T
from paper_2010_04760_gb300 import inputs as I
from _local_scale import assert_local, run_scale, stage_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    T.lib()


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def oracle_dt(g, co):
    """Test-side time step: 0.5 / max(b/h + sqrt(theta frequencies))."""
    b, Kr, Ki, Br, Bi, Cr, Ci, Ath, Bth = co[:9]
    h = (g.rs_max - g.rs_min) / (g.nr - 1)
    dth = np.pi / g.nth
    kap = Ath * (16 / 3) / dth ** 2 + np.abs(Bth) * 1.5 / dth + np.hypot(Cr, Ci)
    return 0.5 / np.max(b / h + np.sqrt(kap))


def compare(got, exp_, scale, tol=TOL, what=""):
    assert_local(got, exp_, scale, tol, what)


SHAPES = [(7, 5), (64, 8), (100, 13), (257, 33), (1000, 17)]
PHYS = [(0.999, -2, 2), (0.0, 0, 0), (1.0, 0, 1), (0.5, -1, 0)]


@pytest.mark.parametrize("theta_mode", [0, 1])
@pytest.mark.parametrize("wprec", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("phys", PHYS)
def test_operator_parity(wprec, shape, phys, theta_mode):
    nr, nth = shape
    a, s, m = phys
    rs0, rs1 = -40.0, 120.0
    seed = nr * 7 + nth
    for smooth in (True, False):
        u = I.multiscale_state(nr, nth, seed, smooth)
        g = o.grid(nr, nth, rs0, rs1, 1.0, a, s, m, 1e-6, wprec, theta_mode)
        co = o.coefficients(g)
        F = o.rhs(g, co, u)
        p = T.make_params(nr, nth, rs0, rs1, 1.0, a, s, m, wprec=wprec, theta_mode=theta_mode)
        coef = dev(T.teuk_build_coefficients(p, 1.0))
        ud = dev(u)
        out = torch.empty_like(ud)
        T.teuk_stage_dev(p, 1.0, coef, None, ud, out, 0)
        compare(host(out), F, stage_scale(g, co, 1.0, u, with_prev=False),
                what=f"{wprec} {shape} {phys} theta={theta_mode} smooth={smooth}")


@pytest.mark.parametrize("theta_mode", [0, 1])
@pytest.mark.parametrize("wprec,step,period", [("fp16", 6, 6), ("bf16", 33, 5), ("fp32", 33, 5)])
def test_operator_parity_where_reduced_weights_underflow(wprec, step, period, theta_mode):
    """Radial lines whose magnitudes fall by 2^-step from node to node
    (repeating every `period` nodes, random signs and 10% jitter): within a
    stencil the scaled first differences, their squares and the ratios of the
    weights reach the format's subnormal range, where every operation must
    still round as the oracle's emulation does (gradual underflow, no flush
    to zero) for the weights to agree bit for bit."""
    nr, nth = 190, 6
    rng = np.random.default_rng(17)
    mag = np.exp2(-step * (np.arange(nr) % period).astype(float))
    u = np.empty((4, nth, nr))
    for c in range(4):
        for j in range(nth):
            u[c, j] = mag * rng.choice([-1.0, 1.0], nr) * (1.0 + 0.1 * rng.random(nr))
    g = o.grid(nr, nth, -40.0, 120.0, 1.0, 0.9, -2, 2, 1e-6, wprec, theta_mode)
    co = o.coefficients(g)
    F = o.rhs(g, co, u)
    p = T.make_params(nr, nth, -40.0, 120.0, 1.0, 0.9, -2, 2, wprec=wprec, theta_mode=theta_mode)
    coef = dev(T.teuk_build_coefficients(p, 1.0))
    out = torch.empty(4, nth, nr, dtype=torch.float64, device="cuda")
    T.teuk_stage_dev(p, 1.0, coef, None, dev(u), out, 0)
    compare(host(out), F, stage_scale(g, co, 1.0, u, with_prev=False),
            what=f"{wprec} underflowing stencils theta={theta_mode}")


@pytest.mark.parametrize("wprec", ["fp64", "fp32"])
def test_rk_stages_parity(wprec):
    nr, nth, a, s, m = 300, 20, 0.9, -2, 1
    rs0, rs1 = -50.0, 150.0
    g = o.grid(nr, nth, rs0, rs1, 1.0, a, s, m, 1e-6, wprec)
    co = o.coefficients(g)
    dt = oracle_dt(g, co)
    un = I.random_state(nr, nth, 1)
    up = I.random_state(nr, nth, 2)
    p = T.make_params(nr, nth, rs0, rs1, 1.0, a, s, m, wprec=wprec)
    coef = dev(T.teuk_build_coefficients(p, dt))
    Fp = o.rhs(g, co, up)
    exp_ = {1: up + dt * Fp, 2: 0.75 * un + 0.25 * (up + dt * Fp),
            3: un / 3.0 + 2.0 / 3.0 * (up + dt * Fp)}
    ab = {1: (0.0, 1.0), 2: (0.75, 0.25), 3: (1.0 / 3.0, 2.0 / 3.0)}
    sc = {k: stage_scale(g, co, dt, up, un, *ab[k]) for k in ab}
    for stage in (1, 2, 3):
        out = torch.empty(4, nth, nr, dtype=torch.float64, device="cuda")
        T.teuk_stage_dev(p, dt, coef, dev(un), dev(up), out, stage)
        compare(host(out), exp_[stage], sc[stage], tol=1e-13, what=f"stage {stage}")
    # stage 3 in place on u_n (the library's own step layout)
    una = dev(un)
    T.teuk_stage_dev(p, dt, coef, una, dev(up), una, 3)
    compare(host(una), exp_[3], sc[3], tol=1e-13, what="stage 3 in place")


@pytest.mark.parametrize("wprec", ["fp64", "fp32", "fp16"])
def test_theta_weno_full_size_kerr(wprec):
    """theta-WENO option on the 2048 x 128 Kerr workload: 2 steps, every node."""
    got, exp_, sc = run_both(I.KERR_GRAV, wprec, 2, theta_mode=1)
    compare(got, exp_, sc, what=f"kerr theta-weno {wprec}")


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("phys", PHYS)
def test_fd6_ko8_operator_parity(shape, phys):
    """The comparison scheme (Sec. 3.1.1): FD6 derivative and KO8 dissipation."""
    nr, nth = shape
    a, s, m = phys
    rs0, rs1 = -40.0, 120.0
    for smooth in (True, False):
        u = I.multiscale_state(nr, nth, nr * 3 + nth, smooth)
        g = o.grid(nr, nth, rs0, rs1, 1.0, a, s, m, scheme=1, ko_sigma=0.2)
        co = o.coefficients(g)
        F = o.rhs(g, co, u)
        p = T.make_params(nr, nth, rs0, rs1, 1.0, a, s, m, scheme=1, ko_sigma=0.2)
        coef = dev(T.teuk_build_coefficients(p, 1.0))
        ud = dev(u)
        out = torch.empty_like(ud)
        T.teuk_stage_dev(p, 1.0, coef, None, ud, out, 0)
        compare(host(out), F, stage_scale(g, co, 1.0, u, with_prev=False),
                what=f"fd6 {shape} {phys} smooth={smooth}")


def test_fd6_ko8_full_size_kerr():
    got, exp_, sc = run_both(I.KERR_GRAV, "fp64", 3, scheme=1)
    compare(got, exp_, sc, what="kerr fd6")


@pytest.mark.parametrize("wprec", ["fp64", "fp32"])
def test_ssprk104_full_size_kerr(wprec):
    """SSP-RK(10,4) (two-register evaluation on the GPU) against the oracle's
    printed Shu-Osher form: 2048 x 128 Kerr workload, 2 steps, every node."""
    got, exp_, sc = run_both(I.KERR_GRAV, wprec, 2, rk=1)
    compare(got, exp_, sc, what=f"kerr ssprk104 {wprec}")


def test_ssprk104_handle_graph_matches_stateless():
    wl = I.KERR_GRAV.with_(nr=300, nth=24)
    p = T.params_from_workload(wl, wprec="fp32", rk=1)
    h = T.teuk_create(p)
    u0 = I.initial_data(wl)
    T.teuk_set_state(h, u0, 0.0)
    T.teuk_step(h, 19)
    ref, t = T.teuk_get_state(h)
    _, dt, _ = T.teuk_get_info(h)
    coef = dev(T.teuk_build_coefficients(p, dt))
    ud = dev(u0)
    work = torch.empty(3, 4, wl.nth, wl.nr, dtype=torch.float64, device="cuda")
    T.teuk_step_dev(p, dt, coef, ud, work, 19)
    np.testing.assert_array_equal(host(ud), ref)
    assert abs(t - 19 * dt) < 1e-12
    assert abs(dt / T.teuk_stable_dt(T.params_from_workload(wl, wprec="fp32")) - 2.8) < 1e-12
    with pytest.raises(T.TeukError):
        T.teuk_stage_dev(p, dt, coef, ud, ud, torch.empty_like(ud), 2)
    with pytest.raises(T.TeukError):
        T.teuk_step_dev_static(p, dt, coef, ud, 1)
    with pytest.raises(T.TeukError):
        T.teuk_batch_create([p])


@pytest.mark.parametrize("theta_mode", [0, 1])
@pytest.mark.parametrize("wprec", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("coords", [0, 1])
def test_scaled_second_stage_is_exact(coords, wprec, theta_mode):
    """The step keeps its second SSP-RK(3,3) stage as v = 4 u^(2) and runs the
    third on v with 16 eps and beta = 1/6. Data scaled by 4 with eps scaled by
    16 gives the same WENO weights and, by powers of two, the same roundings,
    so the step's result equals bit for bit the printed third stage (the
    public single-stage call) applied to v / 4; and v / 4 is the printed second
    stage up to its own roundings (one fewer per row). On multi-scale data
    (rows over 1e-40..1e6, a 1e-200 tail) in both coordinate systems."""
    wl = (I.KERR_GRAV.with_(nr=257, nth=13) if coords == 0
          else I.EXTREMAL_GRAV_HYP.with_(nr=300, nth=10))
    p = T.params_from_workload(wl, wprec=wprec, theta_mode=theta_mode)
    dt = 0.5 * T.teuk_stable_dt(p)
    coef = dev(T.teuk_build_coefficients(p, dt))
    u0 = I.multiscale_state(wl.nr, wl.nth, 13)
    ud = dev(u0)
    work = torch.zeros(2, 4, wl.nth, wl.nr, dtype=torch.float64, device="cuda")
    T.teuk_step_dev(p, dt, coef, ud, work, 1)
    u1, w1, v = host(ud), host(work[0]), host(work[1])
    third = torch.empty_like(ud)
    T.teuk_stage_dev(p, dt, coef, dev(u0), dev(v / 4.0), third, 3)
    np.testing.assert_array_equal(u1, host(third))
    second = torch.empty_like(ud)
    T.teuk_stage_dev(p, dt, coef, dev(u0), dev(w1), second, 2)
    g = o.grid(wl.nr, wl.nth, wl.rs_min, wl.rs_max, wl.M, wl.a, wl.s, wl.m, wl.eps, wprec,
               theta_mode, coords=wl.coords, S=wl.S)
    co = o.coefficients(g)
    compare(v / 4.0, host(second), stage_scale(g, co, dt, w1, u0, 0.75, 0.25), tol=1e-14,
            what=f"second stage {wprec}")


def run_both(wl, wprec, nsteps, u0=None, theta_mode=0, rk=0, scheme=0):
    """nsteps on the GPU (stateless step) and in the oracle."""
    g = o.grid(wl.nr, wl.nth, wl.rs_min, wl.rs_max, wl.M, wl.a, wl.s, wl.m, wl.eps, wprec,
               theta_mode, scheme=scheme)
    co = o.coefficients(g)
    dt = oracle_dt(g, co)
    u0 = I.initial_data(wl) if u0 is None else u0
    if rk == 1:
        dt *= 2.8
    p = T.params_from_workload(wl, wprec=wprec, theta_mode=theta_mode, rk=rk, scheme=scheme)
    coef = dev(T.teuk_build_coefficients(p, dt))
    ud = dev(u0)
    work = torch.empty(3, 4, wl.nth, wl.nr, dtype=torch.float64, device="cuda")
    T.teuk_step_dev(p, dt, coef, ud, work, nsteps)
    step = o.rk104_step if rk == 1 else o.rk3_step
    stages = (10 if rk == 1 else 3) * nsteps
    return host(ud), step(g, co, dt, u0, nsteps), run_scale(g, co, dt, u0, stages)


@pytest.mark.parametrize("wprec", ["fp64", "fp32"])
def test_full_size_kerr_gravitational(wprec):
    """2048 x 128, s=-2, m=2, a=0.999 (the benchmark workload), 3 steps,
    every node compared."""
    got, exp_, sc = run_both(I.KERR_GRAV, wprec, 3)
    compare(got, exp_, sc, what=f"kerr {wprec}")


@pytest.mark.parametrize("wprec", ["fp16", "bf16"])
def test_full_size_extremal_scalar(wprec):
    """8192 x 256, s=0, m=0, a=M, one step, every node compared."""
    got, exp_, sc = run_both(I.EXTREMAL_SCALAR, wprec, 1)
    compare(got, exp_, sc, what=f"extremal {wprec}")


def test_tail_workload_full_size_one_stage():
    """16384 x 512 (tail workload, binary32 weights): one stage, every node."""
    wl = I.TAIL_SCALAR
    u0 = I.initial_data(wl)
    g = o.grid(wl.nr, wl.nth, wl.rs_min, wl.rs_max, wl.M, wl.a, wl.s, wl.m, wl.eps, "fp32")
    p = T.params_from_workload(wl)
    dt = 0.05
    coef = dev(T.teuk_build_coefficients(p, dt))
    ud = dev(u0)
    out = torch.empty_like(ud)
    T.teuk_stage_dev(p, dt, coef, None, ud, out, 1)
    got = host(out)
    del out, ud, coef
    co = o.coefficients(g)
    exp_ = u0 + dt * o.rhs(g, co, u0)
    compare(got, exp_, stage_scale(g, co, dt, u0), what="tail workload")


def test_waveform_parity_schwarzschild_500_steps():
    """256 x 32, s=m=a=0, binary64 weights, 500 steps: waveform at r*=100 over
    the whole run, relative L2 <= 1e-12."""
    wl = I.SCHW_SCALAR
    g = o.grid(wl.nr, wl.nth, wl.rs_min, wl.rs_max, 1.0, 0.0, 0, 0, 1e-6, "fp64")
    co = o.coefficients(g)
    dt = oracle_dt(g, co)
    p = T.params_from_workload(wl, dt=dt)
    h = T.teuk_create(p)
    u = I.initial_data(wl)
    T.teuk_set_state(h, u, 0.0)
    wg, wo = [], []
    uo = u.copy()
    for _ in range(10):
        T.teuk_step(h, 50)
        wave, hor, t = T.teuk_observe(h, 100.0)
        wg.append(wave.copy())
        uo = o.rk3_step(g, co, dt, uo, 50)
        w2, _ = o.observe(g, uo, 100.0)
        wo.append(w2)
    wg, wo = np.array(wg), np.array(wo)
    rel = np.linalg.norm(wg - wo) / np.linalg.norm(wo)
    assert rel <= 1e-12, rel
    assert abs(t - 500 * dt) < 1e-9


def test_handle_checkpoint_and_graph_bitwise():
    wl = I.KERR_GRAV.with_(nr=300, nth=24)
    p = T.params_from_workload(wl, wprec="fp32")
    h1 = T.teuk_create(p)
    u0 = I.initial_data(wl)
    T.teuk_set_state(h1, u0, 0.0)
    T.teuk_step(h1, 37)                                   # graph (2 x 16) + 5 direct
    ref, t1 = T.teuk_get_state(h1)
    h2 = T.teuk_create(p)
    T.teuk_set_state(h2, u0, 0.0)
    T.teuk_step(h2, 20)
    mid, tm = T.teuk_get_state(h2)
    h3 = T.teuk_create(p)
    T.teuk_set_state(h3, mid, tm)
    T.teuk_step(h3, 17)
    res, t3 = T.teuk_get_state(h3)
    np.testing.assert_array_equal(res, ref)
    assert abs(t3 - t1) < 1e-12
    # stateless stepping with caller scratch gives the same bits
    _, dt, _ = T.teuk_get_info(h1)
    coef = dev(T.teuk_build_coefficients(p, dt))
    ud = dev(u0)
    work = torch.empty(2, 4, wl.nth, wl.nr, dtype=torch.float64, device="cuda")
    T.teuk_step_dev(p, dt, coef, ud, work, 37)
    np.testing.assert_array_equal(host(ud), ref)


def test_set_initial_and_observe():
    wl = I.KERR_GRAV.with_(nr=200, nth=16)
    p = T.params_from_workload(wl)
    h = T.teuk_create(p)
    u = I.initial_data(wl)
    T.teuk_set_initial(h, u[0] + 1j * u[1], u[2] + 1j * u[3])
    wave, hor, t = T.teuk_observe(h, 30.0)
    g = o.grid(wl.nr, wl.nth, wl.rs_min, wl.rs_max, 1.0, wl.a, wl.s, wl.m)
    w2, h2 = o.observe(g, u, 30.0)
    np.testing.assert_array_equal(wave, w2)
    np.testing.assert_allclose(hor, h2, rtol=1e-15, atol=0)
    assert t == 0.0


def test_nonfinite_state_is_reported():
    wl = I.SCHW_SCALAR
    h = T.teuk_create(T.params_from_workload(wl))
    u = I.initial_data(wl)
    T.teuk_set_state(h, u)
    assert T.teuk_check_finite(h) == T.TEUK_OK
    u[2, 5, 17] = np.nan                                  # host-made failure
    T.teuk_set_state(h, u)
    assert T.teuk_check_finite(h) == T.TEUK_ERR_NONFINITE
    u[2, 5, 17] = 0.0
    u[0, 3, 0] = np.inf
    T.teuk_set_state(h, u)
    with pytest.raises(T.TeukError) as ei:
        T.teuk_observe(h, 0.0)
    assert ei.value.status == T.TEUK_ERR_NONFINITE


def test_device_entry_points_reject_bad_arguments():
    p = T.make_params(64, 8)
    coef = dev(T.teuk_build_coefficients(p, 0.1))
    u = torch.zeros(4, 8, 64, dtype=torch.float64, device="cuda")
    out = torch.zeros_like(u)
    for stage, un, dt in [(4, None, 0.1), (2, None, 0.1), (1, None, 0.0)]:
        with pytest.raises(T.TeukError) as ei:
            T.teuk_stage_dev(p, dt, coef, un, u, out, stage)
        assert ei.value.status == T.TEUK_ERR_ARG
    with pytest.raises(T.TeukError):
        T.teuk_stage_dev(p, 0.1, coef, None, u, u, 1)       # out aliases u_prev
    # arrays too small for the grid are refused by the binding before the call
    short = torch.zeros(4 * 8 * 64 - 1, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        T.teuk_stage_dev(p, 0.1, coef, None, u, short, 1)
    with pytest.raises(ValueError):
        T.teuk_stage_dev(p, 0.1, coef[:-1], None, u, out, 1)
    with pytest.raises(ValueError):
        T.teuk_step_dev(p, 0.1, coef, u, short, 1)
    h = T.teuk_create(p)
    with pytest.raises(ValueError):
        T.teuk_set_state(h, np.zeros((4, 8, 63)))
    with pytest.raises(ValueError):
        T.teuk_get_state(h, np.zeros((4, 8, 63)))
    h.close()


@pytest.mark.parametrize("a,s,m", [(0.999, -2, 2), (0.0, 0, 0), (0.5, -1, 3)])
def test_set_gaussian_matches_python_construction(a, s, m):
    wl = I.KERR_GRAV.with_(nr=257, nth=33, a=a, s=s, m=m)
    p = T.params_from_workload(wl)
    h = T.teuk_create(p)
    coeffs = [0.7 - 0.2j, 1.1 + 0.4j, -0.3 + 0.9j]
    T.teuk_set_gaussian(h, 30.0, 3.0, coeffs)
    got, t = T.teuk_get_state(h)
    exp_ = I.gaussian_data(wl, 30.0, 3.0, coeffs)
    assert t == 0.0
    assert np.max(np.abs(got - exp_)) <= 1e-13 * np.max(np.abs(exp_))
    # seeded: amplitudes 0.5 + U, phases 2 pi U' from SplitMix64
    T.teuk_set_gaussian(h, -10.0, 4.0, None, nl=2, seed=2026)
    us = I.splitmix64_uniforms(2026, 4)
    seeded = [(0.5 + us[2 * k]) * np.exp(2j * np.pi * us[2 * k + 1]) for k in range(2)]
    got, _ = T.teuk_get_state(h)
    exp_ = I.gaussian_data(wl, -10.0, 4.0, seeded)
    assert np.max(np.abs(got - exp_)) <= 1e-13 * np.max(np.abs(exp_))


def test_async_host_copies_and_pipelined_handles():
    """teuk_set_state_async / teuk_get_state_async / teuk_synchronize: a round
    trip returns the data, and independent steps pipelined over three handles
    (each on its own stream) give bitwise the synchronous results."""
    wl = I.KERR_GRAV.with_(nr=300, nth=24)
    p = T.params_from_workload(wl, wprec="fp32")
    pinned = lambda: torch.empty((4, wl.nth, wl.nr), dtype=torch.float64, pin_memory=True).numpy()
    inputs = [I.initial_data(wl.with_(seed=k)) for k in range(7)]
    ref = []
    h0 = T.teuk_create(p)
    for u in inputs:
        T.teuk_set_state(h0, u, 0.0)
        T.teuk_step(h0, 2)
        ref.append(T.teuk_get_state(h0)[0])
    hs = [T.teuk_create(p) for _ in range(3)]
    ins = [pinned() for _ in range(3)]
    outs = [pinned() for _ in range(3)]
    got = [None] * len(inputs)
    owner = [None] * 3
    for i, u in enumerate(inputs):
        k = i % 3
        if owner[k] is not None:
            T.teuk_synchronize(hs[k])
            got[owner[k]] = outs[k].copy()
        ins[k][...] = u
        T.teuk_set_state_async(hs[k], ins[k], 0.0)
        T.teuk_step(hs[k], 2)
        T.teuk_get_state_async(hs[k], outs[k])
        owner[k] = i
    for k in range(3):
        T.teuk_synchronize(hs[k])
        got[owner[k]] = outs[k].copy()
    for g, r in zip(got, ref):
        np.testing.assert_array_equal(g, r)
    # round trip and the time set by the asynchronous call
    T.teuk_set_state_async(hs[0], ins[1], 4.5)
    T.teuk_get_state_async(hs[0], outs[0])
    T.teuk_synchronize(hs[0])
    np.testing.assert_array_equal(outs[0], ins[1])
    assert T.teuk_get_info(hs[0])[2] == 4.5
    with pytest.raises(ValueError):
        T.teuk_get_state_async(hs[0], np.empty((4, wl.nth, wl.nr), dtype=np.float32))


@pytest.mark.parametrize("wprec", ["fp32", "fp64"])
def test_benchmark_launch_configuration_against_oracle(wprec):
    """Exactly what bench.py times: the 2048 x 128 Kerr workload through a
    handle, the handle's own time step, one teuk_step call per step (the
    stage kernels launched with programmatic dependent launch); three steps,
    every node against the oracle."""
    wl = I.KERR_GRAV
    p = T.params_from_workload(wl, wprec=wprec)
    h = T.teuk_create(p)
    u0 = I.initial_data(wl)
    T.teuk_set_state(h, u0, 0.0)
    for _ in range(3):
        T.teuk_step(h, 1)
    got, t = T.teuk_get_state(h)
    _, dt, _ = T.teuk_get_info(h)
    g = o.grid(wl.nr, wl.nth, wl.rs_min, wl.rs_max, wl.M, wl.a, wl.s, wl.m, wl.eps, wprec)
    co = o.coefficients(g)
    compare(got, o.rk3_step(g, co, dt, u0, 3), run_scale(g, co, dt, u0, 9),
            what=f"bench configuration {wprec}")
    assert abs(t - 3 * dt) < 1e-12


def test_plain_c_client_steps_and_observes(tmp_path):
    """The C client (tests/c/teuk_c_client.c) drives a handle through the C ABI
    alone: seeded Gaussian data, 40 steps, observation, a bitwise checkpoint
    round trip, and a status for a bad call; its observation equals the same
    sequence issued through the Python binding."""
    import test_host_abi as H
    got = H._c_client(tmp_path)("gpu")
    assert got["restart_bitwise"] == "1"
    assert int(got["neg_steps_status"]) == T.TEUK_ERR_ARG
    p = T.params_from_workload(I.KERR_GRAV, wprec="fp32")
    h = T.teuk_create(p)
    T.teuk_set_gaussian(h, 30.0, 3.0, [1.0 + 0.5j])
    T.teuk_step(h, 40)
    wave, _, t = T.teuk_observe(h, 50.0)
    assert float(got["t"]) == t
    seq = 0.0
    for x in wave.ravel():                 # the client's order: (re, im) per row
        seq += abs(float(x))
    assert float(got["wave_abs_sum"]) == seq
    # the hyperboloidal handle created from the range [0, 0]
    rhop = I.horizon_rho(1.0, 1.0, 20.0)
    lo, hi = (float(x) for x in got["hyp_range"].split())
    assert lo == pytest.approx(rhop, rel=1e-15) and hi == 20.0
    q = T.make_params(512, 16, 0.0, 0.0, 1.0, 1.0, -2, 0, wprec="fp32",
                      coords=T.TEUK_COORDS_HYPERBOLOIDAL)
    hh = T.teuk_create(q)
    T.teuk_set_gaussian(hh, 1.0, 0.22, [1.0])
    T.teuk_step(hh, 20)
    _, hor, _ = T.teuk_observe(hh, 20.0)
    seq = 0.0
    for x in hor.ravel():
        seq += abs(float(x))
    assert float(got["hyp_horizon_abs_sum"]) == seq
