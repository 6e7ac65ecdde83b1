"""The fused persistent step (every SSP-RK(3,3) stage of up to 1024 steps in
one launch, work items ordered by per-item completion flags) against the
stage-per-launch path: the per-node arithmetic is the same, only the schedule
differs, so the states must agree bit for bit, on ragged grids (theta rows not
a multiple of the 4-row block, radial nodes not a multiple of the segment),
grids with fewer work items than resident blocks, both coordinate systems,
both theta modes and all four weight formats, and across launches (more than
1024 steps). The timeout path is exercised with a completion flag that
nothing sets: the waits run out, the launch stops, the next synchronising
call returns TEUK_ERR_TIMEOUT, and the handle recovers after teuk_set_state."""
import numpy as np
import pytest

import paper_2010_04760_gb300 as T
from paper_2010_04760_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    T.lib()


def _run(p, u0, nsteps, mode):
    h = T.teuk_create(p)
    T.teuk_set_launch(h, mode)
    assert T.teuk_get_launch(h)[0] == mode
    assert T.teuk_get_launch(h)[2] == (1 if mode == T.TEUK_LAUNCH_FUSED else 0)
    T.teuk_set_state(h, u0, 0.0)
    T.teuk_step(h, nsteps)
    u, t = T.teuk_get_state(h)
    h.close()
    return u, t


CASES = [
    # (workload, weights, theta mode, steps)
    (I.KERR_GRAV, "fp32", 0, 5),                                   # the benchmark grid
    (I.KERR_GRAV.with_(nr=333, nth=13), "fp64", 0, 9),             # ragged, binary64 weights
    (I.KERR_GRAV.with_(nr=257, nth=6, a=0.5, s=-1, m=3, ells=(3,)), "fp16", 1, 7),
    (I.KERR_GRAV.with_(nr=64, nth=5, a=1.0, s=0, m=0, rc=-20.0), "bf16", 0, 11),
    (I.SCHW_SCALAR, "fp32", 1, 6),
    (I.EXTREMAL_GRAV_HYP.with_(nr=1500, nth=22), "fp32", 0, 8),    # horizon to scri
    (I.EXTREMAL_GRAV_HYP.with_(nr=700, nth=9), "bf16", 1, 5),
    (I.EXTREMAL_GRAV_HYP.with_(nr=300, nth=16), "fp64", 0, 4),
    # grids with enough 64-node items that the fused kernel takes 64-node segments
    (I.EXTREMAL_GRAV_HYP, "fp32", 0, 3),                           # the paper's 16384 x 64
    (I.EXTREMAL_SCALAR, "bf16", 0, 2),                             # 8192 x 256
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_fused_step_equals_stage_launches(case):
    wl, wprec, theta, nsteps = CASES[case]
    p = T.params_from_workload(wl, wprec=wprec, theta_mode=theta)
    u0 = I.initial_data(wl)
    ref, t_ref = _run(p, u0, nsteps, T.TEUK_LAUNCH_STAGES)
    got, t_got = _run(p, u0, nsteps, T.TEUK_LAUNCH_FUSED)
    np.testing.assert_array_equal(got, ref)
    assert t_got == t_ref


def test_fused_step_across_launches_and_calls():
    """2100 steps in one call (three launches: the epoch base advances between
    them) and the same in uneven calls, against the stage launches."""
    wl = I.SCHW_SCALAR.with_(nr=96, nth=8)
    p = T.params_from_workload(wl, wprec="fp32")
    u0 = I.initial_data(wl)
    ref, _ = _run(p, u0, 2100, T.TEUK_LAUNCH_STAGES)
    got, _ = _run(p, u0, 2100, T.TEUK_LAUNCH_FUSED)
    np.testing.assert_array_equal(got, ref)
    h = T.teuk_create(p)
    T.teuk_set_launch(h, T.TEUK_LAUNCH_FUSED)
    T.teuk_set_state(h, u0, 0.0)
    for k in (1, 2, 1023, 1, 1024, 49):
        T.teuk_step(h, k)
    got2, _ = T.teuk_get_state(h)
    np.testing.assert_array_equal(got2, ref)


def test_auto_launch_choice():
    """AUTO: the fused step on grids with at least as many work items per
    stage as resident blocks (the benchmark grid, 2048 work items), stage
    launches otherwise (the 256 x 32 grid, 64 items; binary64 weights on the
    benchmark grid, 1024 items of 64-node segments)."""
    h = T.teuk_create(T.params_from_workload(I.KERR_GRAV, wprec="fp32"))
    assert T.teuk_get_launch(h) == (T.TEUK_LAUNCH_AUTO, 2.0, 1)
    h = T.teuk_create(T.params_from_workload(I.KERR_GRAV, wprec="fp64"))
    assert T.teuk_get_launch(h) == (T.TEUK_LAUNCH_AUTO, 2.0, 0)
    p = T.params_from_workload(I.SCHW_SCALAR)
    h = T.teuk_create(p)
    assert T.teuk_get_launch(h) == (T.TEUK_LAUNCH_AUTO, 2.0, 0)
    for over in (dict(rk=T.TEUK_RK_SSP104), dict(scheme=T.TEUK_SCHEME_FD6_KO8)):
        h2 = T.teuk_create(T.params_from_workload(I.SCHW_SCALAR, **over))
        assert T.teuk_get_launch(h2)[2] == 0
        with pytest.raises(T.TeukError) as ei:
            T.teuk_set_launch(h2, T.TEUK_LAUNCH_FUSED)
        assert ei.value.status == T.TEUK_ERR_ARG
        with pytest.raises(T.TeukError):
            T.teuk_test_withhold(h2)
    with pytest.raises(T.TeukError):
        T.teuk_set_launch(h, 7)
    with pytest.raises(T.TeukError):
        T.teuk_set_launch(h, T.TEUK_LAUNCH_FUSED, 0.0)


@pytest.mark.parametrize("coords", [0, 1])
def test_fused_wait_timeout_is_reported_and_recovers(coords):
    """A flag that nothing sets (teuk_test_withhold): the dependent waits run
    out after 20 ms, every block stops, teuk_synchronize returns
    TEUK_ERR_TIMEOUT, and after teuk_set_state the handle steps exactly like a
    fresh one."""
    wl = (I.KERR_GRAV.with_(nr=512, nth=24) if coords == 0
          else I.EXTREMAL_GRAV_HYP.with_(nr=512, nth=24))
    p = T.params_from_workload(wl, wprec="fp32")
    u0 = I.initial_data(wl)
    h = T.teuk_create(p)
    T.teuk_set_launch(h, T.TEUK_LAUNCH_FUSED, 0.02)
    T.teuk_set_state(h, u0, 0.0)
    T.teuk_test_withhold(h)
    T.teuk_step(h, 3)
    with pytest.raises(T.TeukError) as ei:
        T.teuk_synchronize(h)
    assert ei.value.status == T.TEUK_ERR_TIMEOUT
    assert "ran out" in str(ei.value)
    T.teuk_synchronize(h)                      # reported once
    T.teuk_set_state(h, u0, 0.0)
    T.teuk_step(h, 6)
    got, _ = T.teuk_get_state(h)
    ref, _ = _run(p, u0, 6, T.TEUK_LAUNCH_STAGES)
    np.testing.assert_array_equal(got, ref)
