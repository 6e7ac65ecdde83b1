"""Batched evolutions (one persistent launch per stage over all members):
every member must equal an independent single-evolution run bit for bit (the
per-node arithmetic does not depend on how nodes are tiled), and a member must
match the oracle within the parity tolerance, node by node (1e-12 of the size
of the terms over each node's domain of dependence, ``_local_scale``)."""
import numpy as np
import pytest

import oracle as o
import paper_2010_04760_gb300 as T
from paper_2010_04760_gb300 import inputs as I
from _local_scale import assert_local, run_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    T.lib()


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _single(wl, p, dt, nsteps):
    coef = _dev(T.teuk_build_coefficients(p, dt))
    u = _dev(I.initial_data(wl))
    work = torch.empty(2, 4, wl.nth, wl.nr, dtype=torch.float64, device="cuda")
    T.teuk_step_dev(p, dt, coef, u, work, nsteps)
    torch.cuda.synchronize()
    return u.cpu().numpy()


MEMBERS = [I.KERR_GRAV.with_(nr=300, nth=20, a=0.3, s=0, m=1, seed=11),
           I.KERR_GRAV.with_(nr=517, nth=9, seed=12),
           I.KERR_GRAV.with_(nr=64, nth=5, a=1.0, s=0, m=0, rc=-20.0, seed=13),
           I.KERR_GRAV.with_(nr=1000, nth=33, a=0.0, s=-2, m=0, seed=14),
           I.KERR_GRAV.with_(nr=129, nth=16, a=0.7, s=-1, m=3, ells=(3,), seed=15)]


@pytest.mark.parametrize("wprec", ["fp32", "fp64", "bf16"])
@pytest.mark.parametrize("autotune", [True, False])
def test_batch_members_equal_single_runs(wprec, autotune):
    ps = [T.params_from_workload(w, wprec=wprec) for w in MEMBERS]
    b = T.teuk_batch_create(ps, autotune=autotune)
    for k, w in enumerate(MEMBERS):
        T.teuk_batch_set_state(b, k, I.initial_data(w), 0.0)
    T.teuk_batch_step(b, 19)                     # one graph replay of 16 + 3 direct
    for k, w in enumerate(MEMBERS):
        dt, t, seg, ctas = T.teuk_batch_get_info(b, k)
        assert seg in (32, 64) and ctas in (4, 8)
        assert abs(t - 19 * dt) < 1e-12
        got, _ = T.teuk_batch_get_state(b, k)
        np.testing.assert_array_equal(got, _single(w, ps[k], dt, 19))


def test_batch_theta_weno_members_equal_single_runs():
    ps = [T.params_from_workload(w, wprec="fp32", theta_mode=1) for w in MEMBERS]
    b = T.teuk_batch_create(ps, autotune=True)
    for k, w in enumerate(MEMBERS):
        T.teuk_batch_set_state(b, k, I.initial_data(w), 0.0)
    T.teuk_batch_step(b, 7)
    for k, w in enumerate(MEMBERS):
        dt, _, _, _ = T.teuk_batch_get_info(b, k)
        got, _ = T.teuk_batch_get_state(b, k)
        np.testing.assert_array_equal(got, _single(w, ps[k], dt, 7))


HYP_MEMBERS = [I.EXTREMAL_GRAV_HYP.with_(nr=700, nth=16, seed=21),
               I.EXTREMAL_GRAV_HYP.with_(nr=257, nth=9, a=0.6, s=0, m=1, ells=(1,),
                                         rs_min=I.horizon_rho(1.0, 0.6, 20.0), seed=22),
               I.EXTREMAL_GRAV_HYP.with_(nr=1500, nth=24, a=0.3, s=-1, m=2, ells=(2,),
                                         rs_min=I.horizon_rho(1.0, 0.3, 20.0), seed=23)]


@pytest.mark.parametrize("theta_mode", [0, 1])
def test_batch_of_hyperboloidal_members_equal_single_runs(theta_mode):
    """Members on the hyperboloidal slices (the pi rows' own speed, quartic
    ghosts at the horizon and scri) advance in one batch exactly as alone."""
    ps = [T.params_from_workload(w, wprec="fp32", theta_mode=theta_mode) for w in HYP_MEMBERS]
    b = T.teuk_batch_create(ps, autotune=True)
    for k, w in enumerate(HYP_MEMBERS):
        T.teuk_batch_set_state(b, k, I.initial_data(w), 0.0)
    T.teuk_batch_step(b, 21)
    for k, w in enumerate(HYP_MEMBERS):
        dt, t, _, _ = T.teuk_batch_get_info(b, k)
        assert abs(t - 21 * dt) < 1e-12
        got, _ = T.teuk_batch_get_state(b, k)
        np.testing.assert_array_equal(got, _single(w, ps[k], dt, 21))


def test_batch_member_matches_oracle():
    w = MEMBERS[4]
    ps = [T.params_from_workload(x, wprec="fp32") for x in MEMBERS]
    b = T.teuk_batch_create(ps, autotune=False)
    for k, x in enumerate(MEMBERS):
        T.teuk_batch_set_state(b, k, I.initial_data(x), 0.0)
    T.teuk_batch_step(b, 5)
    dt, _, _, _ = T.teuk_batch_get_info(b, 4)
    got, _ = T.teuk_batch_get_state(b, 4)
    g = o.grid(w.nr, w.nth, w.rs_min, w.rs_max, w.M, w.a, w.s, w.m, w.eps, "fp32")
    co = o.coefficients(g)
    u0 = I.initial_data(w)
    exp_ = o.rk3_step(g, co, dt, u0, 5)
    assert_local(got, exp_, run_scale(g, co, dt, u0, 15), 1e-12, "batch member 4")


def test_batch_rejects_mixed_weight_precision():
    ps = [T.params_from_workload(MEMBERS[0], wprec="fp32"),
          T.params_from_workload(MEMBERS[1], wprec="fp16")]
    with pytest.raises(T.TeukError) as ei:
        T.teuk_batch_create(ps)
    assert ei.value.status == T.TEUK_ERR_ARG


def test_uneven_batch_of_64_evolutions():
    """The 64-member uneven batch (nr 1024..8192, ntheta 64..256, a in [0, M],
    s in {0, -2}, m in {0..4}, ~47 M nodes): 2 steps; three members compared bit
    for bit with single-evolution runs."""
    wls = I.batch_workloads()
    ps = [T.params_from_workload(w) for w in wls]
    b = T.teuk_batch_create(ps, autotune=True)
    for k, w in enumerate(wls):
        T.teuk_batch_set_state(b, k, I.initial_data(w), 0.0)
    T.teuk_batch_step(b, 2)
    for k in (0, 31, 63):
        dt, _, _, _ = T.teuk_batch_get_info(b, k)
        got, _ = T.teuk_batch_get_state(b, k)
        np.testing.assert_array_equal(got, _single(wls[k], ps[k], dt, 2))
    # one full-size member against the oracle, every node
    k = 31
    w = wls[k]
    dt, _, _, _ = T.teuk_batch_get_info(b, k)
    got, _ = T.teuk_batch_get_state(b, k)
    b.close()
    g = o.grid(w.nr, w.nth, w.rs_min, w.rs_max, w.M, w.a, w.s, w.m, w.eps, "fp32")
    co = o.coefficients(g)
    u0 = I.initial_data(w)
    exp_ = o.rk3_step(g, co, dt, u0, 2)
    assert_local(got, exp_, run_scale(g, co, dt, u0, 6), 1e-12,
                 f"batch member {k} ({w.nr} x {w.nth})")
