"""Out-of-bounds detection with NaN canaries (compute-sanitizer is not available
on this pool). Every buffer a stage reads lies inside a larger allocation whose
margins hold NaN, so a load outside the buffer would poison the result (a NaN
times a zero stencil weight is still NaN); the output buffer lies between
margins that hold a sentinel pattern, which a store outside it would change.
Each case must return finite values equal to the oracle's and leave every
margin untouched. Shapes are ragged (partial segments and row blocks) and
cover every kernel variant: both coordinate systems, both radial schemes,
both theta modes, binary64 and reduced weights, all stages, the stateless
step with its scratch arrays, and the in-place stage 3."""
import numpy as np
import pytest

import oracle as o
import paper_2010_04760_gb300 as T
from paper_2010_04760_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GUARD = 8192            # doubles of margin on each side of every buffer
SENTINEL = -7.25e300


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    T.lib()


def guarded(values, fill):
    """A device buffer holding `values` (flattened) with `fill` margins;
    returns (whole allocation, view of the payload)."""
    flat = np.ascontiguousarray(values, dtype=np.float64).ravel()
    whole = torch.full((flat.size + 2 * GUARD,), fill, dtype=torch.float64, device="cuda")
    view = whole[GUARD:GUARD + flat.size]
    view.copy_(torch.from_numpy(flat))
    return whole, view


def margins_hold(whole, n, fill):
    w = whole.cpu().numpy()
    lo, hi = w[:GUARD], w[GUARD + n:]
    if np.isnan(fill):
        return bool(np.all(np.isnan(lo)) and np.all(np.isnan(hi)))
    return bool(np.all(lo == fill) and np.all(hi == fill))


CASES = []
for shape in [(7, 5), (33, 6), (100, 13), (257, 33)]:
    for coords in (0, 1):
        for scheme in (0, 1):
            for theta in (0, 1):
                if scheme == 1 and theta == 1:
                    continue
                for wprec in (("fp64", "fp32") if scheme == 0 else ("fp64",)):
                    CASES.append((shape, coords, scheme, theta, wprec))


def _setup(shape, coords, scheme, theta, wprec):
    nr, nth = shape
    a, s, m = (0.9, -2, 1) if coords == 0 else (1.0, -2, 0)
    x0, x1 = (-30.0, 90.0) if coords == 0 else (I.horizon_rho(1.0, a, 20.0), 20.0)
    g = o.grid(nr, nth, x0, x1, 1.0, a, s, m, 1e-6, wprec, theta, scheme=scheme, ko_sigma=0.1,
               coords=coords, S=20.0)
    p = T.make_params(nr, nth, x0, x1, 1.0, a, s, m, wprec=wprec, theta_mode=theta,
                      scheme=scheme, ko_sigma=0.1, coords=coords, hyp_S=20.0)
    return g, p


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(map(str, c)))
def test_stages_stay_inside_their_buffers(case):
    shape, coords, scheme, theta, wprec = case
    nr, nth = shape
    g, p = _setup(*case)
    co = o.coefficients(g)
    dt = 0.01
    un = I.random_state(nr, nth, 3, smooth=False)
    up = I.random_state(nr, nth, 4, smooth=False)
    F = o.rhs(g, co, up)
    exp_ = {0: dt * F, 1: up + dt * F, 2: 0.75 * un + 0.25 * (up + dt * F),
            3: un / 3.0 + 2.0 / 3.0 * (up + dt * F)}
    coef_w, coef = guarded(T.teuk_build_coefficients(p, dt), float("nan"))
    un_w, un_d = guarded(un, float("nan"))
    up_w, up_d = guarded(up, float("nan"))
    n = 4 * nr * nth
    for stage in (0, 1, 2, 3):
        out_w, out = guarded(np.zeros(n), SENTINEL)
        T.teuk_stage_dev(p, dt, coef, un_d if stage >= 2 else None, up_d, out, stage)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(4, nth, nr)
        assert np.all(np.isfinite(got)), f"stage {stage}: a load left its buffer"
        assert margins_hold(out_w, n, SENTINEL), f"stage {stage}: a store left its buffer"
        speed = max(np.max(np.abs(co[0])), np.max(np.abs(co[9])), np.max(np.hypot(co[1], co[2])))
        scale = max(np.max(np.abs(exp_[stage])),
                    dt * speed * np.max(np.abs(up)) * (nr - 1) / (g.rs_max - g.rs_min))
        assert np.max(np.abs(got - exp_[stage])) <= 1e-12 * scale, stage
    for w in (coef_w, un_w, up_w):
        assert margins_hold(w, w.numel() - 2 * GUARD, float("nan"))
    # stage 3 in place on u^n (the library's own step layout)
    T.teuk_stage_dev(p, dt, coef, un_d, up_d, un_d, 3)
    torch.cuda.synchronize()
    np.testing.assert_allclose(un_d.cpu().numpy().reshape(4, nth, nr), exp_[3],
                               rtol=0, atol=1e-12 * np.max(np.abs(exp_[3])) + 1e-300)
    assert margins_hold(un_w, n, float("nan"))


@pytest.mark.parametrize("rk", [0, 1])
@pytest.mark.parametrize("coords", [0, 1])
def test_step_scratch_stays_inside_its_buffers(rk, coords):
    """teuk_step_dev with guarded state, coefficients and scratch arrays."""
    shape = (131, 9)
    nr, nth = shape
    g, p = _setup(shape, coords, 0, 0, "fp32")
    p.rk = rk
    co = o.coefficients(g)
    dt = 0.02
    u0 = I.random_state(nr, nth, 5)
    n = 4 * nr * nth
    coef_w, coef = guarded(T.teuk_build_coefficients(p, dt), float("nan"))
    u_w, u = guarded(u0, float("nan"))
    scratch = 3 if rk == 1 else 2
    work_w, work = guarded(np.zeros(scratch * n), SENTINEL)
    T.teuk_step_dev(p, dt, coef, u, work.view(scratch, 4, nth, nr), 3)
    torch.cuda.synchronize()
    step = o.rk104_step if rk == 1 else o.rk3_step
    ref = step(g, co, dt, u0, 3)
    got = u.cpu().numpy().reshape(4, nth, nr)
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))
    assert margins_hold(u_w, n, float("nan")) and margins_hold(coef_w, coef.numel(), float("nan"))
    assert margins_hold(work_w, scratch * n, SENTINEL)
