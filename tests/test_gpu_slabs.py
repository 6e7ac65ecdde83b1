"""The paper spreads its radial grid over GPUs in slabs (Sec. 4.1, MPI domain
decomposition). The stage operator reaches three nodes each way in the radial
direction (the WENO5 stencil of a node spans its neighbours i-3..i+3), so a
slab that carries three halo nodes on each inner side, refilled from its
neighbour after every Runge-Kutta stage, reproduces the undivided evolution
exactly. Here the slabs are evolved on one GPU through the single-stage entry
point (the printed SSP-RK(3,3) stages), each with its own columns of the
undivided grid's coefficient planes, and the halos are exchanged by device
copies; the interiors must equal the undivided run bit for bit, in r* (edge
copies at the outer ends) and on the hyperboloidal slices (quartic
extrapolation at the horizon and at scri), for two and four slabs of uneven
widths."""
import numpy as np
import pytest

import paper_2010_04760_gb300 as T
from paper_2010_04760_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HALO = 3


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    T.lib()


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _stages(p, dt, coef, u, w1, w2):
    """One printed SSP-RK(3,3) step through the single-stage entry point,
    with a hook after every stage (the halo exchange)."""
    yield T.teuk_stage_dev(p, dt, coef, None, u, w1, 1), w1
    yield T.teuk_stage_dev(p, dt, coef, u, w1, w2, 2), w2
    yield T.teuk_stage_dev(p, dt, coef, u, w2, u, 3), u


@pytest.mark.parametrize("coords", [0, 1])
@pytest.mark.parametrize("cuts", [(250,), (90, 301, 455)])
def test_radial_slabs_with_three_node_halos_are_exact(coords, cuts):
    wl = (I.KERR_GRAV.with_(nr=600, nth=12) if coords == 0
          else I.EXTREMAL_GRAV_HYP.with_(nr=600, nth=12))
    p = T.params_from_workload(wl, wprec="fp32")
    dt = 0.5 * T.teuk_stable_dt(p)
    coef_full = T.teuk_build_coefficients(p, dt)
    u0 = I.initial_data(wl)
    steps = 12
    # the undivided run
    u = _dev(u0)
    w1, w2 = torch.empty_like(u), torch.empty_like(u)
    cf = _dev(coef_full)
    for _ in range(steps):
        for _ in _stages(p, dt, cf, u, w1, w2):
            pass
    ref = u.cpu().numpy()
    # slabs: interior [lo, hi), arrays over [lo - halo, hi + halo) clipped to the grid
    edges = [0, *cuts, wl.nr]
    x = I.rstar_nodes(wl.nr, wl.rs_min, wl.rs_max)
    slabs = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        a, b = max(lo - HALO, 0), min(hi + HALO, wl.nr)
        ps = T.params_from_workload(wl, wprec="fp32", nr=b - a, rstar_min=float(x[a]),
                                    rstar_max=float(x[b - 1]))
        us = _dev(u0[..., a:b])
        slabs.append(dict(lo=lo, hi=hi, a=a, b=b, p=ps, coef=_dev(coef_full[..., a:b]), u=us,
                          w1=torch.empty_like(us), w2=torch.empty_like(us)))

    def exchange(bufs):
        """Refill every slab's halo columns from the neighbours' interiors."""
        for k, s in enumerate(slabs):
            for n in (k - 1, k + 1):
                if 0 <= n < len(slabs):
                    t = slabs[n]
                    lo, hi = max(s["a"], t["lo"]), min(s["b"], t["hi"])
                    if lo < hi:
                        bufs[k][..., lo - s["a"]:hi - s["a"]] = bufs[n][..., lo - t["a"]:hi - t["a"]]

    for _ in range(steps):
        gens = [_stages(s["p"], dt, s["coef"], s["u"], s["w1"], s["w2"]) for s in slabs]
        for _stage in range(3):
            outs = [next(g)[1] for g in gens]
            exchange(outs)
    torch.cuda.synchronize()
    for s in slabs:
        got = s["u"].cpu().numpy()[..., s["lo"] - s["a"]:s["hi"] - s["a"]]
        np.testing.assert_array_equal(got, ref[..., s["lo"]:s["hi"]])
