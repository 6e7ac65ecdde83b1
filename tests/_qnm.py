"""Test helpers for the quasinormal-ringing pins: the golden frequencies and
Prony's linear-prediction fit of damped complex exponentials."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "qnm_frequencies.txt")


def golden_qnm():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                s, l, m, a, wr, g = line.split()
                rows.append((int(s), int(l), int(m), float(a), float(wr), float(g)))
    return rows


def prony_modes(ts, y, t0, t1, order=6):
    """(gamma, omega) of the `order` exponentials y ~ sum c exp((-gamma + i
    omega) t) that best predict the samples in [t0, t1] (uniform spacing)."""
    sel = (ts >= t0) & (ts <= t1)
    y = np.asarray(y)[sel]
    dt = ts[1] - ts[0]
    A = np.array([y[k:k + order][::-1] for k in range(len(y) - order)])
    coef, *_ = np.linalg.lstsq(A, y[order:], rcond=None)
    z = np.roots(np.concatenate([[1.0], -coef]))
    s = np.log(z.astype(complex)) / dt
    return [(-x.real, x.imag) for x in s]


def nearest_mode(modes, omega_r, gamma, signed=False):
    """The fitted mode nearest (omega_r, gamma); with signed=False the sign
    of the frequency is ignored (real fields ring with +-omega)."""
    def dist(md):
        g, w = md
        w = w if signed else abs(w)
        return abs(w - omega_r) / omega_r + abs(g - gamma) / gamma
    return min(modes, key=dist)
