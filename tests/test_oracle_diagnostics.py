"""TGV diagnostics of Sec. 6.2 (not GPU): on the initial Taylor-Green field
the volume-averaged kinetic energy tends to 1/8 and the enstrophy term to
mu 3/4 (the averages of (u^2 + v^2)/2 and of |curl U|^2 of the field), at
second order in h for the cell-centred quadrature."""
import math

import numpy as np

import synth
from oracle.diagnostics import tgv_diagnostics


def _diag(orc, n):
    mu = 1 / 1600
    o = orc.Oracle(3, (n, n, n), lo=(0, 0, 0), hi=(2 * math.pi,) * 3, mu=mu)
    o.init(lambda x, y, z: synth.taylor_green_3d(x, y, z))
    vol, _ = o.metrics()
    return tgv_diagnostics(o.get_state(), 3, vol, mu), mu


def test_tgv_initial_diagnostics_converge(orc):
    (ek1, es1), mu = _diag(orc, 12)
    (ek2, es2), _ = _diag(orc, 24)
    e1, e2 = abs(ek1 - 0.125), abs(ek2 - 0.125)
    s1, s2 = abs(es1 / mu - 0.75), abs(es2 / mu - 0.75)
    assert e2 < 2.5e-3 and s2 < 1.5e-2
    assert 3.0 < e1 / e2 < 5.0 and 3.0 < s1 / s2 < 5.0
