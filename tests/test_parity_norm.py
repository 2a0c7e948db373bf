"""Why the parity norm scales derivative fields by max(max |b|, max |avg| / h)
(tests/parity.py), measured on the oracle alone (not GPU).

A derivative field of the state is a difference quotient of interface values
whose size is that of the averages, so its rounding error is about
eps |avg| / h whatever its own size.  Here the oracle steps a state and the
same state with every entry moved by one unit in the last place, with the
same time step: a perturbation as small as one rounding.  Measured under the
plain norm (derivative fields relative to their own largest entry) that
rounding-sized input change already takes a third of the 1e-12 one-step bar
on the TGV, because the TGV's density and energy gradients are small beside
|avg| / h (Ma 0.1: density varies by 1e-3).  Two correct implementations
that round differently at thousands of operations per cell would breach it.
Under the class-scaled norm the same perturbation stays near 1e-14."""
import math

import numpy as np

import synth
from parity import class_scaled_diff

TGV = dict(mu=1 / 1600, prandtl=0.72, tau_mode=2)


def _ulp_pair(orc, dim, n, lo, hi, fn, kw, steps):
    a = orc.Oracle(dim, n, lo=lo, hi=hi, **kw)
    a.init(fn)
    s0 = a.get_state()
    dt = a.dt()
    rng = np.random.default_rng(1)
    s1 = s0 * (1 + rng.choice([-1.0, 1.0], size=s0.shape) * 2.0 ** -53)
    out = []
    for s in (s0, s1):
        o = orc.Oracle(dim, n, lo=lo, hi=hi, dt_fixed=dt, **kw)
        o.set_state(s)
        o.step(steps)
        out.append(o.get_state())
    h = min((hi[i] - lo[i]) / n[i] for i in range(dim))
    return class_scaled_diff(out[1], out[0]), class_scaled_diff(out[1], out[0], h)


def test_rounding_floor_of_the_two_norms(orc):
    plain, scaled = _ulp_pair(orc, 3, (12,) * 3, (0,) * 3, (2 * math.pi,) * 3,
                              lambda x, y, z: synth.taylor_green_3d(x, y, z), TGV, 1)
    print("TGV 12^3, one step after a one-ulp input change: plain %.2e, class-scaled %.2e" % (plain, scaled))
    assert plain > 1e-13  # within 10x of the 1e-12 bar from one rounding of the input
    assert scaled < 2e-14  # 50x inside the bar
    plain, scaled = _ulp_pair(orc, 2, (64, 64), (0, 0), (10, 10),
                              lambda x, y: synth.isentropic_vortex_2d(x, y), {}, 10)
    print("vortex 64^2, ten steps: plain %.2e, class-scaled %.2e" % (plain, scaled))
    assert plain > 10 * scaled
