"""Failure status and restart through the C-ABI (failure detection on the
host side: nothing here faults the GPU).

- A non-physical state handed to cgks_set_state (a NaN, a negative pressure)
  makes cgks_step return CGKS_ENONPHYS and leaves that state as it was; the
  context stays usable after a fresh cgks_set_state.
- A run that turns non-physical part-way through one cgks_step call (a
  seeded four-quadrant Riemann problem that the plain method cannot advance,
  in the oracle as well) returns CGKS_ENONPHYS with the last good state of
  the call and its time: the same state, bit for bit, as a fresh context
  stepped to that time, within the parity bar of the oracle's state after
  the same steps, and physical in every cell.
- N + M steps in one run equal, bit for bit, N steps, cgks_get_state,
  cgks_set_state into a fresh context, then M steps (every form).
"""
import math

import numpy as np
import pytest

import synth
from parity import class_scaled_diff

pytestmark = pytest.mark.gpu
ENONPHYS = -4


@pytest.fixture(scope="module")
def cg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_08965_gb300 as p
    p.lib()
    return p


def _vortex_mesh(cg, precision):
    m = cg.Mesh(2, (32, 24), lo=(0, 0), hi=(10, 10), precision=precision)
    m.init(lambda x, y: synth.isentropic_vortex_2d(x, y))
    return m


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("bad", ["nan-density", "negative-pressure"])
def test_injected_nonphysical_state(orc, cg, precision, bad):
    m = _vortex_mesh(cg, precision)
    good, _ = m.get_state()
    s = good.copy()
    if bad == "nan-density":
        s[0, 0, 7, 11] = np.nan
    else:
        s[0, 3, 20, 3] = -0.5  # total energy below the kinetic energy
    m.set_state(s, 0.25)
    seen, _ = m.get_state()  # the state as the context holds it (FP32 form: derivative fields rounded)
    with pytest.raises(cg.CgksError) as ex:
        m.step(3)
    assert ex.value.status == ENONPHYS
    after, t = m.get_state()
    assert t == 0.25
    assert np.array_equal(after, seen, equal_nan=True)
    # the context is usable again after a fresh state
    m.set_state(good, 0.0)
    m.step(1)
    sg, _ = m.get_state()
    m.close()
    o = orc.Oracle(2, (32, 24), lo=(0, 0), hi=(10, 10))
    o.set_state(good)
    o.step(1)
    assert class_scaled_diff(sg, o.get_state(), 10 / 32) <= (1e-5 if precision == 1 else 1e-12)


RIEMANN = dict(dim=2, n=(32, 32), lo=(0, 0), hi=(1, 1), bc=[1, 1, 1, 1], tau_mode=1)


def _riemann_field():
    st = synth.riemann4_params(28)  # fails after a few steps at 32^2, in the oracle as well
    return lambda x, y: synth.riemann4_2d(x, y, st)


def _physical(s):
    rho = s[0, 0]
    ke = 0.5 * (s[0, 1] ** 2 + s[0, 2] ** 2) / rho
    p = 0.4 * (s[0, 3] - ke)
    return bool(np.all(rho > 0) and np.all(p > 0))


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_midrun_failure_returns_last_good_step(orc, cg, precision):
    m = cg.Mesh(precision=precision, **RIEMANN)
    m.init(_riemann_field())
    with pytest.raises(cg.CgksError) as ex:
        m.step(60)
    assert ex.value.status == ENONPHYS
    sg, tg = m.get_state()
    m.close()
    assert tg > 0.0 and _physical(sg)
    # a fresh context stepped one call at a time reaches the same time with
    # the same state, bit for bit
    r = cg.Mesh(precision=precision, **RIEMANN)
    r.init(_riemann_field())
    j = 0
    while True:
        t, _ = r.step(1)
        j += 1
        if t >= tg:
            break
    assert t == tg
    sr, _ = r.get_state()
    r.close()
    assert np.array_equal(sg, sr)
    # the failure is real: the returned state cannot be advanced much further
    f = cg.Mesh(precision=precision, **RIEMANN)
    f.set_state(sg, tg)
    with pytest.raises(cg.CgksError):
        f.step(3)
    f.close()
    # and it is the oracle's state after the same j steps
    o = orc.Oracle(**RIEMANN)
    o.init(_riemann_field())
    o.step(j)
    # the FP32 form's time steps follow its FP32-rounded states
    tol, tol_t = (1e-5, 1e-6) if precision == 1 else (1e-10, 1e-13)
    assert abs(o.time() - tg) <= tol_t * tg
    assert class_scaled_diff(sg, o.get_state(), 1 / 32) <= tol


TGV = dict(dim=3, n=(12, 10, 11), lo=(0, 0, 0), hi=(2 * math.pi,) * 3, mu=1 / 1600, prandtl=0.72, tau_mode=2)


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("case", ["tgv", "walls-2d"])
def test_checkpoint_restart_is_bitwise(cg, precision, case):
    if case == "tgv":
        kw, fn = TGV, (lambda x, y, z: synth.taylor_green_3d(x, y, z))
    else:
        # a resting vortex in a box with slip and no-slip walls, viscous
        kw = dict(dim=2, n=(24, 20), lo=(0, 0), hi=(10, 10), bc=[2, 3, 2, 3], mu=1e-3, prandtl=0.72, tau_mode=2)
        fn = lambda x, y: synth.isentropic_vortex_2d(x, y, u_inf=(0.0, 0.0))
    N, M = 3, 4
    a = cg.Mesh(precision=precision, **kw)
    a.init(fn)
    a.step(N + M)
    sa, ta = a.get_state()
    a.close()
    b = cg.Mesh(precision=precision, **kw)
    b.init(fn)
    b.step(N)
    ck, tk = b.get_state()
    b.close()
    c = cg.Mesh(precision=precision, **kw)
    c.set_state(ck, tk)
    c.step(M)
    sc, tc = c.get_state()
    c.close()
    assert tc == ta
    assert np.array_equal(sa, sc)
