"""Boundary pins of the oracle (not GPU).

B5  Inflow: a matching uniform state stays uniform; a stationary normal shock
    between supersonic inflow and outflow stays in place.

B1  Slip wall = mirror symmetry: a walled box evolves exactly like the upper
    half of the periodic box of twice the length holding the state and its
    mirror image (reflection symmetry of the Euler equations), in 2-D and 3-D,
    linear and nonlinear.
B2  No-slip wall, viscous: a shear wave between two walls decays at the
    Stokes rate exp(-nu pi^2 t).
B3  A closed box of walls conserves mass and energy.
B4  Outflow: a uniform moving state stays uniform; Sod's problem in a box with
    outflow ends against the exact Riemann solution.
"""
import math

import numpy as np
import pytest

import mirror
import riemann_exact
from parity import class_scaled_diff

SLIP, NOSLIP, OUTFLOW = 2, 3, 1


def _smooth2(x, y):
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * x + 0.3) * np.cos(2 * np.pi * y)
    u = 0.3 * np.sin(np.pi * x) + 0.1 * np.cos(2 * np.pi * y + 0.7) * x
    v = 0.2 * np.cos(2 * np.pi * y) + 0.1 * x
    p = 1.0 + 0.1 * np.cos(2 * np.pi * x - 0.4)
    return [rho, u, v, p]


def _smooth3(x, y, z):
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * x + 0.3) * np.cos(2 * np.pi * y) + 0.1 * z
    u = 0.2 * np.cos(2 * np.pi * y) + 0.1 * z
    v = 0.2 * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * z + 0.2)
    w = 0.3 * np.sin(np.pi * z) * (1.0 + 0.2 * np.cos(2 * np.pi * x))
    p = 1.0 + 0.1 * np.cos(2 * np.pi * z - 0.4) + 0.05 * np.sin(2 * np.pi * y)
    return [rho, u, v, w, p]


def _wall_vs_doubled(orc, dim, n, a, field, noslip=False, steps=3, **kw):
    lo = [0.0] * dim
    hi = [1.0] * dim
    bc = [0] * 6
    bc[2 * a] = bc[2 * a + 1] = NOSLIP if noslip else SLIP
    w = orc.Oracle(dim, n, lo=lo, hi=hi, bc=bc, **kw)
    w.init(field)
    n2 = list(n)
    n2[a] *= 2
    lo2 = list(lo)
    lo2[a] = -1.0
    p = orc.Oracle(dim, n2, lo=lo2, hi=hi, **kw)
    p.set_state(mirror.extend(w.get_state(), dim, a, noslip))
    for _ in range(steps):
        dt = w.dt()
        assert abs(p.dt() - dt) <= 1e-13 * dt
        w.step_dt(dt)
        p.step_dt(dt)
    sw, sp = w.get_state(), p.get_state()
    h = 1.0 / n[a]
    up = mirror.upper_half(sp, dim, a)
    lowm = mirror.reflect(np.take(sp, np.arange(n[a]), axis=2 + dim - 1 - a), dim, a, noslip)
    return class_scaled_diff(sw, up, h), class_scaled_diff(lowm, sw, h)


@pytest.mark.parametrize("linear", [True, False])
@pytest.mark.parametrize("a", [0, 1])
def test_slip_wall_is_mirror_symmetry_2d(orc, linear, a):
    d_up, d_lo = _wall_vs_doubled(orc, 2, (12, 10), a, _smooth2, linear=linear)
    assert d_up < 1e-12 and d_lo < 1e-12


def test_slip_wall_is_mirror_symmetry_3d(orc):
    d_up, d_lo = _wall_vs_doubled(orc, 3, (6, 5, 8), 2, _smooth3, steps=2)
    assert d_up < 1e-12 and d_lo < 1e-12


def test_slip_wall_shock_capturing(orc):
    """Nonlinear weights, shock-capturing collision time and a jump next to
    the wall still commute with the reflection."""
    def jump(x, y):
        rho = np.where(x < 0.3, 1.0, 0.4) + 0.05 * np.sin(2 * np.pi * y)
        p = np.where(x < 0.3, 1.0, 0.3)
        return [rho, 0.2 + 0 * x, 0.1 * np.cos(2 * np.pi * y), p]
    d_up, d_lo = _wall_vs_doubled(orc, 2, (16, 6), 0, jump, tau_mode=1, steps=4)
    assert d_up < 1e-11 and d_lo < 1e-11


def test_noslip_wall_stokes_shear_decay(orc):
    """A shear wave v = A sin(pi x) between no-slip walls at x = 0 and 1 decays
    as exp(-nu pi^2 t) (Stokes; at Ma 0.1 and A = 0.05 the compressible
    corrections are far below the tolerance).  The wall makes v vanish at
    the walls; slip walls, which let it slide, miss the rate by about 1 %."""
    A, mu, gamma, T = 0.05, 0.01, 1.4, 0.5
    p0 = 1.0 / (gamma * 0.1 ** 2)
    exact = np.exp(-mu * np.pi ** 2 * T)
    rel = {}
    for kind in (NOSLIP, SLIP):
        for n in ((8, 16) if kind == NOSLIP else (8,)):
            h = 1.0 / n
            o = orc.Oracle(2, (n, 4), lo=(0, 0), hi=(1, 4 * h), bc=[kind, kind, 0, 0], mu=mu,
                           tau_mode=2)
            o.init(lambda x, y: [1 + 0 * x, 0 * x, A * np.sin(np.pi * x), p0 + 0 * x])
            o.advance_to(T)
            s = o.get_state()
            xl = np.arange(n) * h
            mode = A * (np.cos(np.pi * xl) - np.cos(np.pi * (xl + h))) / (np.pi * h)
            v = s[0, 2, 0, :] / s[0, 0, 0, :]
            rel[kind, n] = abs((v @ mode) / (mode @ mode) / exact - 1.0)
    assert rel[NOSLIP, 8] < 5e-5 and rel[NOSLIP, 16] < 5e-6
    assert rel[NOSLIP, 16] < rel[NOSLIP, 8]
    assert rel[SLIP, 8] > 5e-3


@pytest.mark.parametrize("kind", [SLIP, NOSLIP])
def test_closed_box_conserves_mass_and_energy(orc, kind):
    o = orc.Oracle(2, (12, 10), bc=[kind] * 4, mu=1e-3 if kind == NOSLIP else 0.0,
                   tau_mode=2 if kind == NOSLIP else 0)
    o.init(_smooth2)
    vol = 1.0 / 120
    s0 = o.get_state()
    o.step(5)
    s1 = o.get_state()
    for v in (0, 3):
        m0, m1 = s0[0, v].sum() * vol, s1[0, v].sum() * vol
        assert abs(m1 - m0) <= 1e-13 * abs(m0)


def test_closed_box_3d_noslip_conserves(orc):
    o = orc.Oracle(3, (5, 4, 6), bc=[NOSLIP, NOSLIP, SLIP, SLIP, NOSLIP, NOSLIP], mu=1e-3,
                   tau_mode=2, prandtl=0.72)
    o.init(_smooth3)
    s0 = o.get_state()
    o.step(2)
    s1 = o.get_state()
    for v in (0, 4):
        assert abs(s1[0, v].sum() - s0[0, v].sum()) <= 1e-13 * abs(s0[0, v].sum())


def test_outflow_keeps_uniform_moving_state(orc):
    o = orc.Oracle(2, (8, 6), bc=[OUTFLOW] * 4)
    o.init(lambda x, y: [1.2 + 0 * x, 0.7 + 0 * x, -0.4 + 0 * x, 0.9 + 0 * x])
    s0 = o.get_state()
    o.step(4)
    s1 = o.get_state()
    assert np.abs(s1 - s0).max() < 1e-13


def test_outflow_sod_against_exact_riemann(orc):
    """Sod on [0, 1] with outflow at both ends: the waves reach neither end by
    t = 0.2, so the boundary must not disturb the exact solution."""
    L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)

    def init(x, y):
        left = x < 0.5
        return [np.where(left, L[0], R[0]), 0 * x, 0 * x, np.where(left, L[2], R[2])]

    errs = []
    for nx in (100, 200):
        h = 1.0 / nx
        o = orc.Oracle(2, (nx, 2), lo=(0, 0), hi=(1, 2 * h), tau_mode=1,
                       bc=[OUTFLOW, OUTFLOW, 0, 0])
        o.init(init)
        o.advance_to(0.2)
        s = o.get_state()
        rho = s[0, 0, 0, :]
        xc = (np.arange(nx) + 0.5) * h
        ex = riemann_exact.sample(L, R, xc, 0.2, x0=0.5)
        errs.append(np.mean(np.abs(rho - ex[0])))
        assert abs(rho[0] - 1.0) < 1e-12 and abs(rho[-1] - 0.125) < 1e-12
    assert errs[1] < errs[0] < 0.01


def test_bad_boundary_codes_rejected(orc):
    with pytest.raises(RuntimeError):
        orc.Oracle(2, (4, 4), bc=[7, 7, 0, 0])
    with pytest.raises(RuntimeError):
        orc.Oracle(2, (4, 4), bc=[SLIP, 0, 0, 0])


def test_strong_riemann_first_order_fallback(orc):
    """Four-quadrant data whose jumps defeat even the chi = 0 polynomial in
    the first step: the first-order fallback keeps every average physical
    (rho > 0, p > 0) and the domain sums of an outflow box change only
    through the boundary."""
    import synth
    states = synth.riemann4_params(328031897)
    o = orc.Oracle(2, (32, 32), bc=[OUTFLOW] * 4, tau_mode=1)
    o.init(lambda x, y: synth.riemann4_2d(x, y, states))
    for _ in range(20):
        o.step(1)
    s = o.get_state()
    rho, m, E = s[0, 0], s[0, 1:3], s[0, 3]
    p = 0.4 * (E - 0.5 * (m * m).sum(0) / rho)
    assert o.positivity_fallbacks() > 0
    assert rho.min() > 0 and p.min() > 0 and np.all(np.isfinite(s))


INFLOW = 4


def _cons(rho, u, v, p, gamma=1.4):
    return (rho, rho * u, rho * v, p / (gamma - 1) + 0.5 * rho * (u * u + v * v))


def test_inflow_keeps_matching_uniform_state(orc):
    q = (1.1, 0.6, -0.2, 0.9)
    o = orc.Oracle(2, (10, 6), bc=[INFLOW, OUTFLOW, 0, 0], bc_state=[_cons(*q)])
    o.init(lambda x, y: [q[0] + 0 * x, q[1] + 0 * x, q[2] + 0 * x, q[3] + 0 * x])
    s0 = o.get_state()
    o.step(5)
    assert np.abs(o.get_state() - s0).max() < 1e-13


def rankine_hugoniot(mach, rho1=1.0, p1=1.0, gamma=1.4):
    """post-shock state of a stationary normal shock with upstream Mach number `mach`"""
    c1 = (gamma * p1 / rho1) ** 0.5
    u1 = mach * c1
    r = (gamma + 1) * mach ** 2 / ((gamma - 1) * mach ** 2 + 2)
    p2 = p1 * (1 + 2 * gamma * (mach ** 2 - 1) / (gamma + 1))
    return (rho1, u1, p1), (rho1 * r, u1 / r, p2)


def test_stationary_shock_between_inflow_and_outflow(orc):
    """A Mach-2 normal shock between supersonic inflow and outflow stays
    where it is: the upstream state exactly, the Rankine-Hugoniot downstream
    state within the start-up waves, the shock within 1.5 cells of x = 0.5
    after 100 steps."""
    (r1, u1, p1), (r2, u2, p2) = rankine_hugoniot(2.0)
    nx = 40
    o = orc.Oracle(2, (nx, 2), lo=(0, 0), hi=(1, 2.0 / nx), tau_mode=1,
                   bc=[INFLOW, OUTFLOW, 0, 0], bc_state=[_cons(r1, u1, 0.0, p1)])
    o.init(lambda x, y: [np.where(x < 0.5, r1, r2), np.where(x < 0.5, u1, u2), 0 * x, np.where(x < 0.5, p1, p2)])
    o.step(100)
    rho = o.get_state()[0, 0, 0, :]
    xc = (np.arange(nx) + 0.5) / nx
    assert np.all(np.abs(rho[xc < 0.4] - r1) < 1e-6 * r1)
    # the start-up of a captured steady shock leaves waves of about 1% behind it
    assert np.all(np.abs(rho[xc > 0.6] - r2) < 2e-2 * r2)
    mid = 0.5 * (r1 + r2)
    i = int(np.argmax(rho > mid))
    xs = xc[i - 1] + (mid - rho[i - 1]) / (rho[i] - rho[i - 1]) / nx
    assert abs(xs - 0.5) < 1.5 / nx


def test_shock_vortex_field_satisfies_rankine_hugoniot():
    """The shock-vortex initial field: mass, momentum and energy fluxes agree
    across the shock (vortex strength 0), the upstream Mach number is the one
    asked for, and the vortex is isentropic."""
    import synth
    g = 1.4
    for mach in (1.1, 2.0, 3.0):
        x = np.array([0.49, 0.51])
        y = np.array([0.5, 0.5])
        r, u, v, p = synth.shock_vortex_2d(x, y, mach, eps=0.0)
        e = p / (g - 1) + 0.5 * r * u * u
        for a in (r * u, r * u * u + p, (e + p) * u):
            assert abs(a[0] - a[1]) <= 1e-13 * abs(a[0])
        assert r[1] > r[0] and p[1] > p[0]
        assert abs(u[0] / math.sqrt(g * p[0] / r[0]) - mach) < 1e-12
        xv = 0.25 + 0.03 * np.cos(np.linspace(0, 6, 7))
        yv = 0.5 + 0.03 * np.sin(np.linspace(0, 6, 7))
        rv, uv, vv, pv = synth.shock_vortex_2d(xv, yv, mach, eps=5.0)
        assert np.allclose(pv / rv ** g, 1.0, rtol=0, atol=1e-13)
        assert np.all(rv < 1.0)


@pytest.mark.parametrize("eps", [1.0, 5.0])
def test_shock_vortex_vortex_is_steady(eps):
    """The scaled vortex is a steady Euler solution: in its own frame the
    velocity is azimuthal and the pressure balances the centripetal term,
    dp/dr = rho v_theta^2 / r (central differences, step 1e-5 rc)."""
    import synth
    mach, rc, (xc, yc) = 2.0, 0.05, (0.25, 0.5)
    u1 = synth.shock_vortex_upstream(mach)[1]
    th = np.linspace(0.1, 6.0, 9)
    for rr in (0.3, 1.0, 2.0):
        x, y = xc + rr * rc * np.cos(th), yc + rr * rc * np.sin(th)
        rho, u, v, p = synth.shock_vortex_2d(x, y, mach, eps, rc=rc)
        ur = (u - u1) * np.cos(th) + v * np.sin(th)
        vt = -(u - u1) * np.sin(th) + v * np.cos(th)
        assert np.abs(ur).max() < 1e-14
        d = 1e-5 * rc
        pp = synth.shock_vortex_2d(x + d * np.cos(th), y + d * np.sin(th), mach, eps, rc=rc)[3]
        pm = synth.shock_vortex_2d(x - d * np.cos(th), y - d * np.sin(th), mach, eps, rc=rc)[3]
        dpdr = (pp - pm) / (2 * d)
        assert np.allclose(dpdr, rho * vt * vt / (rr * rc), rtol=1e-7, atol=0)


def test_shock_vortex_oracle_keeps_shock_and_upstream(orc):
    """Mach-1.5 shock-vortex on a coarse 48 x 24 mesh of [0, 2] x [0, 1]
    (inflow, outflow, slip walls): upstream of the vortex the inflow state is
    kept, and far from the vortex (y < 0.15) the shock stays within two
    cells of x = 0.5."""
    import synth
    mach = 1.5
    nx, ny = 48, 24
    o = orc.Oracle(2, (nx, ny), lo=(0, 0), hi=(2, 1), tau_mode=1, bc=[INFLOW, OUTFLOW, 2, 2],
                   bc_state=[synth.shock_vortex_inflow(mach)])
    o.init(lambda x, y: synth.shock_vortex_2d(x, y, mach, 3.0))
    o.step(30)
    rho = o.get_state()[0, 0]
    assert np.all(np.isfinite(rho))
    assert np.abs(rho[:, 0] - 1.0).max() < 2e-2
    xc = (np.arange(nx) + 0.5) * 2 / nx
    for j in range(3):
        row = rho[j]
        i = int(np.argmax(np.abs(np.diff(row))))
        assert abs(0.5 * (xc[i] + xc[i + 1]) - 0.5) <= 2 * 2 / nx
