"""GPU parity of the CUDA path (through the C-ABI) against the CPU oracle.

Bar: max relative difference 1e-12 after one S2O4 step and 1e-9 after 100
steps, relative to the variable-class scale of parity.class_scaled_diff
(derivative fields relative to max(their size, |average|/h), the precision of
a difference quotient).  Inputs are the oracle's initial states of seeded
analytic fields, so no oracle input comes from the CUDA path.
"""
import math

import numpy as np
import pytest

import synth
from parity import class_scaled_diff

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_08965_gb300 as p
    p.lib()
    return p


def vortex(x, y):
    return synth.isentropic_vortex_2d(x, y)


def tgv(x, y, z):
    return synth.taylor_green_3d(x, y, z)


def hmin(n, lo, hi, nodes):
    h = min((hi[a] - lo[a]) / n[a] for a in range(len(n)))
    return 0.7 * h if nodes is not None else h


def pair(orc, cg, dim, n, lo, hi, fn, nodes=None, **kw):
    o = orc.Oracle(dim, n, lo=lo, hi=hi, nodes=nodes, **kw)
    o.init(fn)
    s0 = o.get_state()
    m = cg.Mesh(dim, n, lo=lo, hi=hi, nodes=nodes, **kw)
    m.set_state(s0)
    return o, m


CASES = [
    ("vortex64", 2, (64, 64), (0, 0), (10, 10), vortex, None, {}),
    ("vortex-ragged", 2, (37, 29), (0, 0), (10, 10), vortex, None, {"tau_mode": 1}),
    ("tgv12", 3, (12, 12, 12), (0, 0, 0), (2 * math.pi,) * 3, tgv, None,
     {"mu": 1 / 1600, "prandtl": 0.72, "tau_mode": 2}),
    ("tgv-ragged", 3, (7, 9, 11), (0, 0, 0), (2 * math.pi,) * 3, tgv, None,
     {"mu": 1 / 1600, "prandtl": 0.72, "tau_mode": 2}),
    ("tgv-curvilinear", 3, (10, 10, 10), (0, 0, 0), (2 * math.pi,) * 3, tgv, "perturbed",
     {"mu": 1 / 1600, "prandtl": 0.72, "tau_mode": 2}),
    ("sine-linear", 3, (10, 10, 10), (0, 0, 0), (2, 2, 2),
     lambda x, y, z: synth.density_sine_3d(x, y, z), None, {"linear": True}),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_one_step(orc, cg, case):
    name, dim, n, lo, hi, fn, nodes, kw = case
    if nodes == "perturbed":
        nodes = synth.perturbed_nodes_3d(n)
    o, m = pair(orc, cg, dim, n, lo, hi, fn, nodes=nodes, **kw)
    dt_o = o.dt()
    dt_g = m.compute_dt()
    assert abs(dt_g - dt_o) <= 1e-14 * dt_o
    o.step(1)
    m.step(1)
    sg, tg = m.get_state()
    assert abs(tg - o.time()) <= 1e-14 * o.time()
    d = class_scaled_diff(sg, o.get_state(), hmin(n, lo, hi, nodes))
    # the plain norm (derivative fields by their own size) is reported beside
    # the bar's: its rounding floor is measured in tests/test_parity_norm.py
    print("%s one step: class-scaled %.2e, plain %.2e" % (name, d, class_scaled_diff(sg, o.get_state())))
    assert d <= 1e-12
    m.close()


@pytest.mark.parametrize("case", [CASES[0], CASES[2], CASES[4]], ids=["vortex64", "tgv12", "tgv-curvilinear"])
def test_many_steps(orc, cg, case):
    name, dim, n, lo, hi, fn, nodes, kw = case
    if nodes == "perturbed":
        nodes = synth.perturbed_nodes_3d(n)
    steps = 100
    o, m = pair(orc, cg, dim, n, lo, hi, fn, nodes=nodes, **kw)
    o.step(steps)
    m.step(steps)
    sg, _ = m.get_state()
    d = class_scaled_diff(sg, o.get_state(), hmin(n, lo, hi, nodes))
    print("%s 100 steps: class-scaled %.2e, plain %.2e" % (name, d, class_scaled_diff(sg, o.get_state())))
    assert d <= 1e-9
    m.close()


def test_config1_vortex_10_steps(orc, cg):
    """2-D isentropic vortex, 64^2 over [0,10]^2, eps = 5, CFL 0.5, 10 steps."""
    o, m = pair(orc, cg, 2, (64, 64), (0, 0), (10, 10), vortex)
    s0 = o.get_state()
    o.step(10)
    m.step(10)
    sg, _ = m.get_state()
    so = o.get_state()
    assert class_scaled_diff(sg, so) <= 1e-11
    # conservation of the domain sums on the GPU
    assert np.all(np.abs(sg[0].sum(axis=(1, 2)) - s0[0].sum(axis=(1, 2))) <= 1e-13 * np.abs(s0[0]).sum())
    m.close()


def test_sod_strip_nonlinear(orc, cg):
    """Shock problem with tau mode 1 and the GENO blend active (chi < 1)."""
    L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)

    def init(x, y):
        xp = np
        try:
            import torch
            if isinstance(x, torch.Tensor):
                xp = torch
        except ImportError:
            pass
        inside = (x >= -0.5) & (x < 0.5)
        return [xp.where(inside, L[0] + 0 * x, R[0] + 0 * x), 0 * x, 0 * x, xp.where(inside, L[2] + 0 * x, R[2] + 0 * x)]

    n = (120, 4)
    o, m = pair(orc, cg, 2, n, (-1.5, 0), (1.5, 0.1), init, tau_mode=1)
    for _ in range(3):
        o.step(5)
        m.step(5)
        sg, _ = m.get_state()
        assert class_scaled_diff(sg, o.get_state()) <= 1e-10
    # chi of one more step.  Where the stencil holds only rounding noise (the
    # undisturbed states) the smoothness indicators are noise and chi is not
    # determined; compare chi where the density varies by more than 1e-6
    rho = o.get_state()[0, 0]
    var = np.zeros_like(rho)
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            var = np.maximum(var, np.abs(np.roll(np.roll(rho, dj, 0), di, 1) - rho))
    o.step(1)
    m.step(1)
    mask = var > 1e-6
    co, cgp = o.chi(), m.chi()
    assert (co[:, mask] < 0.5).any()
    assert np.abs(co[:, mask] - cgp[:, mask]).max() <= 1e-9
    m.close()


def test_free_stream_curvilinear_100_steps(cg):
    n = (16, 16, 16)
    nodes = synth.perturbed_nodes_3d(n)
    prim = (1.0, 0.3, 0.2, 0.1, 1.0 / 1.4)
    m = cg.Mesh(3, n, nodes=nodes, tau_mode=1)
    m.init(lambda x, y, z: synth.uniform_state(prim, x, y, z))
    s0, _ = m.get_state()
    m.step(100)
    s1, _ = m.get_state()
    assert np.abs(s1[0] - s0[0]).max() <= 1e-12
    assert np.abs(s1[1:]).max() <= 1e-11
    m.close()


def test_library_init_matches_oracle_init(orc, cg):
    for dim, n, lo, hi, fn, nodes in [
        (2, (20, 16), (0, 0), (10, 10), vortex, None),
        (3, (8, 8, 8), (0, 0, 0), (2 * math.pi,) * 3, tgv, synth.perturbed_nodes_3d((8, 8, 8))),
    ]:
        o = orc.Oracle(dim, n, lo=lo, hi=hi, nodes=nodes)
        o.init(fn)
        m = cg.Mesh(dim, n, lo=lo, hi=hi, nodes=nodes)
        m.init(fn)
        sg, _ = m.get_state()
        assert class_scaled_diff(sg, o.get_state()) <= 1e-12
        m.close()


def _random_state(dim, n, seed, mach_max):
    """Averages of random states spanning Mach 1e-3..mach_max (derivative
    fields zero): the time step must not depend on how the maximum is found."""
    rng = np.random.default_rng(seed)
    shape = tuple(reversed(n))
    rho = 10 ** rng.uniform(-2, 1, shape)
    c = 10 ** rng.uniform(-1, 1, shape)
    p = rho * c * c / 1.4
    u = rng.normal(size=(dim,) + shape)
    u *= (10 ** rng.uniform(-3, np.log10(mach_max), shape) * c / np.linalg.norm(u, axis=0))
    nf = 1 + dim + dim * (4 if dim == 3 else 2)
    s = np.zeros((nf, dim + 2) + shape)
    s[0, 0] = rho
    s[0, 1:1 + dim] = rho * u
    s[0, dim + 1] = p / 0.4 + 0.5 * rho * (u * u).sum(0)
    return s


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("dim,n,curvi,mu", [(2, (64, 48), False, 0.0), (3, (10, 11, 12), True, 1e-3),
                                             (3, (16, 16, 16), False, 1e-3)])
def test_time_step_equals_fp64_maximum(orc, cg, precision, dim, n, curvi, mu):
    lo, hi = (0,) * dim, ((2 * math.pi,) * 3 if curvi else (1,) * dim)
    nodes = synth.perturbed_nodes_3d(n) if curvi else None
    for seed, mach in ((1, 0.5), (2, 300.0)):
        s = _random_state(dim, n, seed, mach)
        o = orc.Oracle(dim, n, lo=lo, hi=hi, nodes=nodes, mu=mu)
        o.set_state(s)
        m = cg.Mesh(dim, n, lo=lo, hi=hi, nodes=nodes, mu=mu, precision=precision)
        m.set_state(s)
        dg, do = m.compute_dt(), o.dt()
        assert abs(dg - do) <= 1e-14 * do, (seed, dg, do)
        m.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_diagnostics_match_oracle(orc, cg, precision):
    """Kinetic energy and enstrophy averages of a TGV state after a few steps
    (curvilinear and Cartesian) against the oracle's sums of the same
    state."""
    from oracle.diagnostics import tgv_diagnostics
    for nodes in (None, "perturbed"):
        n = (12, 12, 12)
        nd = synth.perturbed_nodes_3d(n) if nodes else None
        kw = dict(lo=(0, 0, 0), hi=(2 * math.pi,) * 3, nodes=nd, mu=1 / 1600, prandtl=0.72, tau_mode=2)
        o = orc.Oracle(3, n, **kw)
        o.init(tgv)
        o.step(3)
        s = o.get_state()
        vol, _ = o.metrics()
        ek, es = tgv_diagnostics(s, 3, vol, 1 / 1600)
        m = cg.Mesh(3, n, precision=precision, **kw)
        m.set_state(s)
        gk, gs = m.diagnostics()
        tol = 1e-12 if precision == 0 else 1e-6
        assert abs(gk - ek) <= tol * ek and abs(gs - es) <= tol * es
        m.close()
