"""Pins of the oracle's reconstruction (not GPU).

P1: the constrained least squares of Eq. (compact-big-5)/(compact-big-ref)
reproduces every polynomial of degree <= 4 exactly (values and gradients at all
face Gauss points).  P2: the linear sub-stencil polynomials of
Eq. (compact-sub-2) reproduce linear data.  P14: GENO path function sanity.
"""
import math

import numpy as np
import pytest

import refgeom as rg


@pytest.mark.parametrize("dim", [2, 3])
def test_quartic_exactness(orc, dim):
    rng = np.random.default_rng(1234 + dim)
    gps = rg.all_gps(dim)
    for trial in range(3):
        f, grad = rg.random_poly(dim, 4, rng)
        d = rg.data_vector(dim, f, grad)
        out, chi = orc.recon_reference(dim, d, linear=True)
        for gi, x in enumerate(gps):
            assert abs(out[gi, 0] - f(x)) <= 1e-12 * (1 + abs(f(x)))
            g = grad(x)
            for k in range(dim):
                assert abs(out[gi, 1 + k] - g[k]) <= 1e-11 * (1 + np.abs(g).max())


@pytest.mark.parametrize("dim", [2, 3])
def test_quintic_not_reproduced(orc, dim):
    # guard against a trivially passing P1: degree-5 data must leave a residual
    rng = np.random.default_rng(7)
    f, grad = rg.random_poly(dim, 5, rng)
    d = rg.data_vector(dim, f, grad)
    out, _ = orc.recon_reference(dim, d, linear=True)
    err = max(abs(out[gi, 0] - f(x)) for gi, x in enumerate(rg.all_gps(dim)))
    assert err > 1e-6


@pytest.mark.parametrize("dim", [2, 3])
def test_matrix_shape_and_constraints(orc, dim):
    M, ex = orc.recon_matrix(dim)
    nb = 34 if dim == 3 else 14
    nd = 73 if dim == 3 else 25
    assert M.shape == (nb, nd)
    assert all(1 <= e.sum() <= 4 for e in ex)
    # the face-neighbour averages hold exactly for arbitrary (non-polynomial) data
    rng = np.random.default_rng(3)
    d = rng.standard_normal(nd)
    a = orc.recon_coeffs(dim, d)
    exps = ex[:, :dim]

    def P(x):
        from math import factorial
        v = d[0]
        for c, e in zip(a, exps):
            mono = lambda y: np.prod([y[i] ** e[i] / factorial(e[i]) for i in range(dim)])
            v += c * (mono(x) - rg.cell_avg(mono, [0] * dim, dim))
        return v

    for m, o in enumerate(rg.face_offsets(dim)):
        assert abs(rg.cell_avg(P, o, dim) - d[1 + m]) < 1e-11
    assert abs(rg.cell_avg(P, [0] * dim, dim) - d[0]) < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_linear_substencils_exact(orc, dim):
    rng = np.random.default_rng(11)
    f, grad = rg.random_poly(dim, 1, rng)
    d = rg.data_vector(dim, f, grad)
    g = grad(np.zeros(dim))
    for m in range(2 * dim):
        b = orc.linear_sub(dim, m, d)
        assert np.allclose(b, g, atol=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_linear_substencil_uses_only_its_data(orc, dim):
    # P_m^1 depends on Q0, Q_{1,m} and the lines not parallel to axis m only
    nd = 73 if dim == 3 else 25
    gpf = rg.gpf(dim)
    nfo = 2 * dim
    ne = 12 if dim == 3 else 4
    line0 = 1 + nfo + ne + nfo * dim + ne * (2 if dim == 3 else 1)
    for m in range(2 * dim):
        allowed = {0, 1 + m}
        for ax in range(dim):
            if ax != m // 2:
                allowed |= {line0 + ax * gpf + k for k in range(gpf)}
        for j in range(nd):
            e = np.zeros(nd)
            e[j] = 1.0
            b = orc.linear_sub(dim, m, e)
            if j not in allowed:
                assert np.all(b == 0.0), (m, j)


@pytest.mark.parametrize("dim", [2, 3])
def test_geno_linear_data_gives_chi_one(orc, dim):
    rng = np.random.default_rng(5)
    f, grad = rg.random_poly(dim, 1, rng)
    d = rg.data_vector(dim, f, grad)
    out, chi = orc.recon_reference(dim, d, linear=False)
    assert chi == 1.0
    out_lin, _ = orc.recon_reference(dim, d, linear=True)
    assert np.array_equal(out, out_lin)


@pytest.mark.parametrize("dim", [2, 3])
def test_geno_constant_data(orc, dim):
    nd = 73 if dim == 3 else 25
    gpf = rg.gpf(dim)
    d = np.zeros(nd)
    d[0] = 2.5
    d[1:1 + 2 * dim + (12 if dim == 3 else 4)] = 2.5
    out, chi = orc.recon_reference(dim, d, linear=False)
    assert chi == 1.0
    assert np.allclose(out[:, 0], 2.5, rtol=0, atol=1e-14) and np.abs(out[:, 1:]).max() < 1e-14


@pytest.mark.parametrize("dim", [2, 3])
def test_geno_step_function_is_troubled(orc, dim):
    # a unit jump between the target cell and its +x neighbours: chi small
    def f(x):
        return 1.0 if x[0] > 0.5 else 0.0

    def grad(x):
        return np.zeros(dim)

    d = rg.data_vector(dim, f, grad)
    _, chi = orc.recon_reference(dim, d, linear=False)
    assert chi < 0.1


@pytest.mark.parametrize("dim", [2, 3])
def test_geno_low_order_weights(orc, dim):
    """chi = 0 leaves the weighted linear sub-stencil polynomials of
    Eq. (weno-new): sum_m w_m P_m^1 with w_m proportional to
    d_m / (IS_m + eps)^5, d_m = 1 / (2 dim), IS_m = |grad P_m^1|^2 on the unit
    cell (reading C5).  Data: a linear field whose face-neighbour averages are
    moved so that each sub-stencil sees its own slope along its axis
    (P_m^1 matches Q_{1,m} exactly and fits the perpendicular lines, which
    stay those of the linear field), so every P_m^1 is known in closed form."""
    g = np.array([0.3, -0.2, 0.1])[:dim]
    q0 = 0.7
    f = lambda x: q0 + float(np.dot(g, x))
    d = rg.data_vector(dim, f, lambda x: g)
    beta = [0.45, 0.8, -0.3, 0.35, 0.6, -0.25][:2 * dim]  # slope of P_m^1 along its axis
    slopes = []
    for m, o in enumerate(rg.face_offsets(dim)):
        a, s = m // 2, o[m // 2]
        d[1 + m] = q0 + s * beta[m]
        b = g.copy()
        b[a] = beta[m]
        slopes.append(b)
        assert np.allclose(orc.linear_sub(dim, m, d), b, atol=1e-14)
    w = np.array([(1.0 / (2 * dim)) / (float(b @ b) + 1e-15) ** 5 for b in slopes])
    w /= w.sum()
    assert w.max() < 0.9 and np.sort(w)[-2] > 1e-3  # several sub-stencils matter
    out, chi = orc.recon_reference(dim, d, low_order=True)
    assert chi == 0.0
    for gi, x in enumerate(rg.all_gps(dim)):
        val = sum(w[m] * (q0 + slopes[m] @ x) for m in range(2 * dim))
        grad = sum(w[m] * slopes[m] for m in range(2 * dim))
        assert abs(out[gi, 0] - val) <= 1e-14
        assert np.abs(out[gi, 1:] - grad).max() <= 1e-14


@pytest.mark.parametrize("dim", [2, 3])
def test_geno_chi_from_integrated_indicators(orc, dim):
    """chi of the GENO path function (reading C5) on quartic data, with the
    indicators integrated here from the polynomial itself: IS^H = sum over
    multi-indices 1 <= |l| <= 4 (each once) of the integral over the unit cell
    of (D^l P)^2, IS^L its |l| = 1 part, IS^tau = IS^H - IS^L, then
    alpha = 2 a_H / (a_H + a_L) with a = 1 + (IS^tau / (IS + eps))^2 and
    chi = tanh(C alpha) / tanh(C).  The reconstruction reproduces quartics
    (P1), so P is the data's polynomial; a wrong Gram entry, a missing order
    or a cross term counted twice changes chi."""
    import itertools
    import sympy as sp
    X = sp.symbols("x0:%d" % dim)
    t = sp.Symbol("t")
    rng = np.random.default_rng(77 + dim)
    c_chi = 0.3
    exps = [e for e in itertools.product(range(5), repeat=dim) if 1 <= sum(e) <= 4]
    coef = rng.standard_normal(len(exps))
    # P = linear part + t (orders 2-4): the indicators are quadratics in t
    P = sum(sp.Float(c, 30) * (1 if sum(e) == 1 else t) * sp.prod([X[a] ** e[a] for a in range(dim)])
            for c, e in zip(coef, exps))
    dom = [(X[a], -sp.Rational(1, 2), sp.Rational(1, 2)) for a in range(dim)]
    ish = isl = sp.Integer(0)
    for l in itertools.product(range(5), repeat=dim):
        if not 1 <= sum(l) <= 4:
            continue
        D = P
        for a in range(dim):
            D = sp.diff(D, X[a], l[a])
        v = sp.integrate(sp.expand(D * D), *dom)
        ish += v
        if sum(l) == 1:
            isl += v
    ishf, islf = sp.lambdify(t, ish), sp.lambdify(t, isl)
    for target in (0.5, 1.0, 2.0):  # IS^tau / IS^L, set by t (bisection)
        lo_t, hi_t = 0.0, 10.0
        for _ in range(80):
            tm = 0.5 * (lo_t + hi_t)
            if (ishf(tm) - islf(tm)) / islf(tm) < target:
                lo_t = tm
            else:
                hi_t = tm
        tv = 0.5 * (lo_t + hi_t)
        Pt = P.subs(t, tv)
        fn = sp.lambdify(X, Pt, "math")
        gr = [sp.lambdify(X, sp.diff(Pt, X[a]), "math") for a in range(dim)]
        d = rg.data_vector(dim, lambda x: fn(*x), lambda x: np.array([gk(*x) for gk in gr]))
        _, chi = orc.recon_reference(dim, d, c_chi=c_chi)
        eps = 1e-15
        vh, vl = float(ishf(tv)), float(islf(tv))
        ist = max(vh - vl, 0.0)
        ah = 1 + (ist / (vh + eps)) ** 2
        al = 1 + (ist / (vl + eps)) ** 2
        expect = math.tanh(c_chi * 2 * ah / (ah + al)) / math.tanh(c_chi)
        assert 0.05 < expect < 0.95  # chi away from its bounds, where a wrong indicator shows
        assert abs(chi - expect) <= 1e-11, (target, chi, expect)
