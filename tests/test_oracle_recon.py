"""Pins of the oracle's reconstruction (not GPU).

P1: the constrained least squares of Eq. (compact-big-5)/(compact-big-ref)
reproduces every polynomial of degree <= 4 exactly (values and gradients at all
face Gauss points).  P2: the linear sub-stencil polynomials of
Eq. (compact-sub-2) reproduce linear data.  P14: GENO path function sanity.
"""
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
