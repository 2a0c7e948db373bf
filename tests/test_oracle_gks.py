"""Pins of the oracle's gas-kinetic interface solution (Sec. 2), not GPU.

P4: Maxwellian moments against brute-force quadrature.
P5: a uniform state gives the Euler flux and no time change, for every tau mode.
P6: tau = 0 with identical smooth sides gives F(W) and F_t = A_x(W) Q_t with
    Q_t = -sum_j A_j dW/dx_j (Euler Jacobians by complex step); this also pins
    the compatibility condition that defines A.
Micro-slopes: <a psi psi^T> = b checked with an independently built matrix.
Navier-Stokes limits (tau = mu/p): shear stress mu dV/dx and heat flux
    -mu c_p/Pr dT/dx.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats


def euler_flux(W, dim, gamma):
    rho = W[0]
    u = [W[1 + i] / rho for i in range(dim)]
    E = W[dim + 1]
    p = (gamma - 1.0) * (E - 0.5 * rho * sum(x * x for x in u))
    F = [rho * u[0]]
    for i in range(dim):
        F.append(rho * u[0] * u[i] + (p if i == 0 else 0.0))
    F.append(u[0] * (E + p))
    return np.array(F)


def euler_flux_dir(W, dim, gamma, j):
    """flux along local axis j: permute the momentum components."""
    perm = list(range(dim))
    perm[0], perm[j] = perm[j], perm[0]
    Wp = W.copy()
    for i in range(dim):
        Wp[1 + i] = W[1 + perm[i]]
    Fp = euler_flux(Wp, dim, gamma)
    F = Fp.copy()
    for i in range(dim):
        F[1 + perm[i]] = Fp[1 + i]
    return F


def jac(fn, W):
    n = len(W)
    J = np.zeros((n, n))
    for k in range(n):
        Wc = W.astype(complex)
        Wc[k] += 1e-30j
        J[:, k] = np.imag(fn(Wc)) / 1e-30
    return J


def cons(dim, rho, u, p, gamma=1.4):
    return np.array([rho] + [rho * x for x in u] + [p / (gamma - 1) + 0.5 * rho * sum(x * x for x in u)])


@pytest.mark.parametrize("U,lam", [(0.3, 0.7), (-1.2, 2.5), (2.0, 0.35), (0.0, 1.0)])
def test_moments_against_quadrature(orc, U, lam):
    full, pos, neg = orc.moments_u(U, lam)
    xh, wh = np.polynomial.hermite.hermgauss(200)
    g = lambda u: math.sqrt(lam / math.pi) * math.exp(-lam * (u - U) ** 2)
    for n in range(7):
        q = np.sum(wh * (U + xh / math.sqrt(lam)) ** n) / math.sqrt(math.pi)
        assert abs(full[n] - q) <= 1e-13 * max(1.0, abs(q))
        qp = integrate.quad(lambda u: u ** n * g(u), 0, np.inf, epsabs=1e-15, epsrel=1e-14)[0]
        qn = integrate.quad(lambda u: u ** n * g(u), -np.inf, 0, epsabs=1e-15, epsrel=1e-14)[0]
        assert abs(pos[n] - qp) <= 1e-13 * max(1.0, abs(qp))
        assert abs(neg[n] - qn) <= 1e-13 * max(1.0, abs(qn))


def _moment_matrix(dim, rho_u_lam, gamma):
    """<psi_i psi_j> by tensor Gauss-Hermite quadrature in velocity and
    chi-square moments for the internal energy (independent of the oracle)."""
    U = rho_u_lam[1:1 + dim]
    lam = rho_u_lam[dim + 1]
    K = (5 - 3 * gamma) / (gamma - 1) if dim == 3 else (4 - 2 * gamma) / (gamma - 1)
    xh, wh = np.polynomial.hermite.hermgauss(20)
    s = 1.0 / (2 * lam)
    xi2 = K * s
    xi4 = stats.chi2(K).moment(2) * s * s
    nv = dim + 2
    M = np.zeros((nv, nv))
    import itertools
    for idx in itertools.product(range(len(xh)), repeat=dim):
        w = np.prod([wh[i] for i in idx]) / math.pi ** (dim / 2)
        c = [U[a] + xh[idx[a]] / math.sqrt(lam) for a in range(dim)]
        c2 = sum(x * x for x in c)
        # psi = (1, c, 1/2 (c^2 + xi^2)); average over xi analytically
        base = [1.0] + c
        for i in range(nv):
            for j in range(nv):
                if i < nv - 1 and j < nv - 1:
                    M[i, j] += w * base[i] * base[j]
                elif i == nv - 1 and j == nv - 1:
                    M[i, j] += w * 0.25 * (c2 * c2 + 2 * c2 * xi2 + xi4)
                else:
                    k = i if i < nv - 1 else j
                    M[i, j] += w * base[k] * 0.5 * (c2 + xi2)
    return M


@pytest.mark.parametrize("dim", [2, 3])
def test_micro_slope_solves_moment_system(orc, dim):
    rng = np.random.default_rng(dim)
    for _ in range(3):
        prim = np.concatenate([[1.3], rng.uniform(-1, 1, dim), [rng.uniform(0.3, 2.0)]])
        b = rng.standard_normal(dim + 2)
        a = orc.micro_slope(dim, prim, b)
        M = _moment_matrix(dim, prim, 1.4)
        assert np.allclose(M @ a, b, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_uniform_state_is_euler_flux(orc, dim, mode):
    W = cons(dim, 1.3, [0.7, -0.4, 0.25][:dim], 0.9)
    z = np.zeros((dim, dim + 2))
    out = orc.gks_point(dim, W, z, W, z, 0.01, mu=1e-3 if mode == 2 else 0.0,
                        prandtl=0.72, tau_mode=mode)
    F = euler_flux(W, dim, 1.4)
    assert np.allclose(out[0], F, rtol=1e-13, atol=1e-14)
    assert np.abs(out[1]).max() < 1e-11
    for k in (2, 4):
        assert np.allclose(out[k], W, rtol=1e-14, atol=1e-14)
    for k in (3, 5):
        assert np.abs(out[k]).max() < 1e-11


@pytest.mark.parametrize("dim", [2, 3])
def test_tau0_smooth_gives_euler_and_jacobian_time_derivative(orc, dim):
    rng = np.random.default_rng(40 + dim)
    for _ in range(3):
        W = cons(dim, rng.uniform(0.5, 2), rng.uniform(-1, 1, dim), rng.uniform(0.5, 2))
        dW = rng.standard_normal((dim, dim + 2)) * 0.3
        out = orc.gks_point(dim, W, dW, W, dW, 0.01, tau_mode=0)
        F = euler_flux(W, dim, 1.4)
        Qt = np.zeros(dim + 2)
        for j in range(dim):
            Aj = jac(lambda w, j=j: euler_flux_dir(w, dim, 1.4, j), W)
            Qt -= Aj @ dW[j]
        Ax = jac(lambda w: euler_flux(w, dim, 1.4), W)
        Ft = Ax @ Qt
        assert np.allclose(out[0], F, rtol=1e-13, atol=1e-13)
        assert np.allclose(out[1], Ft, rtol=1e-11, atol=1e-11)
        assert np.allclose(out[2], W, rtol=1e-14) and np.allclose(out[4], W, rtol=1e-14)
        assert np.allclose(out[3], Qt, rtol=1e-11, atol=1e-11)
        assert np.allclose(out[5], Qt, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("dim", [2, 3])
def test_navier_stokes_shear_stress(orc, dim):
    mu, s, gamma = 2e-3, 0.8, 1.4
    W = cons(dim, 1.1, [0.0] * dim, 0.9)
    dW = np.zeros((dim, dim + 2))
    dW[0, 2] = W[0] * s  # d(rho V)/dx with V = 0 at the point
    out = orc.gks_point(dim, W, dW, W, dW, 1e-3, mu=mu, prandtl=1.0, tau_mode=2)
    assert abs(out[0][2] - (-mu * s)) < 1e-12
    assert abs(out[0][0]) < 1e-14


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("pr", [1.0, 0.72])
def test_navier_stokes_heat_flux_with_prandtl_fix(orc, dim, pr):
    mu, gamma = 2e-3, 1.4
    rho, p = 1.1, 0.9
    drho, dp = 0.3, -0.2
    W = cons(dim, rho, [0.0] * dim, p)
    dW = np.zeros((dim, dim + 2))
    dW[0, 0] = drho
    dW[0, dim + 1] = dp / (gamma - 1)
    out = orc.gks_point(dim, W, dW, W, dW, 1e-3, mu=mu, prandtl=pr, tau_mode=2)
    dT = dp / rho - p * drho / rho ** 2
    cp = gamma / (gamma - 1)
    q = -mu * cp / pr * dT
    assert abs(out[0][dim + 1] - q) < 1e-12 * max(1, abs(q)) + 1e-14


def test_s2o4_is_fourth_order_taylor(orc):
    # dQ/dt = lam Q: L = lam Q, dL/dt = lam^2 Q (temporal discretisation section)
    for lam, dt in [(-1.3, 0.1), (0.7, 0.05), (-5.0, 0.2)]:
        Q = 1.7
        qs = orc.s2o4(Q, dt, lam * Q, lam * lam * Q)
        _, qn = orc.s2o4(Q, dt, lam * Q, lam * lam * Q, lam * lam * qs)
        z = lam * dt
        assert abs(qn - Q * (1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24)) < 1e-14 * abs(Q)


# --- pins of the collision state (reading C3), the two-sided interface
# values (reading C4) and the heat-flux fix of F_t (reading C16) ---------------

def _prim(W, dim, gamma=1.4):
    rho = W[0]
    u = W[1:1 + dim] / rho
    p = (gamma - 1.0) * (W[dim + 1] - 0.5 * rho * np.dot(u, u))
    return rho, u, p


def _half_space_closed(W, dim, side, gamma=1.4):
    """Conservative moments of the half Maxwellian of W over u > 0 (side 0) or
    u < 0 (side 1): the normal-velocity integrals by erfc, the transverse
    velocity and internal energy full-space.  Works on complex W (complex
    step)."""
    from scipy.special import erfc
    rho = W[0]
    u = [W[1 + i] / rho for i in range(dim)]
    ke = sum(W[1 + i] * u[i] for i in range(dim))
    p = (gamma - 1.0) * (W[dim + 1] - 0.5 * ke)
    lam = rho / (2.0 * p)
    K = (5 - 3 * gamma) / (gamma - 1) if dim == 3 else (4 - 2 * gamma) / (gamma - 1)
    s = 1.0 if side == 0 else -1.0
    sl = np.sqrt(lam)
    m0 = 0.5 * erfc(-s * sl * u[0])
    e = np.exp(-lam * u[0] ** 2) / (2.0 * np.sqrt(np.pi * lam))
    m1 = u[0] * m0 + s * e
    m2 = u[0] * m1 + m0 / (2.0 * lam)
    ut2 = sum(u[i] ** 2 for i in range(1, dim))
    out = [rho * m0, rho * m1] + [rho * u[i] * m0 for i in range(1, dim)]
    out.append(0.5 * rho * (m2 + (ut2 + (dim - 1 + K) / (2.0 * lam)) * m0))
    return np.array(out)


def _half_space_quad(W, dim, side, gamma=1.4):
    """The same moments by adaptive quadrature over the half line of normal
    velocities (independent of the erfc recurrences)."""
    rho, u, p = _prim(W, dim, gamma)
    lam = rho / (2.0 * p)
    K = (5 - 3 * gamma) / (gamma - 1) if dim == 3 else (4 - 2 * gamma) / (gamma - 1)
    g = lambda x: math.sqrt(lam / math.pi) * math.exp(-lam * (x - u[0]) ** 2)
    lo, hi = (0.0, np.inf) if side == 0 else (-np.inf, 0.0)
    mn = [integrate.quad(lambda x, n=n: x ** n * g(x), lo, hi, epsabs=1e-15, epsrel=1e-14)[0] for n in range(3)]
    ut2 = float(np.dot(u[1:], u[1:]))
    out = [rho * mn[0], rho * mn[1]] + [rho * u[i] * mn[0] for i in range(1, dim)]
    out.append(0.5 * rho * (mn[2] + (ut2 + (dim - 1 + K) / (2.0 * lam)) * mn[0]))
    return np.array(out)


def _half_space_jvp(W, dW, dim, side):
    """d/de of the half-space moments of W + e dW (complex step): the moments
    of the half Maxwellian's spatial derivative g (a . psi)"""
    return np.imag(_half_space_closed(W.astype(complex) + 1e-30j * dW, dim, side)) / 1e-30


def _euler_dt(W, dW, dim, gamma=1.4):
    """Q_t = -sum_j (dF_j/dW) dW_j (Euler Jacobians by complex step)"""
    Qt = np.zeros(dim + 2)
    for j in range(dim):
        Aj = jac(lambda w, j=j: euler_flux_dir(w, dim, gamma, j), W)
        Qt -= Aj @ dW[j]
    return Qt


@pytest.mark.parametrize("dim", [2, 3])
def test_half_space_moments_closed_form_vs_quadrature(dim):
    # the test's own closed form (used below) against quadrature
    for W in (cons(dim, 1.2, [0.4, -0.3, 0.2][:dim], 0.8), cons(dim, 0.3, [-1.1, 0.5, 0.0][:dim], 0.2)):
        for side in (0, 1):
            a, b = _half_space_closed(W, dim, side), _half_space_quad(W, dim, side)
            assert np.allclose(a, b, rtol=1e-12, atol=1e-14)


STATES = [  # (rho, u, p) left | right, pressure jumps giving blend weights far from 1/2
    ((1.0, [0.2, 0.1, -0.3], 1.0), (0.4, [-0.1, 0.3, 0.2], 0.1)),
    ((0.9, [0.5, -0.2, 0.1], 0.8), (1.1, [0.3, 0.0, -0.1], 1.0)),
    ((0.2, [-0.6, 0.4, 0.3], 0.15), (1.3, [-0.2, -0.1, 0.5], 1.4)),
]


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("k", range(len(STATES)))
def test_collision_state_and_euler_limit_with_unequal_sides(orc, dim, k):
    """tau = 0 (smooth-flow mode) with different left and right states and
    slopes: the interface distribution is g0 (1 + A t) only, so F^n is the
    Euler flux of the collision state W0 = int psi (g_l H(u) + g_r (1 - H(u)))
    and F_t^n = A_x(W0) (dQ/dt)_0, with (dQ/dt)_0 = -sum_j A_j(W0) dW0_j and
    dW0_j the same half-space combination of the two sides' slopes (C3)."""
    (rl, ul, pl), (rr, ur, pr) = STATES[k]
    WL, WR = cons(dim, rl, ul[:dim], pl), cons(dim, rr, ur[:dim], pr)
    rng = np.random.default_rng(100 + 10 * dim + k)
    dWL = rng.standard_normal((dim, dim + 2)) * 0.2
    dWR = rng.standard_normal((dim, dim + 2)) * 0.2
    out = orc.gks_point(dim, WL, dWL, WR, dWR, 0.01, tau_mode=0)
    W0 = _half_space_quad(WL, dim, 0) + _half_space_quad(WR, dim, 1)
    dW0 = np.array([_half_space_jvp(WL, dWL[j], dim, 0) + _half_space_jvp(WR, dWR[j], dim, 1) for j in range(dim)])
    Qt0 = _euler_dt(W0, dW0, dim)
    Ax = jac(lambda w: euler_flux(w, dim, 1.4), W0)
    sc = np.abs(euler_flux(W0, dim, 1.4)).max()
    assert np.abs(out[0] - euler_flux(W0, dim, 1.4)).max() <= 1e-12 * sc
    assert np.abs(out[1] - Ax @ Qt0).max() <= 1e-11 * max(1.0, np.abs(Ax @ Qt0).max())


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("k", range(len(STATES)))
def test_two_sided_interface_values(orc, dim, mode, k):
    """The interface values of the derivative update (C4): with
    tau0 = 5 |pl - pr| / (pl + pr) dt and w = exp(-dt / tau0), each side gets
    (1 - w) Q^e + w Q_0^side, where Q^e = W0 + t (dQ/dt)_0 is the collision
    state's and Q_0^side = W_side + t (dQ/dt)_side the side's own Euler
    evolution; the weight does not depend on the flux's tau mode."""
    (rl, ul, pl), (rr, ur, pr) = STATES[k]
    WL, WR = cons(dim, rl, ul[:dim], pl), cons(dim, rr, ur[:dim], pr)
    rng = np.random.default_rng(200 + 10 * dim + k)
    dWL = rng.standard_normal((dim, dim + 2)) * 0.2
    dWR = rng.standard_normal((dim, dim + 2)) * 0.2
    dt = 0.01
    out = orc.gks_point(dim, WL, dWL, WR, dWR, dt, mu=1e-3 if mode == 2 else 0.0, prandtl=0.72, tau_mode=mode)
    W0 = _half_space_quad(WL, dim, 0) + _half_space_quad(WR, dim, 1)
    dW0 = np.array([_half_space_jvp(WL, dWL[j], dim, 0) + _half_space_jvp(WR, dWR[j], dim, 1) for j in range(dim)])
    Qt0 = _euler_dt(W0, dW0, dim)
    w = math.exp(-(pl + pr) / (5.0 * abs(pl - pr)))
    assert 0.05 < w < 0.95 and abs(w - 0.5) > 0.1
    for part, W, dW in ((2, WL, dWL), (4, WR, dWR)):
        exp0 = (1 - w) * W0 + w * W
        expt = (1 - w) * Qt0 + w * _euler_dt(W, dW, dim)
        assert np.abs(out[part] - exp0).max() <= 1e-12 * np.abs(exp0).max()
        assert np.abs(out[part + 1] - expt).max() <= 1e-11 * max(1.0, np.abs(expt).max())


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("pr", [1.0, 0.72])
def test_viscous_smooth_time_derivative_is_euler(orc, dim, pr):
    """Identical smooth sides, viscous tau = mu/p: the interface distribution
    is f(t) = g0 - tau (a.u + A) g0 + t A g0 exactly, so its time derivative is
    the equilibrium's, A g0, whose flux is the Euler one, A_x Q_t, whatever mu
    and Pr.  The heat-flux fix (C16) acts on the non-equilibrium part of f,
    which does not change in time here, so it must leave F_t alone; a fix that
    took the heat flux of all of f_t would count the work of the pressure
    gradient at the interface velocity, (E + p) dU/dt, as heat."""
    rng = np.random.default_rng(300 + dim)
    for trial in range(3):
        u = rng.uniform(-0.5, 0.5, dim) if trial else np.zeros(dim)
        W = cons(dim, rng.uniform(0.6, 1.5), u, rng.uniform(0.6, 1.5))
        dW = rng.standard_normal((dim, dim + 2)) * 0.3
        out = orc.gks_point(dim, W, dW, W, dW, 1e-3, mu=2e-3, prandtl=pr, tau_mode=2)
        Qt = _euler_dt(W, dW, dim)
        Ft = jac(lambda w: euler_flux(w, dim, 1.4), W) @ Qt
        assert np.abs(out[1] - Ft).max() <= 1e-10 * max(1.0, np.abs(Ft).max()), (trial, out[1], Ft)
        assert np.allclose(out[3], Qt, rtol=1e-11, atol=1e-11) and np.allclose(out[5], Qt, rtol=1e-11, atol=1e-11)
