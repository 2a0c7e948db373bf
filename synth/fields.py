"""Analytic primitive fields (rho, U, V[, W], p) used as initial data.

Each function takes coordinate arrays (numpy or torch, any shape) and returns a
list of primitive arrays of the same shape.  Formulas:

* isentropic vortex: the standard 2-D vortex on a periodic box, with the
  minimum-image displacement from the (advected) centre.
* Taylor-Green vortex: the paper's Sec. 6.2 initial field with L = U0 = rho0 = 1,
  p0 = 1/(gamma Ma^2).
* density sine wave: the paper's Sec. 6.1 accuracy test (exact at any t).
* Riemann data: Sod along x and seeded four-quadrant problems.
"""
import math

import numpy as np


def _ns(a):
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return torch
    except ImportError:  # pragma: no cover
        pass
    return np


def _min_image(d, period):
    return d - period * _ns(d).round(d / period)


def isentropic_vortex_2d(x, y, eps=5.0, center=(5.0, 5.0), u_inf=(1.0, 1.0),
                         p_inf=1.0, rho_inf=1.0, gamma=1.4, t=0.0,
                         period=(10.0, 10.0)):
    """Isentropic vortex advected by the free stream; exact for all t on the
    unbounded plane, taken here with the minimum-image displacement."""
    xp = _ns(x)
    xc = center[0] + u_inf[0] * t
    yc = center[1] + u_inf[1] * t
    dx = _min_image(x - xc, period[0])
    dy = _min_image(y - yc, period[1])
    r2 = dx * dx + dy * dy
    e = xp.exp(0.5 * (1.0 - r2))
    du = -(eps / (2.0 * math.pi)) * e * dy
    dv = (eps / (2.0 * math.pi)) * e * dx
    t_inf = p_inf / rho_inf
    temp = t_inf - (gamma - 1.0) * eps * eps / (8.0 * gamma * math.pi ** 2) * e * e
    rho = rho_inf * (temp / t_inf) ** (1.0 / (gamma - 1.0))
    p = rho * temp
    return [rho, u_inf[0] + du, u_inf[1] + dv, p]


def taylor_green_3d(x, y, z, mach=0.1, gamma=1.4):
    """Taylor-Green vortex initial field (Sec. 6.2), L = U0 = rho0 = 1."""
    xp = _ns(x)
    p0 = 1.0 / (gamma * mach * mach)
    u = xp.sin(x) * xp.cos(y) * xp.cos(z)
    v = -xp.cos(x) * xp.sin(y) * xp.cos(z)
    w = 0.0 * x
    f = 1.0 + gamma * mach * mach / 16.0 * (xp.cos(2.0 * x) + xp.cos(2.0 * y)) * (xp.cos(2.0 * z) + 2.0)
    return [f, u, v, w, p0 * f]


def density_sine_3d(x, y, z, t=0.0, amp=0.2):
    """Sec. 6.1 accuracy test: rho = 1 + 0.2 sin(pi (x+y+z-3t)), U=V=W=p=1."""
    xp = _ns(x)
    rho = 1.0 + amp * xp.sin(math.pi * (x + y + z - 3.0 * t))
    one = 1.0 + 0.0 * x
    return [rho, one, one, one, one]


def uniform_state(prims, *coords):
    """A constant primitive state broadcast to the shape of the coordinates."""
    x = coords[0]
    return [c + 0.0 * x for c in prims]


def sod_x(x, *coords, x0=0.5, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1)):
    """Sod's shock tube along x (rho, u, p); other velocities zero."""
    xp = _ns(x)
    lft = x < x0
    rho = xp.where(lft, left[0] + 0.0 * x, right[0] + 0.0 * x)
    u = xp.where(lft, left[1] + 0.0 * x, right[1] + 0.0 * x)
    p = xp.where(lft, left[2] + 0.0 * x, right[2] + 0.0 * x)
    out = [rho, u] + [0.0 * x for _ in coords] + [p]
    return out


def riemann4_params(seed):
    """Seeded four-quadrant states: rho, p ~ U[0.1, 2], u, v ~ U[-1, 1]."""
    rng = np.random.default_rng(seed)
    q = []
    for _ in range(4):
        rho = rng.uniform(0.1, 2.0)
        u = rng.uniform(-1.0, 1.0)
        v = rng.uniform(-1.0, 1.0)
        p = rng.uniform(0.1, 2.0)
        q.append((rho, u, v, p))
    return q


def riemann4_2d(x, y, states, split=(0.5, 0.5)):
    """Four-quadrant Riemann data; quadrants ordered (x>,y>), (x<,y>), (x<,y<), (x>,y<)."""
    xp = _ns(x)
    right = x >= split[0]
    top = y >= split[1]
    out = []
    for c in range(4):
        q1, q2, q3, q4 = (s[c] for s in states)
        val = xp.where(right & top, q1 + 0.0 * x,
                       xp.where(~right & top, q2 + 0.0 * x,
                                xp.where(~right & ~top, q3 + 0.0 * x, q4 + 0.0 * x)))
        out.append(val)
    return out


def turbulence_velocity_grid(n, seed, k0=8.0):
    """Seeded solenoidal velocity on an n^3 periodic grid over [0, 2 pi)^3 with
    energy spectrum E(k) ~ k^4 exp(-2 (k/k0)^2), unit rms (numpy, float64)."""
    rng = np.random.default_rng(seed)
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    kx, ky, kz = np.meshgrid(k1, k1, k1, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    kk = np.sqrt(k2)
    kk[0, 0, 0] = 1.0
    ek = kk ** 4 * np.exp(-2.0 * (kk / k0) ** 2)
    amp = np.sqrt(ek / (4.0 * np.pi * kk * kk))
    amp[0, 0, 0] = 0.0
    comps = []
    for _ in range(3):
        comps.append(amp * (rng.standard_normal(kk.shape) + 1j * rng.standard_normal(kk.shape)))
    div = (kx * comps[0] + ky * comps[1] + kz * comps[2]) / np.where(k2 == 0, 1.0, k2)
    comps = [comps[0] - kx * div, comps[1] - ky * div, comps[2] - kz * div]
    vel = [np.real(np.fft.ifftn(c)) for c in comps]
    rms = np.sqrt(np.mean(vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2) / 3.0)
    return [v / rms for v in vel]


def random_smooth_3d(x, y, z, seed, nmodes=4, mach=0.1, gamma=1.4, length=2.0 * math.pi):
    """Seeded smooth periodic 3-D flow on [0, length)^3: density, velocity and
    pressure perturbed by `nmodes` random Fourier modes each (wave numbers
    1..3 per axis, random phases), velocity amplitude 1, mean density 1 and
    mean pressure 1/(gamma mach^2)."""
    xp = _ns(x)
    rng = np.random.default_rng(seed)
    two_pi = 2.0 * math.pi / length

    def modes(amp):
        out = 0.0 * x
        for _ in range(nmodes):
            k = rng.integers(-3, 4, 3)
            if not np.any(k):
                k[0] = 1
            ph = rng.uniform(0, 2 * math.pi)
            a = amp * rng.uniform(0.5, 1.0) / nmodes
            out = out + a * xp.sin(two_pi * (k[0] * x + k[1] * y + k[2] * z) + ph)
        return out
    p0 = 1.0 / (gamma * mach * mach)
    rho = 1.0 + modes(0.1)
    u, v, w = modes(1.0), modes(1.0), modes(1.0)
    p = p0 * (1.0 + modes(0.05))
    return [rho, u, v, w, p]


def turbulence_field(seed, n=128, k0=8.0, mach_t=0.5, re_lambda=72.0, gamma=1.4):
    """Decaying isotropic turbulence initial data on the periodic [0, 2 pi)^3:
    the seeded solenoidal velocity of turbulence_velocity_grid (spectrum
    E(k) ~ k^4 exp(-2 (k/k0)^2)) on an n^3 grid, scaled so that
    Ma_t = sqrt(<|u|^2>) / c = mach_t with rho = 1, p = 1/gamma (c = 1), and
    evaluated anywhere by periodic trilinear interpolation.  Returns
    (field(x, y, z) -> [rho, u, v, w, p], mu) with mu from
    Re_lambda = rho u_rms lambda / mu, u_rms = sqrt(<|u|^2>/3) and
    lambda = u_rms / (du/dx)_rms, the derivative taken spectrally on the
    grid."""
    vel = turbulence_velocity_grid(n, seed, k0)
    scale = mach_t / math.sqrt(np.mean(vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2))
    vel = [v * scale for v in vel]
    u_rms = math.sqrt(np.mean(vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2) / 3.0)
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    dudx = np.real(np.fft.ifftn(1j * k1[:, None, None] * np.fft.fftn(vel[0])))
    lam = u_rms / math.sqrt(np.mean(dudx ** 2))
    mu = u_rms * lam / re_lambda
    h = 2.0 * math.pi / n
    grids = {}

    def field(x, y, z):
        xp = _ns(x)
        key = id(xp)
        if key not in grids:
            if xp is np:
                grids[key] = [np.asarray(v) for v in vel]
            else:
                grids[key] = [xp.as_tensor(v, dtype=x.dtype, device=x.device) for v in vel]
        g = grids[key]
        fx, fy, fz = x / h, y / h, z / h
        i0, j0, k0_ = xp.floor(fx), xp.floor(fy), xp.floor(fz)
        tx, ty, tz = fx - i0, fy - j0, fz - k0_
        out = []
        for comp in g:
            acc = 0.0 * x
            for dx in (0, 1):
                for dy in (0, 1):
                    for dz in (0, 1):
                        ii = ((i0 + dx) % n).long() if xp is not np else ((i0 + dx) % n).astype(np.int64)
                        jj = ((j0 + dy) % n).long() if xp is not np else ((j0 + dy) % n).astype(np.int64)
                        kk = ((k0_ + dz) % n).long() if xp is not np else ((k0_ + dz) % n).astype(np.int64)
                        w = (tx if dx else 1 - tx) * (ty if dy else 1 - ty) * (tz if dz else 1 - tz)
                        acc = acc + w * comp[ii, jj, kk]
            out.append(acc)
        return [1.0 + 0.0 * x, out[0], out[1], out[2], 1.0 / gamma + 0.0 * x]

    return field, mu


def shock_vortex_params(seed, mach_range=(1.1, 3.0), eps_range=(1.0, 5.0)):
    """Seeded (shock Mach number, vortex strength), uniform in the ranges."""
    rng = np.random.default_rng(seed)
    return float(rng.uniform(*mach_range)), float(rng.uniform(*eps_range))


def shock_vortex_upstream(mach, gamma=1.4):
    """Upstream (rho, u, v, p) of the stationary normal shock: rho = p = 1,
    u = mach * sqrt(gamma) (the upstream sound speed is sqrt(gamma))."""
    return (1.0, mach * math.sqrt(gamma), 0.0, 1.0)


def shock_vortex_2d(x, y, mach, eps=3.0, rc=0.05, center=(0.25, 0.5), x_shock=0.5, gamma=1.4):
    """Shock-vortex interaction on [0, 2] x [0, 1]: a stationary normal shock
    at x = x_shock with upstream Mach number `mach` (Rankine-Hugoniot state
    behind it) and, superposed on the upstream flow at `center`, the
    isentropic vortex of the vortex-advection test with lengths in units of
    the core radius rc (r = |x - center| / rc):
        u' = -(eps / 2 pi) e^{(1 - r^2)/2} (y - yc) / rc,
        v' =  (eps / 2 pi) e^{(1 - r^2)/2} (x - xc) / rc,
        T' = -(gamma - 1) eps^2 / (8 gamma pi^2) e^{1 - r^2},
    T = p / rho, with the upstream entropy p / rho^gamma.  The scaled vortex
    is still a steady solution of the Euler equations (the radial balance
    dp/dr = rho v_theta^2 / r scales by 1/rc on both sides)."""
    xp = _ns(x)
    r1, u1, _, p1 = shock_vortex_upstream(mach, gamma)
    m2 = mach * mach
    r2 = r1 * (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    p2 = p1 * (1.0 + 2.0 * gamma * (m2 - 1.0) / (gamma + 1.0))
    u2 = u1 * r1 / r2
    dx = (x - center[0]) / rc
    dy = (y - center[1]) / rc
    e = xp.exp(0.5 * (1.0 - dx * dx - dy * dy))
    du = -(eps / (2.0 * math.pi)) * e * dy
    dv = (eps / (2.0 * math.pi)) * e * dx
    t1 = p1 / r1
    temp = t1 - (gamma - 1.0) * eps * eps / (8.0 * gamma * math.pi ** 2) * e * e
    rho_v = r1 * (temp / t1) ** (1.0 / (gamma - 1.0))
    p_v = rho_v * temp
    up = x < x_shock
    zero = 0.0 * x
    rho = xp.where(up, rho_v, r2 + zero)
    u = xp.where(up, u1 + du, u2 + zero)
    v = xp.where(up, dv, zero)
    p = xp.where(up, p_v, p2 + zero)
    return [rho, u, v, p]


def shock_vortex_inflow(mach, gamma=1.4):
    """Conservative upstream state for the inflow face of the shock-vortex
    problem: the unperturbed stream (the vortex's tail at x = 0, five core
    radii from its centre, is below 1e-4 of the stream)."""
    r, u, v, p = shock_vortex_upstream(mach, gamma)
    return [r, r * u, r * v, p / (gamma - 1.0) + 0.5 * r * (u * u + v * v)]
