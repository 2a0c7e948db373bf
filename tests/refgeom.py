"""Independent description of the standard reference cell used by the pins.

Written from the paper's definitions (Sec. 3.2 stencil, Eq. stencil-5 data,
Eq. base zero-mean basis, Sec. 4 standard cell [0,1]^dim with centroid 1/2):
the target cell is [-1/2, 1/2]^dim in delta = xi - 1/2, neighbours are unit
cells at integer offsets, face Gauss points sit at +-1/(2 sqrt 3) on each face.
The data vector order matches the oracle's documented layout.
"""
import itertools
import math

import numpy as np

G = 1.0 / (2.0 * math.sqrt(3.0))


def face_offsets(dim):
    out = []
    for m in range(2 * dim):
        o = [0] * dim
        o[m // 2] = 1 if m & 1 else -1
        out.append(tuple(o))
    return out


def edge_offsets_and_tau(dim):
    offs, taus = [], []
    for p in range(dim):
        for q in range(p + 1, dim):
            for sp in (-1, 1):
                for sq in (-1, 1):
                    o = [0] * dim
                    o[p], o[q] = sp, sq
                    offs.append(tuple(o))
                    t2 = np.zeros(dim)
                    t2[p], t2[q] = sp / math.sqrt(2), sq / math.sqrt(2)
                    if dim == 3:
                        t1 = np.zeros(3)
                        t1[3 - p - q] = 1.0
                        taus.append([t1, t2])
                    else:
                        taus.append([t2])
    return offs, taus


def gpf(dim):
    return 4 if dim == 3 else 2


def gp_delta(dim, axis, side, k):
    ta = [a for a in range(dim) if a != axis]
    d = np.zeros(dim)
    d[axis] = 0.5 if side else -0.5
    d[ta[0]] = G if (k & 1) else -G
    if dim == 3:
        d[ta[1]] = G if (k & 2) else -G
    return d


def all_gps(dim):
    return [gp_delta(dim, f // 2, f & 1, k) for f in range(2 * dim) for k in range(gpf(dim))]


_GX, _GW = np.polynomial.legendre.leggauss(4)


def cell_avg(fn, off, dim):
    """average of fn over the unit cell centred at `off` (4-point Gauss, exact to degree 7)."""
    s = 0.0
    for idx in itertools.product(range(4), repeat=dim):
        x = np.array([off[a] + 0.5 * _GX[idx[a]] for a in range(dim)])
        w = np.prod([_GW[i] for i in idx]) / 2 ** dim
        s = s + w * fn(x)
    return s


def data_vector(dim, f, grad):
    """Exact data (Eq. stencil-5, reference frame) of a smooth function f with gradient grad."""
    fo = face_offsets(dim)
    eo, taus = edge_offsets_and_tau(dim)
    d = [cell_avg(f, [0] * dim, dim)]
    d += [cell_avg(f, o, dim) for o in fo]
    d += [cell_avg(f, o, dim) for o in eo]
    for o in fo:
        g = cell_avg(grad, o, dim)
        d += list(g)
    for o, ts in zip(eo, taus):
        g = cell_avg(grad, o, dim)
        d += [float(np.dot(t, g)) for t in ts]
    for ax in range(dim):
        for k in range(gpf(dim)):
            d.append(f(gp_delta(dim, ax, 1, k)) - f(gp_delta(dim, ax, 0, k)))
    return np.array(d, dtype=np.float64)


def random_poly(dim, deg, rng):
    """random polynomial sum c_e x^e, |e| <= deg, with its gradient."""
    exps = [e for e in itertools.product(range(deg + 1), repeat=dim) if sum(e) <= deg]
    coef = rng.standard_normal(len(exps))

    def f(x):
        return sum(c * np.prod([x[a] ** e[a] for a in range(dim)]) for c, e in zip(coef, exps))

    def grad(x):
        g = np.zeros(dim)
        for c, e in zip(coef, exps):
            for a in range(dim):
                if e[a] == 0:
                    continue
                t = c * e[a]
                for b in range(dim):
                    t = t * x[b] ** (e[b] - (1 if b == a else 0))
                g[a] += t
        return g

    return f, grad
