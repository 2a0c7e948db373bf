"""Mirror image of a state in the public layout, written independently of
both the oracle and the library, for the wall-boundary pins.

Reflecting the domain across a plane normal to axis `a` maps the flow to
another flow of the Euler / Navier-Stokes equations: the momentum component
along `a` changes sign, so do derivatives along `a`, and the Gauss points of a
face swap their coordinate along `a` (1/2 - g <-> 1/2 + g).  With data that do
not depend on the tangential coordinates, negating the tangential momentum as
well (the no-slip image) is again a symmetry, since the tangential momentum is
then a passive scalar that enters the other equations only quadratically.

State array shape: (nf, nv, [n2,] n1, n0); field f = 0 average, f = 1..dim
gradient components, f = 1 + dim + axis*gpf + k line derivatives.
"""
import numpy as np


def _sign_var(dim, v, a, noslip):
    if 1 <= v <= dim and (noslip or v == 1 + a):
        return -1.0
    return 1.0


def reflect(S, dim, a, noslip=False):
    """Mirror image of S across a plane normal to axis a (cells reversed)."""
    gpf = 4 if dim == 3 else 2
    nf, nv = S.shape[:2]
    arr_axis = 2 + (dim - 1 - a)
    F = np.flip(S, axis=arr_axis)
    R = np.empty_like(S)
    for v in range(nv):
        sv = _sign_var(dim, v, a, noslip)
        R[0, v] = sv * F[0, v]
        for k in range(dim):
            R[1 + k, v] = sv * (-1.0 if k == a else 1.0) * F[1 + k, v]
        for b in range(dim):
            tang = [x for x in range(dim) if x != b]
            for q in range(gpf):
                src = 1 + dim + b * gpf + q
                if b == a:
                    R[src, v] = -sv * F[src, v]
                else:
                    bit = tang.index(a)
                    dst = 1 + dim + b * gpf + (q ^ (1 << bit))
                    R[dst, v] = sv * F[src, v]
    return R


def extend(S, dim, a, noslip=False):
    """[mirror image, S] along axis a: a periodic state of twice the length
    whose restriction to the upper half obeys walls at both ends of S."""
    arr_axis = 2 + (dim - 1 - a)
    return np.concatenate([reflect(S, dim, a, noslip), S], axis=arr_axis)


def upper_half(S, dim, a):
    arr_axis = 2 + (dim - 1 - a)
    n = S.shape[arr_axis] // 2
    return np.take(S, np.arange(n, 2 * n), axis=arr_axis)
