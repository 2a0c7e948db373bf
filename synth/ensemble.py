"""Seeded ensembles of independent 2-D cases (uneven sizes), for the batched
path: each case is an isentropic vortex on a periodic box or a four-quadrant
Riemann problem with outflow boundaries.  Case descriptions only; no scheme
arithmetic."""
import numpy as np

from .fields import isentropic_vortex_2d, riemann4_2d, riemann4_params

SIZES = (64, 128, 256, 512)


def ensemble_stream(seed=20250811, sizes=SIZES):
    """Endless seeded stream of case descriptions.  Per case: mesh size
    (nx, ny) drawn independently from `sizes`; kind vortex (strength
    eps ~ U[1, 5], centre ~ U[2, 8]^2 on the periodic [0, 10]^2, free stream
    (1, 1, 1, 1)) or riemann (states of riemann4_params(case seed) on
    [0, 1]^2, split at (0.5, 0.5), outflow boundaries, shock-capturing
    collision time), each with probability 1/2."""
    rng = np.random.default_rng(seed)
    while True:
        nx, ny = (int(rng.choice(sizes)) for _ in range(2))
        if rng.random() < 0.5:
            yield dict(kind="vortex", n=(nx, ny), eps=float(rng.uniform(1.0, 5.0)),
                       center=tuple(float(c) for c in rng.uniform(2.0, 8.0, 2)))
        else:
            yield dict(kind="riemann", n=(nx, ny), seed=int(rng.integers(0, 2 ** 31 - 1)))


def ensemble_specs(ncase=256, seed=20250811, sizes=SIZES):
    """The first ncase descriptions of ensemble_stream(seed)."""
    it = ensemble_stream(seed, sizes)
    return [next(it) for _ in range(ncase)]


def spec_mesh(spec):
    """Keyword arguments of the case's mesh (dim, n, lo, hi, bc, tau_mode)."""
    if spec["kind"] == "vortex":
        return dict(dim=2, n=spec["n"], lo=(0.0, 0.0), hi=(10.0, 10.0), bc=[0, 0, 0, 0], tau_mode=0)
    return dict(dim=2, n=spec["n"], lo=(0.0, 0.0), hi=(1.0, 1.0), bc=[1, 1, 1, 1], tau_mode=1)


def spec_field(spec):
    """The case's initial primitive field f(x, y) -> [rho, u, v, p]."""
    if spec["kind"] == "vortex":
        eps, center = spec["eps"], spec["center"]
        return lambda x, y: isentropic_vortex_2d(x, y, eps=eps, center=center)
    states = riemann4_params(spec["seed"])
    return lambda x, y: riemann4_2d(x, y, states)
