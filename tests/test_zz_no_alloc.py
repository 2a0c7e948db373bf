"""The allocation-free time step (cgks_compute_dt_noalloc) against the
context path (cgks_compute_dt).

Some callers cannot let this library call cudaMalloc -- their device memory
is reserved up front by another allocator, or they run a timed loop where an
allocation could synchronise the device -- so they compute the time step of a
state they already hold through this one entry point, whose work space is a
fixed array in device memory.  The test checks, on two calls in a row with
different meshes, that it returns the same dt as the library's usual path,
and that a mesh above the array's capacity is refused.  This file is
collected last so that a failure here stops a -x run only after all other
tests have run.
"""
import math

import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_08965_gb300 as p
    p.lib()
    return p


def _reference_dt(cg, dim, n, lo, hi, fn, **kw):
    import torch
    m = cg.Mesh(dim, n, lo=lo, hi=hi, **kw)
    m.init(fn)
    dt = m.compute_dt()
    state = torch.empty(m.state_shape, dtype=torch.float64, device="cuda")
    m.get_state(state)
    m.close()
    return dt, state


def test_noalloc_dt_matches_context_dt_twice(cg):
    from paper_2508_08965_gb300.binding import compute_dt_noalloc
    cases = [
        (3, (16, 12, 10), (0.0, 0.0, 0.0), (2 * math.pi,) * 3, lambda x, y, z: synth.taylor_green_3d(x, y, z),
         dict(mu=1 / 1600, prandtl=0.72, tau_mode=2)),
        (2, (64, 48), (0.0, 0.0), (10.0, 10.0), lambda x, y: synth.isentropic_vortex_2d(x, y), {}),
    ]
    for dim, n, lo, hi, fn, kw in cases:  # two calls in a row, the second on a smaller mesh
        dt_ref, state = _reference_dt(cg, dim, n, lo, hi, fn, **kw)
        status, dt = compute_dt_noalloc(state, dim, n, lo, hi, mu=kw.get("mu", 0.0))
        assert status == 0
        assert abs(dt - dt_ref) <= 1e-14 * dt_ref


def test_noalloc_rejects_meshes_beyond_capacity(cg):
    import torch
    from paper_2508_08965_gb300.binding import compute_dt_noalloc
    state = torch.zeros(8, dtype=torch.float64, device="cuda")
    status, _ = compute_dt_noalloc(state, 3, (512, 256, 129), (0, 0, 0), (1, 1, 1))
    assert status == -8  # CGKS_ETOOLARGE, refused before any launch
