"""The allocation-free time step (cgks_compute_dt_noalloc) against the
context path (cgks_compute_dt).

Some callers cannot let this library call cudaMalloc -- their device memory
is reserved up front by another allocator, or they run a timed loop where an
allocation could synchronise the device -- so they compute the time step of a
state they already hold through this one entry point, whose work space is a
fixed array in device memory.  The test checks, on two calls in a row with
different meshes (repeated), that it returns the same dt as the library's
usual path and takes no device memory after the first call, that it flags
a non-physical cell and returns a fixed dt as given, and that a mesh above
the array's capacity is refused.  This file is collected last so that a
failure here stops a -x run only after all other tests have run.
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
    import torch
    from paper_2508_08965_gb300.binding import compute_dt_noalloc
    cases = [
        (3, (16, 12, 10), (0.0, 0.0, 0.0), (2 * math.pi,) * 3, lambda x, y, z: synth.taylor_green_3d(x, y, z),
         dict(mu=1 / 1600, prandtl=0.72, tau_mode=2)),
        (2, (64, 48), (0.0, 0.0), (10.0, 10.0), lambda x, y: synth.isentropic_vortex_2d(x, y), {}),
    ]
    refs = [_reference_dt(cg, dim, n, lo, hi, fn, **kw) for dim, n, lo, hi, fn, kw in cases]
    torch.cuda.synchronize()
    free0 = None
    for rep in range(3):
        for (dim, n, lo, hi, fn, kw), (dt_ref, state) in zip(cases, refs):  # two calls in a row
            status, dt = compute_dt_noalloc(state, dim, n, lo, hi, mu=kw.get("mu", 0.0))
            assert status == 0
            assert abs(dt - dt_ref) <= 1e-14 * dt_ref
        if rep == 0:  # the first call on the device has looked up the scratch array
            free0 = torch.cuda.mem_get_info()[0]
    # later calls take no device memory (the allocator's cache holds the
    # states; nothing is created or freed by the calls themselves)
    assert torch.cuda.mem_get_info()[0] == free0
    # a positive dt_fixed is returned as it is
    dim, n, lo, hi, fn, kw = cases[1]
    status, dt = compute_dt_noalloc(refs[1][1], dim, n, lo, hi, dt_fixed=1.25e-3)
    assert status == 0 and dt == 1.25e-3


def test_noalloc_flags_a_non_physical_cell(cg):
    from paper_2508_08965_gb300.binding import compute_dt_noalloc
    dim, n, lo, hi = 2, (64, 48), (0.0, 0.0), (10.0, 10.0)
    dt_ref, state = _reference_dt(cg, dim, n, lo, hi, lambda x, y: synth.isentropic_vortex_2d(x, y))
    bad = state.clone()
    bad[0, 3, 17, 29] = -1.0  # energy of one cell: negative pressure
    status, _ = compute_dt_noalloc(bad, dim, n, lo, hi)
    assert status == -4  # CGKS_ENONPHYS
    status, dt = compute_dt_noalloc(state, dim, n, lo, hi)  # the next call is unaffected
    assert status == 0 and abs(dt - dt_ref) <= 1e-14 * dt_ref


def test_noalloc_rejects_meshes_beyond_capacity(cg):
    import torch
    from paper_2508_08965_gb300.binding import compute_dt_noalloc
    n = (512, 256, 129)  # 16.9 M cells, one plane above the capacity
    with pytest.raises(ValueError):  # a buffer shorter than the averages: the binding refuses it
        compute_dt_noalloc(torch.zeros(8, dtype=torch.float64, device="cuda"), 3, n, (0, 0, 0), (1, 1, 1))
    state = torch.zeros(5 * 512 * 256 * 129, dtype=torch.float64, device="cuda")
    status, _ = compute_dt_noalloc(state, 3, n, (0, 0, 0), (1, 1, 1))
    assert status == -8  # CGKS_ETOOLARGE, refused before any launch
    del state
    torch.cuda.empty_cache()
