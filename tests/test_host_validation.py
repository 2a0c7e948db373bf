"""Argument checks of the C-ABI that return before any CUDA call, so they
run without a GPU: degenerate and empty meshes, unknown boundary codes,
periodic faces opposite non-periodic ones, walls and inflow faces on
curvilinear meshes, invalid physics, and the batch's mixed descriptors.
Every rejected descriptor must give its documented status and no context."""
import ctypes as C

import pytest

import synth

EINVAL, EUNSUPPORTED = -1, -7


@pytest.fixture(scope="module")
def cg():
    from paper_2508_08965_gb300 import binding
    binding.lib()
    return binding


def create(cg, **kw):
    d, keep = cg.make_desc(**kw)
    h = C.c_void_p()
    st = cg.lib().cgks_create_mesh(C.byref(d), C.byref(h))
    return st, h, keep


CASES = [
    ("zero cells", dict(dim=2, n=(0, 8)), EINVAL),
    ("two cells along an axis", dict(dim=3, n=(8, 2, 8)), EINVAL),
    ("dimension 1", dict(dim=1, n=(8,)), EINVAL),
    ("dimension 4", dict(dim=4, n=(8, 8, 8)), EINVAL),
    ("boundary code 5", dict(dim=2, n=(8, 8), bc=[5, 5, 0, 0]), EINVAL),
    ("negative boundary code", dict(dim=2, n=(8, 8), bc=[-1, 1, 0, 0]), EINVAL),
    ("periodic opposite a wall", dict(dim=2, n=(8, 8), bc=[0, 2, 0, 0]), EINVAL),
    ("periodic opposite inflow", dict(dim=3, n=(6, 6, 6), bc=[1, 1, 4, 0, 0, 0]), EINVAL),
    ("gamma 1", dict(dim=2, n=(8, 8), gamma=1.0), EINVAL),
    ("negative viscosity", dict(dim=2, n=(8, 8), mu=-1e-3), EINVAL),
    ("zero CFL", dict(dim=2, n=(8, 8), cfl=0.0), EINVAL),
    ("collision-time mode 3", dict(dim=2, n=(8, 8), tau_mode=3), EINVAL),
    ("precision 3", dict(dim=2, n=(8, 8), precision=3), EUNSUPPORTED),
    ("negative precision", dict(dim=2, n=(8, 8), precision=-1), EUNSUPPORTED),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_create_mesh_rejects(cg, case):
    name, kw, want = case
    st, h, _ = create(cg, **kw)
    assert st == want and not h.value


@pytest.mark.parametrize("bc", [[2, 2, 0, 0, 0, 0], [3, 1, 0, 0, 0, 0], [4, 1, 0, 0, 0, 0]],
                         ids=["slip", "no-slip", "inflow"])
def test_walls_and_inflow_need_a_box(cg, bc):
    nodes = synth.perturbed_nodes_3d((6, 6, 6))
    st, h, _ = create(cg, dim=3, n=(6, 6, 6), nodes=nodes, bc=bc)
    assert st == EUNSUPPORTED and not h.value


def test_null_arguments(cg):
    L = cg.lib()
    h = C.c_void_p()
    assert L.cgks_create_mesh(None, C.byref(h)) == EINVAL
    d, _ = cg.make_desc(dim=2, n=(8, 8))
    assert L.cgks_create_mesh(C.byref(d), None) == EINVAL
    assert L.cgks_set_state(None, None, 0, 0.0) == EINVAL
    assert L.cgks_get_state(None, None, 0, None) == EINVAL
    assert L.cgks_step(None, 1, 0.0, None, None) == EINVAL
    assert L.cgks_flux_staging(None) == -1


def test_batch_rejects_mixed_and_invalid_cases(cg):
    L = cg.lib()
    ok, _ = cg.make_desc(dim=2, n=(8, 8))
    for bad, want in ((dict(dim=3, n=(8, 8, 8)), EINVAL),             # mixed dimensions
                      (dict(dim=2, n=(8, 8), precision=1), EINVAL),   # mixed precisions
                      (dict(dim=2, n=(8, 8), precision=2), EINVAL),
                      (dict(dim=2, n=(8, 2)), EINVAL),
                      (dict(dim=2, n=(8, 8), bc=[2, 0, 0, 0]), EINVAL),
                      (dict(dim=2, n=(8, 8), nodes=synth.uniform_nodes((8, 8), (0, 0), (1, 1))), EUNSUPPORTED)):
        d, _ = cg.make_desc(**bad)
        arr = (cg.MeshDesc * 2)(ok, d)
        h = C.c_void_p()
        assert L.cgks_batch_create(arr, 2, None, C.byref(h)) == want, bad
        assert not h.value
    pd, _ = cg.make_desc(dim=2, n=(8, 8), precision=2)
    arr = (cg.MeshDesc * 2)(pd, pd)
    h = C.c_void_p()
    assert L.cgks_batch_create(arr, 2, None, C.byref(h)) == EUNSUPPORTED and not h.value   # paired form
    assert L.cgks_batch_create(None, 1, None, C.byref(h)) == EINVAL
    arr = (cg.MeshDesc * 1)(ok)
    assert L.cgks_batch_create(arr, 0, None, C.byref(h)) == EINVAL


def test_async_copy_buffers(cg):
    """the binding's checks on the buffers of the asynchronous copies"""
    import numpy as np
    import torch
    buf = cg.Mesh._buffer
    a = np.zeros((3, 4))
    p, dev, keep = buf(a, True)
    assert p == a.ctypes.data and dev == 0 and keep is a
    t = torch.zeros(12, dtype=torch.float64)
    p, dev, keep = buf(t, False)
    assert p == t.data_ptr() and dev == 0 and keep is t
    for bad in (np.zeros(4, dtype=np.float32), np.zeros((4, 4))[:, 1], torch.zeros(4, dtype=torch.float32),
                torch.zeros((4, 4), dtype=torch.float64)[:, 1], [0.0] * 4):
        with pytest.raises(ValueError):
            buf(bad, False)
    ro = np.zeros(4)
    ro.flags.writeable = False
    assert buf(ro, False)[2] is ro
    with pytest.raises(ValueError):
        buf(ro, True)


def test_state_copies_refuse_bad_buffers(cg):
    """The binding checks every buffer the library would read or write
    before the call: size, dtype, contiguity, writability, device.  (Objects
    built without a context: each refusal happens before any library call.)"""
    import numpy as np
    import torch
    m = object.__new__(cg.Mesh)
    m._h, m._pending = None, []
    m.dim, m.n, m.nf, m.nv, m.ncell = 2, (4, 3), 7, 4, 12
    size = 7 * 4 * 12
    for bad in (np.zeros(size - 1), np.zeros(size, dtype=np.float32), np.zeros(2 * size)[::2],
                torch.zeros(size, dtype=torch.float32), torch.zeros(size + 1, dtype=torch.float64)):
        with pytest.raises(ValueError):
            m.get_state(out=bad)
    ro = np.zeros(size)
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        m.get_state(out=ro)
    for bad in (np.zeros(size - 1), np.zeros(size + 7)):
        with pytest.raises(ValueError):
            m.set_state(bad)
    b = object.__new__(cg.Batch)
    b._h, b.ncase, b.dims = None, 2, [(2, (4, 3)), (2, (8, 8))]
    with pytest.raises(ValueError):
        b.set_state(1, np.zeros(size))  # case 0's size given for case 1
    with pytest.raises(IndexError):
        b.set_state(2, np.zeros(size))
    # the allocation-free time step and the network kernels take CUDA tensors only
    with pytest.raises(ValueError):
        cg.compute_dt_noalloc(torch.zeros(4 * 12, dtype=torch.float64), 2, (4, 3), (0, 0), (1, 1))
    with pytest.raises(ValueError):
        cg._f32(torch.zeros(16, dtype=torch.float32), 16, "X")
