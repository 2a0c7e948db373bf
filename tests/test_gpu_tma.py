"""The interface flux's two ways of staging a face point's Gauss-point
states in shared memory give the same results bit for bit: one TMA tile
(cp.async.bulk.tensor) per block of 128 points, which the library takes on
Cartesian meshes whose cell count is a multiple of 128, and one cp.async
per value and thread (forced by CGKS_FLUX_STAGING=cp.async when the
context is created).  Every form: FP64, the FP32 form, the paired form, in
2-D and 3-D, with and without walls."""
import math
import os

import numpy as np
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


def _run(cg, kw, fn, steps, staging):
    if staging == "cp.async":
        os.environ["CGKS_FLUX_STAGING"] = "cp.async"
    try:
        m = cg.Mesh(**kw)
    finally:
        os.environ.pop("CGKS_FLUX_STAGING", None)
    assert m.flux_staging == staging
    m.init(fn)
    m.step(steps)
    s, t = m.get_state()
    m.close()
    return s, t


CASES = [
    ("tgv16", dict(dim=3, n=(16, 16, 16), lo=(0, 0, 0), hi=(2 * math.pi,) * 3, mu=1 / 1600, prandtl=0.72,
                   tau_mode=2), lambda x, y, z: synth.taylor_green_3d(x, y, z)),
    ("box3d-walls", dict(dim=3, n=(16, 8, 8), lo=(0, 0, 0), hi=(1, 1, 1), bc=[2, 2, 0, 0, 3, 3], mu=1e-3,
                         prandtl=0.72, tau_mode=2), lambda x, y, z: synth.taylor_green_3d(2 * math.pi * x,
                                                                                          2 * math.pi * y,
                                                                                          2 * math.pi * z)),
    ("vortex64", dict(dim=2, n=(64, 64), lo=(0, 0), hi=(10, 10)), lambda x, y: synth.isentropic_vortex_2d(x, y)),
]


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_tma_and_cp_async_staging_agree(cg, case, precision):
    _, kw, fn = case
    kw = dict(kw, precision=precision)
    s_tma, t_tma = _run(cg, kw, fn, 5, "tma")
    s_cpa, t_cpa = _run(cg, kw, fn, 5, "cp.async")
    assert t_tma == t_cpa
    assert np.array_equal(s_tma, s_cpa)


def test_staging_falls_back_where_tiles_do_not_fit(cg):
    """cell counts that are not a multiple of 128, and curvilinear meshes,
    stage by cp.async"""
    m = cg.Mesh(3, (7, 9, 11), lo=(0, 0, 0), hi=(1, 1, 1))
    assert m.flux_staging == "cp.async"
    m.close()
    n = (8, 8, 8)
    m = cg.Mesh(3, n, nodes=synth.perturbed_nodes_3d(n), bc=[0] * 6)
    assert m.flux_staging == "cp.async"
    m.close()


def test_staging_wait_gives_up_with_a_status(cg):
    """The flux blocks' wait for their TMA tiles is bounded (about a second):
    with the test hook CGKS_TEST_STAGING_STALL=1 every barrier waits for 16
    bytes that never come, the first wave of blocks gives up, later blocks
    skip their wait, and cgks_step returns CGKS_ETIMEOUT with the state and
    time of the last good step (here the initial ones).  Nothing faults: the
    tiles themselves land; only the barrier is held back."""
    import time
    kw = dict(dim=3, n=(16, 16, 16), lo=(0, 0, 0), hi=(2 * math.pi,) * 3, mu=1 / 1600, prandtl=0.72,
              tau_mode=2, precision=1)
    fn = lambda x, y, z: synth.taylor_green_3d(x, y, z)
    os.environ["CGKS_TEST_STAGING_STALL"] = "1"
    try:
        m = cg.Mesh(**kw)
    finally:
        os.environ.pop("CGKS_TEST_STAGING_STALL", None)
    assert m.flux_staging == "tma"
    m.init(fn)
    s0, t0 = m.get_state()
    w0 = time.perf_counter()
    with pytest.raises(cg.CgksError) as err:
        m.step(2)
    assert err.value.status == -5  # CGKS_ETIMEOUT
    assert time.perf_counter() - w0 < 30.0
    s1, t1 = m.get_state()
    assert t1 == t0 and np.array_equal(s1, s0)
    m.close()
    # a context without the hook steps normally from the same state
    m = cg.Mesh(**kw)
    m.set_state(s0, t0)
    m.step(2)
    m.close()
