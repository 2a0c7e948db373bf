"""GPU parity of the paired form (precision 2: FP64 storage and arithmetic,
the interior interface flux solved in paired-FP32 arithmetic) against the
FP64 CPU oracle, at the FP64 bars: 1e-12 after one S2O4 step, 1e-9 after
100 steps (class-scaled as in tests/parity.py).  The same cases pass on the
host build of the kernels (tests/test_host_parity.py)."""
import math

import pytest

import synth
from parity import class_scaled_diff

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_08965_gb300 as p
    p.lib()
    return p


TGV = {"mu": 1 / 1600, "prandtl": 0.72, "tau_mode": 2}
CASES = [
    ("vortex-ragged", 2, (37, 29), (0, 0), (10, 10), lambda x, y: synth.isentropic_vortex_2d(x, y), None,
     {"tau_mode": 1}),
    ("tgv16", 3, (16, 16, 16), (0, 0, 0), (2 * math.pi,) * 3, lambda x, y, z: synth.taylor_green_3d(x, y, z),
     None, TGV),
    ("tgv-ragged", 3, (7, 9, 11), (0, 0, 0), (2 * math.pi,) * 3, lambda x, y, z: synth.taylor_green_3d(x, y, z),
     None, TGV),
    ("tgv-curvilinear", 3, (10, 10, 10), (0, 0, 0), (2 * math.pi,) * 3,
     lambda x, y, z: synth.taylor_green_3d(x, y, z), "perturbed", TGV),
    ("walls-3d", 3, (8, 7, 9), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), lambda x, y, z: synth.taylor_green_3d(x, y, z),
     None, dict(TGV, bc=[3, 3, 2, 2, 1, 1])),
]


def _run(orc, cg, case, steps):
    name, dim, n, lo, hi, fn, nodes, kw = case
    if nodes == "perturbed":
        nodes = synth.perturbed_nodes_3d(n)
    o = orc.Oracle(dim, n, lo=lo, hi=hi, nodes=nodes, **kw)
    o.init(fn)
    m = cg.Mesh(dim, n, lo=lo, hi=hi, nodes=nodes, precision=2, **kw)
    m.set_state(o.get_state())
    o.step(steps)
    m.step(steps)
    sg, _ = m.get_state()
    m.close()
    h = min((hi[a] - lo[a]) / n[a] for a in range(dim)) * (0.7 if nodes is not None else 1.0)
    return class_scaled_diff(sg, o.get_state(), h)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_paired_one_step(orc, cg, case):
    d = _run(orc, cg, case, 1)
    print("%s: %.2e" % (case[0], d))
    assert d <= 1e-12


@pytest.mark.parametrize("case", [
    ("vortex-100", 2, (24, 24), (0, 0), (10, 10), lambda x, y: synth.isentropic_vortex_2d(x, y), None, {}),
    ("tgv12", 3, (12, 12, 12), (0, 0, 0), (2 * math.pi,) * 3, lambda x, y, z: synth.taylor_green_3d(x, y, z),
     None, TGV),
    CASES[3]], ids=["vortex24", "tgv12", "tgv-curvilinear"])
def test_paired_hundred_steps(orc, cg, case):
    d = _run(orc, cg, case, 100)
    print("%s 100 steps: %.2e" % (case[0], d))
    assert d <= 1e-9
