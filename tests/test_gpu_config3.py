"""The non-orthogonal-mesh configuration: the periodic [0, 2 pi]^3 mesh of
192^3 cells perturbed by x_i = xi_i + 0.1 sin(xi_1) sin(xi_2) sin(xi_3), FP64
metrics.  Free-stream preservation at full size (a property that holds at
any size), decaying isotropic turbulence (Ma_t 0.5, Re_lambda 72) in FP32
against FP64 at full size, and oracle parity of the same recipe on a small
mesh."""
import math

import numpy as np
import pytest

import synth
from parity import class_scaled_diff

pytestmark = pytest.mark.gpu

N192 = (192, 192, 192)
SEED = 20250811


@pytest.fixture(scope="module")
def cg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_08965_gb300 as p
    p.lib()
    return p


def box(n):
    return dict(dim=3, n=n, lo=(0, 0, 0), hi=(2 * math.pi,) * 3, nodes=synth.perturbed_nodes_3d(n))


def test_free_stream_192(cg):
    """Uniform flow (1, 0.3, 0.2, 0.1, 1/gamma) stays uniform for 100 steps."""
    q = (1.0, 0.3, 0.2, 0.1, 1.0 / 1.4)
    m = cg.Mesh(mu=1e-3, prandtl=0.72, tau_mode=2, **box(N192))
    m.init(lambda x, y, z: [q[0] + 0 * x, q[1] + 0 * x, q[2] + 0 * x, q[3] + 0 * x, q[4] + 0 * x])
    s0, _ = m.get_state()
    m.step(100)
    s1, _ = m.get_state()
    m.close()
    # averages relative to their size; derivative fields (zero for a uniform
    # flow) relative to the size of a difference quotient, |Q| / h_min
    hmin = 0.7 * 2 * math.pi / 192
    dev_avg = np.abs(s1[0] - s0[0]).max() / np.abs(s0[0]).max()
    dev_der = np.abs(s1[1:]).max() * hmin / np.abs(s0[0]).max()
    print("free stream 192^3, 100 steps: averages %.2e, derivative fields %.2e" % (dev_avg, dev_der))
    assert dev_avg <= 1e-12 and dev_der <= 1e-12


def test_turbulence_192_fp32_vs_fp64(cg):
    import torch
    field, mu = synth.turbulence_field(SEED)
    kw = dict(mu=mu, prandtl=0.72, tau_mode=2, **box(N192))
    m64 = cg.Mesh(**kw)
    m64.init(field)
    s0 = torch.empty((m64.nf, m64.nv) + tuple(reversed(N192)), dtype=torch.float64, device="cuda")
    m64.get_state(out=s0)
    m32 = cg.Mesh(precision=1, **kw)
    m32.set_state(s0)
    steps = 10
    m64.step(steps)
    m32.step(steps)
    a, _ = m64.get_state()
    b, _ = m32.get_state()
    m64.close()
    m32.close()
    e = b[0, 0] - a[0, 0]
    l2 = math.sqrt(np.mean(e * e))

    def ke(st):
        return float(np.mean(0.5 * (st[0, 1:4] ** 2).sum(axis=0) / st[0, 0]))
    kerel = abs(ke(b) - ke(a)) / ke(a)
    print("turbulence 192^3, %d steps, FP32 vs FP64: density L2 %.2e, kinetic energy %.2e, mu %.3e" % (
        steps, l2, kerel, mu))
    assert l2 <= 1e-5 and kerel <= 1e-5


def test_turbulence_parity_small(orc, cg):
    """The same recipe on a 16^3 perturbed mesh: one step against the oracle."""
    field, mu = synth.turbulence_field(SEED, n=32)
    n = (16, 16, 16)
    kw = dict(mu=mu, prandtl=0.72, tau_mode=2, **box(n))
    o = orc.Oracle(**kw)
    o.init(field)
    m = cg.Mesh(**kw)
    m.set_state(o.get_state())
    o.step(1)
    m.step(1)
    assert class_scaled_diff(m.get_state()[0], o.get_state(), 0.7 * 2 * math.pi / 16) <= 1e-12
    m.close()
