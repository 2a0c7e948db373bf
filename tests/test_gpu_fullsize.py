"""Parity at the full sizes the bench times, on sampled cells.

One S2O4 step of a cell depends only on the cells within Chebyshev distance
4 (stage 2 needs U* within 2, stage 1 reconstructs within 3 from data within
4).  So the oracle steps a 9^3 patch around each sampled cell, built from the
same analytic field and geometry, and the patch's centre must equal the
GPU's full-size result.  Both sides take the same fixed time step, derived
here from bounds of the analytic field (no input comes from the GPU)."""
import math

import numpy as np
import pytest

import synth
from parity import class_scaled_diff

pytestmark = pytest.mark.gpu
R = 4


@pytest.fixture(scope="module")
def cg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_08965_gb300 as p
    p.lib()
    return p


def patch_oracle(orc, n, lo, hi, nodes, cell, **kw):
    """oracle on the (2R+1)^3 patch of cells around `cell` (i, j, k)"""
    i, j, k = cell
    h = [(hi[a] - lo[a]) / n[a] for a in range(3)]
    plo = (lo[0] + (i - R) * h[0], lo[1] + (j - R) * h[1], lo[2] + (k - R) * h[2])
    phi = (plo[0] + (2 * R + 1) * h[0], plo[1] + (2 * R + 1) * h[1], plo[2] + (2 * R + 1) * h[2])
    pn = None
    if nodes is not None:
        pn = np.ascontiguousarray(nodes[k - R:k + R + 2, j - R:j + R + 2, i - R:i + R + 2])
    return orc.Oracle(3, (2 * R + 1,) * 3, lo=plo, hi=phi, nodes=pn, bc=[1] * 6, **kw)


def centre(s):
    return s[:, :, R:R + 1, R:R + 1, R:R + 1]


def cell_of(s, cell):
    i, j, k = cell
    return s[:, :, k:k + 1, j:j + 1, i:i + 1]


SAMPLES = [(37, 64, 90), (5, 100, 17), (120, 9, 61), (64, 64, 64)]


def tgv_class_magnitudes():
    """(density, momentum, energy) magnitudes of the TGV initial field: the
    scale floors of sampled cells (at a symmetry point the momentum of the
    sampled cell itself is O(h))"""
    x = np.linspace(0.0, 2 * math.pi, 33)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    rho, u, v, w, p = synth.taylor_green_3d(X, Y, Z)
    mom = rho * np.sqrt(u * u + v * v + w * w)
    rhoe = p / 0.4 + 0.5 * rho * (u * u + v * v + w * w)
    return (float(np.abs(rho).max()), float(mom.max()), float(np.abs(rhoe).max()))


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_tgv128_sampled_cells(orc, cg, precision):
    import torch
    n, lo, hi = (128,) * 3, (0.0,) * 3, (2 * math.pi,) * 3
    kw = dict(mu=1 / 1600, prandtl=0.72, tau_mode=2)
    # |U| <= 1 and c <= 10.02 for the Ma 0.1 field: the rate bound gives dt
    h = 2 * math.pi / 128
    dt = 0.5 / (3 * (1.0 + 10.02) / h)
    m = cg.Mesh(3, n, lo=lo, hi=hi, dt_fixed=dt, precision=precision, **kw)
    m.init(lambda x, y, z: synth.taylor_green_3d(x, y, z))
    m.step(1)
    st = torch.empty((m.nf, m.nv) + n, dtype=torch.float64, device="cuda")
    m.get_state(out=st)
    m.close()
    # FP32 form: every field, derivative fields included, within FP32's reach;
    # the paired form (FP32 pairs in the flux only) at the FP64 bar
    tol = 1e-5 if precision == 1 else 1e-12
    for cell in SAMPLES:
        o = patch_oracle(orc, n, lo, hi, None, cell, dt_fixed=dt, **kw)
        o.init(lambda x, y, z: synth.taylor_green_3d(x, y, z))
        o.step(1)
        i, j, k = cell
        g = st[:, :, k:k + 1, j:j + 1, i:i + 1].cpu().numpy()
        d = class_scaled_diff(g, centre(o.get_state()), h, tgv_class_magnitudes())
        print("TGV 128^3 precision %d cell %s: %.2e" % (precision, cell, d))
        assert d <= tol, cell


def test_turbulence192_perturbed_sampled_cells(orc, cg):
    import torch
    n, lo, hi = (192,) * 3, (0.0,) * 3, (2 * math.pi,) * 3
    nodes = synth.perturbed_nodes_3d(n)
    field, mu = synth.turbulence_field(20250811)
    kw = dict(mu=mu, prandtl=0.72, tau_mode=2)
    # |u| <= 2.5 (five times the rms Mach 0.5 of the field), c <= 1.2, h >= 0.7 h0
    h = 0.7 * 2 * math.pi / 192
    dt = 0.5 / (3 * (2.5 + 1.2) / h)
    m = cg.Mesh(3, n, lo=lo, hi=hi, nodes=nodes, dt_fixed=dt, **kw)
    m.init(field)
    m.step(1)
    st = torch.empty((m.nf, m.nv) + n, dtype=torch.float64, device="cuda")
    m.get_state(out=st)
    m.close()
    for cell in [(40, 150, 77), (180, 20, 100), (96, 96, 96)]:
        o = patch_oracle(orc, n, lo, hi, nodes, cell, dt_fixed=dt, **kw)
        o.init(field)
        o.step(1)
        i, j, k = cell
        g = st[:, :, k:k + 1, j:j + 1, i:i + 1].cpu().numpy()
        assert class_scaled_diff(g, centre(o.get_state()), h) <= 1e-12, cell


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_tgv256_sampled_cells(orc, cg, precision):
    """The largest configuration (TGV 256^3, ~150 GB of device memory in
    FP64), cells in the interior and next to the periodic wrap."""
    import torch
    torch.cuda.empty_cache()  # earlier tests' cached blocks: the library allocates with cudaMalloc
    n, lo, hi = (256,) * 3, (0.0,) * 3, (2 * math.pi,) * 3
    kw = dict(mu=1 / 1600, prandtl=0.72, tau_mode=2)
    h = 2 * math.pi / 256
    dt = 0.5 / (3 * (1.0 + 10.02) / h)
    m = cg.Mesh(3, n, lo=lo, hi=hi, dt_fixed=dt, precision=precision, **kw)
    m.init(lambda x, y, z: synth.taylor_green_3d(x, y, z))
    m.step(1)
    st = torch.empty((m.nf, m.nv) + n, dtype=torch.float64, device="cuda")
    m.get_state(out=st)
    m.close()
    tol = 1e-5 if precision == 1 else 1e-12
    for cell in [(0, 255, 128), (255, 0, 3), (77, 190, 250), (128, 128, 128)]:
        o = patch_oracle(orc, n, lo, hi, None, cell, dt_fixed=dt, **kw)
        o.init(lambda x, y, z: synth.taylor_green_3d(x, y, z))
        o.step(1)
        i, j, k = cell
        g = st[:, :, k:k + 1, j:j + 1, i:i + 1].cpu().numpy()
        d = class_scaled_diff(g, centre(o.get_state()), h, tgv_class_magnitudes())
        print("TGV 256^3 precision %d cell %s: %.2e" % (precision, cell, d))
        assert d <= tol, cell
    del st
    torch.cuda.empty_cache()
