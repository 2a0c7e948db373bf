"""The library's kernels built for the host (tests/host_kernels.cpp: the
same device routines run one work item at a time) against the oracle, on
small meshes, without a GPU.  The bar is the GPU's: class-scaled 1e-12
after one FP64 step (1e-5 for the FP32 form), selector features bit for
bit.  It checks the kernels' arithmetic; their parallel execution is the
GPU tests' part."""
import ctypes as C
import hashlib
import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import synth
from parity import class_scaled_diff

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2508_08965_gb300", "csrc")
SRC = os.path.join(HERE, "host_kernels.cpp")


def _cuda_include():
    for base in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if base and os.path.exists(os.path.join(base, "include", "cuda_bf16.h")):
            return os.path.join(base, "include")
    return None


@pytest.fixture(scope="module")
def hk():
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("no g++ or CUDA headers for the host build")
    h = hashlib.sha1()
    for p in [SRC] + sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))):
        with open(p, "rb") as f:
            h.update(f.read())
    out = os.path.join(tempfile.gettempdir(), "cgks_host_kernels_%s.so" % h.hexdigest()[:16])
    if not os.path.exists(out):
        tmp = out + ".%d.tmp" % os.getpid()
        subprocess.run([cxx, "-std=c++17", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-I" + inc,
                        "-D__host__=", "-D__device__=", "-D__forceinline__=", "-D__noinline__=", "-o", tmp, SRC],
                       check=True, capture_output=True)
        os.replace(tmp, out)
    lib = C.CDLL(out)
    dp, ip, fp = C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_float)
    lib.host_set_bc.argtypes = [ip, dp]
    lib.host_run.argtypes = [C.c_int, C.c_int, ip, dp, dp, dp, dp, dp, C.c_int, dp]
    lib.host_features.argtypes = [C.c_int, ip, dp, dp, dp, C.c_int, fp]
    lib.host_gp_perm_check.argtypes = [C.c_int, C.c_uint]
    lib.host_gp_perm_check.restype = C.c_double
    return lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def run_pair(orc, hk, dim, n, fn, steps, precision=0, lo=None, hi=None, nodes=None, bc=None, bc_state=None, **kw):
    """one oracle run and one host-kernel run from the oracle's initial state"""
    lo = lo or (0.0,) * dim
    hi = hi or (1.0,) * dim
    o = orc.Oracle(dim, n, lo=lo, hi=hi, nodes=nodes, bc=bc, bc_state=bc_state, **kw)
    o.init(fn)
    U = np.ascontiguousarray(o.get_state(), dtype=np.float64).copy()
    bcs = np.zeros(30)
    for f, st in enumerate(bc_state or []):
        if st is not None:
            bcs[5 * f:5 * f + len(st)] = st
    hk.host_set_bc((C.c_int * 6)(*(list(bc or []) + [0] * (6 - len(bc or [])))), _dp(bcs))
    phys = np.array([kw.get("gamma", 1.4), kw.get("mu", 0.0), kw.get("prandtl", 1.0), kw.get("cfl", 0.5),
                     kw.get("c_chi", 100.0), kw.get("tau_mode", 0), int(kw.get("linear", False)),
                     kw.get("dt_fixed", 0.0)])
    nn = (C.c_int * 3)(*(list(n) + [1] * (3 - dim)))
    lo3 = np.array(list(lo) + [0.0] * (3 - dim), dtype=np.float64)
    hi3 = np.array(list(hi) + [1.0] * (3 - dim), dtype=np.float64)
    nd = None if nodes is None else _dp(np.ascontiguousarray(nodes, dtype=np.float64))
    dt = C.c_double(0)
    rc = hk.host_run(dim, precision, nn, _dp(lo3), _dp(hi3), nd, _dp(phys), _dp(U), steps, C.byref(dt))
    assert rc == 0
    o.step(steps)
    return U, o.get_state()


def s2(x, y):
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * x + 0.3) * np.cos(2 * np.pi * y)
    u = 0.3 * np.sin(np.pi * x) + 0.1 * np.cos(2 * np.pi * y + 0.7) * x
    v = 0.2 * np.cos(2 * np.pi * y) + 0.1 * x
    p = 1.0 + 0.1 * np.cos(2 * np.pi * x - 0.4)
    return [rho, u, v, p]


def s3(x, y, z):
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * x + 0.3) * np.cos(2 * np.pi * y) + 0.1 * z
    u = 0.2 * np.cos(2 * np.pi * y) + 0.1 * z
    v = 0.2 * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * z + 0.2)
    w = 0.3 * np.sin(np.pi * z) * (1.0 + 0.2 * np.cos(2 * np.pi * x))
    p = 1.0 + 0.1 * np.cos(2 * np.pi * z - 0.4) + 0.05 * np.sin(2 * np.pi * y)
    return [rho, u, v, w, p]


VISC = dict(mu=2e-3, prandtl=0.72, tau_mode=2)
CASES = [
    ("vortex-periodic-2d", dict(dim=2, n=(16, 12), lo=(0, 0), hi=(10, 10)),
     lambda x, y: synth.isentropic_vortex_2d(x, y)),
    ("walls-viscous-2d", dict(dim=2, n=(12, 10), bc=[3, 3, 1, 1], **VISC), s2),
    ("slip-shock-2d", dict(dim=2, n=(12, 10), bc=[1, 1, 3, 2], tau_mode=1), s2),
    ("shock-vortex-inflow", dict(dim=2, n=(24, 12), lo=(0, 0), hi=(2, 1), bc=[4, 1, 2, 2], tau_mode=1,
                                 bc_state=[synth.shock_vortex_inflow(2.0)]),
     lambda x, y: synth.shock_vortex_2d(x, y, 2.0, 3.0, rc=0.15)),
    ("walls-3d", dict(dim=3, n=(6, 5, 7), bc=[3, 3, 2, 2, 1, 1], **VISC), s3),
    ("inflow-3d", dict(dim=3, n=(6, 5, 7), bc=[4, 1, 2, 3, 0, 0], bc_state=[
        [1.2, 2.4, 0.12, -0.24, 1.0 / 0.4 + 0.6 * (4 + 0.01 + 0.04)]], **VISC), s3),
]


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_host_kernels_one_step(orc, hk, case, precision):
    """precision 2: FP64 with the interface flux solved in paired FP32, held
    to the FP64 bar"""
    name, kw, fn = case
    kw = dict(kw)
    dim, n = kw.pop("dim"), kw.pop("n")
    U, so = run_pair(orc, hk, dim, n, fn, 1, precision=precision, **kw)
    lo, hi = kw.get("lo", (0.0,) * dim), kw.get("hi", (1.0,) * dim)
    h = min((hi[a] - lo[a]) / n[a] for a in range(dim))
    d = class_scaled_diff(U.reshape(so.shape), so, h)
    assert d <= (1e-5 if precision == 1 else 1e-12), d


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_host_kernels_curvilinear_tgv(orc, hk, precision):
    n = (6, 6, 6)
    nodes = synth.perturbed_nodes_3d(n)
    U, so = run_pair(orc, hk, 3, n, lambda x, y, z: synth.taylor_green_3d(x, y, z), 2, precision=precision,
                     lo=(0, 0, 0), hi=(2 * math.pi,) * 3, nodes=nodes, bc=[1, 1, 0, 0, 1, 1], mu=1 / 1600,
                     prandtl=0.72, tau_mode=2)
    d = class_scaled_diff(U.reshape(so.shape), so, 0.7 * 2 * math.pi / 6)
    assert d <= (1e-5 if precision == 1 else 1e-12), d


@pytest.mark.parametrize("precision", [0, 2])
def test_host_kernels_many_steps(orc, hk, precision):
    """the 100-step bar of the GPU parity, on a 2-D wall box"""
    U, so = run_pair(orc, hk, 2, (12, 10), s2, 100, precision=precision, bc=[2, 2, 0, 0])
    assert class_scaled_diff(U.reshape(so.shape), so, 0.1) <= 1e-9


def test_host_paired_flux_tgv(orc, hk):
    """the paired form on the Taylor-Green vortex (Ma 0.1, Re 1600): one step
    of 16^3 and ten of 10^3 at the FP64 bar"""
    for n, steps in (((16, 16, 16), 1), ((10, 10, 10), 10)):
        U, so = run_pair(orc, hk, 3, n, lambda x, y, z: synth.taylor_green_3d(x, y, z), steps, precision=2,
                         lo=(0, 0, 0), hi=(2 * math.pi,) * 3, mu=1 / 1600, prandtl=0.72, tau_mode=2)
        assert class_scaled_diff(U.reshape(so.shape), so, 2 * math.pi / n[0]) <= 1e-12


@pytest.mark.parametrize("precision", [0, 1])
def test_host_selector_features_bit_exact(orc, hk, precision):
    kw = dict(dim=2, n=(24, 20), lo=(0, 0), hi=(1, 1), bc=[1, 1, 1, 1], tau_mode=1)
    o = orc.Oracle(**kw)
    o.init(lambda x, y: synth.riemann4_2d(x, y, synth.riemann4_params(9)))
    fo = o.selector_features()
    U = np.ascontiguousarray(o.get_state(), dtype=np.float64)
    hk.host_set_bc((C.c_int * 6)(1, 1, 1, 1, 0, 0), _dp(np.zeros(30)))
    out = np.zeros((o.ncell, 16), dtype=np.float32)
    hk.host_features(2, (C.c_int * 3)(24, 20, 1), _dp(np.zeros(3)), _dp(np.ones(3)), _dp(U), precision,
                     out.ctypes.data_as(C.POINTER(C.c_float)))
    assert np.array_equal(out, fo)


@pytest.mark.parametrize("dim", [2, 3])
def test_gauss_point_transform_axis_symmetry(hk, dim):
    """The face Gauss-point transform of axis ax equals the axis-0 transform
    of the coefficients relabelled by the permutation pi of the coordinates
    (pi(0) = ax, tangential axes in order; gen_perm), with the axis-0
    derivative j read as the physical derivative pi(j): the reference cell
    and the basis (all monomials of degree 1..4) are symmetric under
    relabelling.  The paired reconstruction evaluates all three axes this
    way through one copy of the axis-0 code."""
    worst = max(hk.host_gp_perm_check(dim, seed) for seed in (1, 2, 3))
    assert worst <= 1e-14, worst
