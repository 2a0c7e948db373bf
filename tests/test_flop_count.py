"""The algorithmic operation counts behind the bench's roofline, recounted
from the kernels' source (tests/flop_count.cpp: the device routines built
for the host with a value-numbering compute type), not GPU.

The bench divides these counts, times the units of a launch, by the
launch's CUDA-event time: the figures must be those of the code as it
stands, so this test fails when the arithmetic of a kernel changes until
the bench's table is updated."""
import ctypes as C
import hashlib
import math
import os
import shutil
import subprocess
import sys
import tempfile

import numpy as np
import pytest

import synth

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2508_08965_gb300", "csrc")
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def fc():
    from test_host_parity import _cuda_include
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("no g++ or CUDA headers for the host build")
    h = hashlib.sha1()
    srcs = [os.path.join(HERE, "flop_count.cpp"), os.path.join(HERE, "host_kernels.cpp")]
    for p in srcs + sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))):
        with open(p, "rb") as f:
            h.update(f.read())
    out = os.path.join(tempfile.gettempdir(), "cgks_flop_count_%s.so" % h.hexdigest()[:16])
    if not os.path.exists(out):
        tmp = out + ".%d.tmp" % os.getpid()
        subprocess.run([cxx, "-std=c++17", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-I" + inc,
                        "-D__host__=", "-D__device__=", "-D__forceinline__=", "-D__noinline__=", "-o", tmp,
                        srcs[0]], check=True, capture_output=True)
        os.replace(tmp, out)
    lib = C.CDLL(out)
    dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
    lib.count_stage_ops.argtypes = [C.c_int, ip, dp, dp, dp, dp, C.c_double, C.c_long, dp]
    return lib


def per_unit(fc, orc, dim, n, fn, kw, phys, stride):
    lo, hi = (0.0,) * dim, (2 * math.pi,) * dim
    o = orc.Oracle(dim, n, lo=lo, hi=hi, **kw)
    o.init(fn)
    s = np.ascontiguousarray(o.get_state())
    nn = np.array(list(n) + [1] * (3 - dim), dtype=np.int32)
    lo3 = np.array(list(lo) + [0.0] * (3 - dim))
    hi3 = np.array(list(hi) + [1.0] * (3 - dim))
    ph = np.array(phys, dtype=np.float64)
    out = np.zeros(18)
    d = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    assert fc.count_stage_ops(dim, nn.ctypes.data_as(C.POINTER(C.c_int)), d(lo3), d(hi3), d(ph), d(s), o.dt(), stride,
                              d(out)) == 0
    res = {}
    for k, name in enumerate(("recon", "flux", "update")):
        add, mul, fma, div, sfu = out[5 * k:5 * k + 5] / out[15 + k]
        res[name] = dict(flops=add + mul + 2 * fma + div, div=div, sfu=sfu)
    return res


def _field3(x, y, z):
    return synth.random_smooth_3d(x, y, z, 2001)


def _field2(x, y):
    r = synth.random_smooth_3d(x, y, 0.37 + 0 * x, 2001)
    return [r[0], r[1], r[2], r[4]]


VISC = dict(mu=1 / 1600, prandtl=0.72, tau_mode=2)


@pytest.mark.parametrize("dim,viscous", [(3, True), (2, True), (2, False)])
def test_flux_counts_match_the_bench_table(fc, orc, dim, viscous):
    import bench
    n = (4, 4, 4) if dim == 3 else (8, 8)
    kw = VISC if viscous else {}
    phys = [1.4, kw.get("mu", 0.0), kw.get("prandtl", 1.0), 0.5, 100.0, kw.get("tau_mode", 0), 0, 0]
    r = per_unit(fc, orc, dim, n, _field3 if dim == 3 else _field2, kw, phys, 7 if dim == 3 else 3)
    f = r["flux"]
    print("flux %d-D %s: %.1f flops, %.2f divisions, %.2f special functions per Gauss point"
          % (dim, "viscous" if viscous else "tau = 0", f["flops"], f["div"], f["sfu"]))
    assert f["flops"] == bench.ALG_FLOPS_PER_UNIT[("flux", dim, viscous)]


def test_reconstruction_count(fc, orc):
    """printed for the record: the FP64 work of a cell that the FP32 screen
    does not certify (the random field is under-resolved on 4^3, so every
    cell takes the full GENO path)"""
    r = per_unit(fc, orc, 3, (4, 4, 4), _field3, VISC, [1.4, 1 / 1600, 0.72, 0.5, 100.0, 2, 0, 0], 7)
    print("reconstruction 3-D, full GENO path: %.0f flops per cell" % r["recon"]["flops"])
    assert 5e3 < r["recon"]["flops"] < 2e4
