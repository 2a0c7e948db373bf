"""The paired-FP32 type of the paired flux form, built for the host: its
two-sums are error-free, and sums, products, quotients and conversions
from double keep about 48 bits (relative errors below 2^-44 ~ 5.7e-14)."""
import ctypes as C
import hashlib
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pair_arith.cpp")
HDR = os.path.join(os.path.dirname(HERE), "paper_2508_08965_gb300", "csrc", "cgks_pair.cuh")


@pytest.fixture(scope="module")
def lib():
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no g++")
    h = hashlib.sha1()
    for p in (SRC, HDR):
        with open(p, "rb") as f:
            h.update(f.read())
    out = os.path.join(tempfile.gettempdir(), "cgks_pair_arith_%s.so" % h.hexdigest()[:16])
    if not os.path.exists(out):
        tmp = out + ".%d.tmp" % os.getpid()
        subprocess.run([cxx, "-std=c++17", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, SRC],
                       check=True, capture_output=True)
        os.replace(tmp, out)
    L = C.CDLL(out)
    L.pair_stats.argtypes = [C.c_int, C.c_uint, C.POINTER(C.c_double)]
    return L


@pytest.mark.parametrize("seed", [1, 2])
def test_pair_arithmetic(lib, seed):
    out = (C.c_double * 7)()
    lib.pair_stats(200000, seed, out)
    two_sum_fail, fast_fail, e_sum, e_diff, e_mul, e_div, e_cvt = list(out)
    assert two_sum_fail == 0 and fast_fail == 0
    bound = 2.0 ** -44
    assert e_cvt <= 2.0 ** -48
    assert e_sum <= bound and e_diff <= bound and e_mul <= bound and e_div <= bound, list(out)


@pytest.mark.parametrize("seed", [3, 4])
def test_pair_special_functions(lib, seed):
    """exp, expm1, erfc and 1/sqrt of the paired form in pair arithmetic,
    against long double references: within a few units of 2^-48."""
    lib.pair_func_stats.argtypes = [C.c_int, C.c_uint, C.POINTER(C.c_double)]
    out = (C.c_double * 5)()
    lib.pair_func_stats(100000, seed, out)
    e_exp, e_expm1, e_erfc, e_rsqrt, e_exp1 = list(out)
    print("exp %.2e expm1 %.2e erfc %.2e rsqrt %.2e exp[-1,1] %.2e" % tuple(out))
    assert e_exp1 <= 2.0 ** -46 and e_exp <= 2.0 ** -44
    assert e_expm1 <= 2.0 ** -45 and e_erfc <= 2.0 ** -45 and e_rsqrt <= 2.0 ** -46


@pytest.mark.parametrize("seed", [5, 6])
def test_pair_reconstruction_conversions(lib, seed):
    """The unnormalised pairs of the paired reconstruction: the integer-pipe
    split of a double keeps 47 bits (hi a truncation, never above |x|), the
    float -> double rebuild is exact for normal floats (subnormal ones give
    signed zeros), zeros and magnitudes below 2^-103 split to signed zeros, inf and NaN carry through, and 80-term sums of products
    (compensated, Sum2/Dot2 style) stay within 2^-42 of the sum of the
    products' magnitudes (measured about 14 units of 2^-48; the low part's
    own FP32 rounding grows with the number of terms, and a plain FP64 sum
    of 80 terms may err by up to 80 units of 2^-53)."""
    lib.pair_conv_stats.argtypes = [C.c_int, C.c_uint, C.POINTER(C.c_double)]
    out = (C.c_double * 5)()
    lib.pair_conv_stats(200000, seed, out)
    e_split, overshoot, f2d_bad, special_bad, e_dot = list(out)
    print("split %.2e dot %.2e" % (e_split, e_dot))
    assert e_split <= 2.0 ** -47 * (1 + 2.0 ** -20) and overshoot == 0 and f2d_bad == 0 and special_bad == 0
    assert e_dot <= 2.0 ** -42


def test_float_to_double_on_the_integer_pipe(lib):
    """The FP32 form's update converts its FP32 face sums to FP64 by bit
    operations (fp_f2d_exact) instead of the FP64 pipe's conversion: the
    result is the same double, bit for bit, for every float kind (normal,
    subnormal, zero, inf; NaN stays NaN)."""
    lib.f2d_exact_mismatches.argtypes = [C.c_int, C.c_uint]
    lib.f2d_exact_mismatches.restype = C.c_long
    assert lib.f2d_exact_mismatches(2000000, 11) == 0
