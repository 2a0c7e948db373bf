"""In-tree build of the CUDA library for sm_103a (nvcc only, no cmake)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc", "cgks.cu")
SRC_NOALLOC = os.path.join(HERE, "csrc", "cgks_noalloc.cu")
LIB = os.path.join(HERE, "libcgks.so")
DEPS = [os.path.join(HERE, "csrc", f) for f in ("cgks.cu", "cgks_noalloc.cu", "cgks_device.cuh", "cgks_kernels.cuh",
                                                "cgks_tables.h", "cgks_recon_gen.cuh")] + \
    [os.path.join(ROOT, "include", "cgks.h")]

NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-gencode", "arch=compute_103a,code=sm_103a",
              "-Xcompiler", "-fPIC", "-shared", "--fmad=true"]


def nvcc():
    cand = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = os.path.join(cand, "bin", "nvcc")
    return p if os.path.exists(p) else "nvcc"


def build(force=False, verbose=False):
    """Compile libcgks.so next to this file; returns its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(d) for d in DEPS):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc()] + NVCC_FLAGS + ["-o", tmp, SRC, SRC_NOALLOC]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
