"""In-tree build of the CUDA library for sm_103a (nvcc only, no cmake)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
# translation units, compiled in parallel and linked into one library
SRCS = [os.path.join(CSRC, f) for f in ("cgks.cu", "cgks_stage_f64.cu", "cgks_stage_f32.cu", "cgks_stage_pair.cu",
                                        "cgks_stage_pair_curvi.cu", "cgks_recon_pair.cu", "cgks_batch.cu", "cgks_mlp.cu", "cgks_noalloc.cu")]
LIB = os.path.join(HERE, "libcgks.so")
DEPS = SRCS + [os.path.join(CSRC, f) for f in ("cgks_device.cuh", "cgks_pair.cuh", "cgks_kernels.cuh", "cgks_ctx.h",
                                               "cgks_stage.inc",
                                               "cgks_batch_kernels.cuh", "cgks_selector.cuh",
                                               "cgks_tables.h", "cgks_recon_gen.cuh")] + \
    [os.path.join(ROOT, "include", "cgks.h")]

NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-gencode", "arch=compute_103a,code=sm_103a",
              "-Xcompiler", "-fPIC", "--fmad=true"]


def nvcc():
    cand = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = os.path.join(cand, "bin", "nvcc")
    return p if os.path.exists(p) else "nvcc"


def build(force=False, verbose=False):
    """Compile libcgks.so next to this file; returns its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(d) for d in DEPS):
        return LIB
    tag = ".tmp%d" % os.getpid()
    objs, procs = [], []
    for src in SRCS:
        obj = os.path.join(CSRC, os.path.basename(src)[:-3] + tag + ".o")
        cmd = [nvcc()] + NVCC_FLAGS + ["-c", "-o", obj, src]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        objs.append(obj)
        procs.append(subprocess.Popen(cmd))
    failed = [p.wait() for p in procs]
    try:
        if any(failed):
            raise subprocess.CalledProcessError(max(failed), "nvcc")
        tmp = LIB + tag
        cmd = [nvcc(), "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp] + objs
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
