"""Builds libgfmom.so (the C-ABI library) in-tree with nvcc for sm_103a.

One nvcc invocation per translation unit, run in parallel, then one link.
Host code is compiled without floating-point contraction so the table
sample placement rounds identically on x86-64 and aarch64.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgfmom.so")
SOURCES = ["gf_host.cpp", "gf_batch.cpp", "gf_fill.cu", "gf_regular.cu", "gf_mfie.cu", "gf_adjoint.cu", "gf_sparse_kernels.cu",
           "gf_batch_kernels.cu", "gf_noalloc.cu", "gf_rcs.cu", "gf_sparse.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
# The regular-pair kernels flush FP32 subnormals: their distances, Green
# values and moments stay far above 2^-126 for any mesh the lattice serves,
# and the flush drops the subnormal handling around rsqrt and sincospi.
EXTRA_FLAGS = {"gf_regular.cu": ["-ftz=true"]}


def _deps():
    out = [os.path.join(CSRC, s) for s in os.listdir(CSRC)]
    out.append(os.path.join(INCLUDE, "gfmom.h"))
    return out


def needs_build():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in _deps())


def _compile(src):
    obj = os.path.join(OUT_DIR, os.path.basename(src) + ".o")
    cmd = [NVCC, "-c", "-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-ffp-contract=off",
           "-I", INCLUDE, "-I", CSRC, "-o", obj, os.path.join(CSRC, src)]
    if src.endswith(".cu"):
        cmd[4:4] = ["-Xptxas", "-v"] if os.environ.get("GF_PTXAS_VERBOSE") else []
    cmd[4:4] = EXTRA_FLAGS.get(src, [])
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(force=False, verbose=False):
    if not force and not needs_build():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        results = list(ex.map(_compile, SOURCES))
    if verbose:
        for _, err in results:
            if err:
                print(err, file=sys.stderr)
    objs = [o for o, _ in results]
    tmp = LIB + ".tmp"
    cmd = [NVCC, "-shared", *ARCH, "-o", tmp, *objs, "-lcudart", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
