"""Build the CUDA/C++ library in-tree with nvcc for sm_103a.

    python -m paper_2602_24155_gb300.build      (or call build())

Produces paper_2602_24155_gb300/libzeta.so.  Sources are compiled in
parallel (nvcc --threads) with one -gencode.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libzeta.so")
SOURCES = ["zeta_host.cpp", "zeta_policy.cpp", "zeta_learn.cpp", "zeta_capi.cpp", "zeta_kernels.cu", "zeta_mlp.cu",
           "zeta_selftest.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return [os.path.join(CSRC, s) for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def needs_build():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "zeta.h"))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force=False, verbose=False):
    if not force and not needs_build():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    if not os.path.isabs(nvcc):
        cand = "/usr/local/cuda/bin/nvcc"
        if os.path.exists(cand):
            nvcc = cand
    cmd = [nvcc, "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-lineinfo", "--threads", "0",
           *ARCH, "-I", os.path.join(os.path.dirname(HERE), "include"), "-o", LIB + ".tmp", *sources()]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv)
    print(LIB)
