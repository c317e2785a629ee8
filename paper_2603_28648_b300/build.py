"""Build libqcdmrg.so in-tree for sm_103a with nvcc."""

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = ["csrc/core.cpp", "csrc/rules.cpp", "csrc/rules_su2.cpp", "csrc/su2.cpp", "csrc/init.cpp", "csrc/engine.cpp", "csrc/tiled.cpp", "csrc/capi.cpp", "csrc/orbitals.cpp", "csrc/su2expand.cpp", "csrc/entanglement.cpp", "csrc/configs.cpp", "csrc/kernels.cu", "csrc/tc_gemm.cu", "csrc/noalloc.cu", "csrc/graph.cu", "csrc/tc_tiled.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def build(verbose=False):
    out = os.path.join(HERE, "libqcdmrg.so")
    cmd = (["nvcc", "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-pthread", "-shared"] + ARCH +
           ["-Xptxas", "-v" if verbose else "-O3"] + [os.path.join(HERE, s) for s in SRC] +
           ["-o", out, "-lcudart", "-lcusolver"])
    subprocess.run(cmd, check=True, cwd=HERE)
    return out


if __name__ == "__main__":
    print(build(verbose=True))
