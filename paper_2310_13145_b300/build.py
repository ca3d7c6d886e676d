"""Builds the CUDA library in-tree for sm_103a (nvcc, no JIT cache)."""
from __future__ import annotations

import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "libucac.so")
# the index-checked build (UCAC_CHECK=1): every table-derived index of the
# sweep kernels is tested before use and a failure is reported by
# ucac_iterate instead of touching memory outside its buffer
SO_CHECK = os.path.join(HERE, "libucac_check.so")
SRC = os.path.join(HERE, "csrc", "ucac.cu")
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-shared"]


def _stale(so: str) -> bool:
    if not os.path.exists(so):
        return True
    deps = glob.glob(os.path.join(HERE, "csrc", "*")) + [os.path.join(HERE, "..", "include", "ucac.h")]
    t = os.path.getmtime(so)
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, check: bool = False) -> str:
    """Builds libucac.so, or with check=True the index-checked libucac_check.so."""
    so = SO_CHECK if check else SO
    if force or _stale(so):
        nvcc = os.environ.get("NVCC", "nvcc")
        tmp = so + ".tmp%d" % os.getpid()
        cmd = [nvcc] + NVCC_FLAGS + (["-DUCAC_CHECK=1"] if check else []) + \
            (["-Xptxas", "-v"] if verbose else []) + ["-o", tmp, SRC]
        subprocess.check_call(cmd)
        os.replace(tmp, so)
    return so


if __name__ == "__main__":
    print(build(force=True, verbose=True))
