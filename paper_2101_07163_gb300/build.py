"""Build the CUDA library liblbmice.so in-tree with nvcc for sm_103a (no torch extension)."""
from __future__ import annotations

import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "liblbmice.so")
LIB_CHECKED = os.path.join(HERE, "liblbmice_checked.so")  # -DLBMICE_CHECKED: bounds-checked
SOURCES = [os.path.join(HERE, "csrc", "lbmice.cu")]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-shared", "-Xptxas", "-v"]


def _deps():
    return (SOURCES + glob.glob(os.path.join(HERE, "csrc", "*.cuh"))
            + [os.path.join(ROOT, "include", "lbmice.h")])


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile liblbmice.so (checked: liblbmice_checked.so, every step-kernel index tested
    against its buffer) if it is missing or older than its sources; return its path."""
    lib = LIB_CHECKED if checked else LIB
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= max(os.path.getmtime(p) for p in _deps())):
        return lib
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = ([nvcc()] + NVCC_FLAGS + (["-DLBMICE_CHECKED"] if checked else [])
           + ["-o", tmp] + SOURCES)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + res.stdout + res.stderr)
    if verbose:
        print(res.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
