"""Builds libmphf.so (all CUDA kernels and the C ABI) in-tree for sm_103a.

    python -m paper_2212_09562_b300.build [--force]

nvcc cross-compiles without a GPU; the library lands next to this file so
that it travels with the source tree.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libmphf.so")
PEAKS_SRC = os.path.join(HERE, "peaks", "int_peaks.cu")
PEAKS_LIB = os.path.join(HERE, "libintpeaks.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
    deps.append(os.path.join(INCLUDE, "mphf.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build_peaks(force: bool = False, verbose: bool = False) -> str:
    """Compiles the integer issue-rate microbenchmark (libintpeaks.so, measurement only)."""
    if not force and os.path.exists(PEAKS_LIB) and os.path.getmtime(PEAKS_LIB) >= os.path.getmtime(PEAKS_SRC):
        return PEAKS_LIB
    tmp = PEAKS_LIB + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-O2,-Wall,-Wextra",
           "-shared", PEAKS_SRC, "-o", tmp]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.check_call(cmd)
    os.replace(tmp, PEAKS_LIB)
    return PEAKS_LIB


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None,
          out: str | None = None) -> str:
    """Compiles the library (to `out` instead of the package's libmphf.so if given)."""
    target = out or LIB
    if not force and out is None and not _stale():
        return LIB
    tmp = target + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-O2,-Wall,-Wextra",
           "-shared", f"-I{INCLUDE}", f"-I{CSRC}", *(extra or []), *sources(), "-o", tmp]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.check_call(cmd)
    os.replace(tmp, target)
    return target


if __name__ == "__main__":
    extra = [a for a in sys.argv[1:] if a.startswith("-X") or a.startswith("--ptxas")]
    build(force="--force" in sys.argv, verbose=True, extra=extra)
    build_peaks(force="--force" in sys.argv, verbose=True)
