"""Binding of libintpeaks.so: measured integer issue rates of the current GPU.

The search kernels of a build are integer arithmetic, so their roofline is
the rate at which the SMs retire integer instructions.  ``measure(kind)``
runs one instruction class of ``peaks/int_peaks.cu`` over a full grid and
returns its rate and the SM clock it ran at.  Measurement only: the build
does not use this library.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libintpeaks.so")

KINDS = {"imad": 0, "imad_wide": 1, "imad_hi": 2, "lop3": 3, "shf": 4, "imad+lop3": 5,
         "eval_lower1_l16": 6, "mul64": 7, "remix": 8}


class Result(ctypes.Structure):
    _fields_ = [("ops", ctypes.c_double), ("ms", ctypes.c_double), ("sm_mhz", ctypes.c_double),
                ("per_s", ctypes.c_double), ("blocks", ctypes.c_uint32), ("threads", ctypes.c_uint32)]


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2212_09562_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        L.ip_run.restype = ctypes.c_int
        L.ip_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.POINTER(Result)]
        _lib = L
    return _lib


def measure(kind: str, reps: int = 5, target_ms: float = 20.0) -> dict:
    """Rate of one instruction class (thread-level operations per second) on the
    current device, the best of ``reps`` launches of about ``target_ms``."""
    r = Result()
    rc = lib().ip_run(KINDS[kind], reps, target_ms, ctypes.byref(r))
    if rc != 0:
        raise RuntimeError(f"ip_run({kind}) failed ({rc})")
    return {"kind": kind, "per_s": r.per_s, "ms": r.ms, "sm_mhz": r.sm_mhz, "ops": r.ops,
            "grid": [r.blocks, r.threads]}
