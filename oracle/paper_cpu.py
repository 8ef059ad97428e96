"""ctypes wrapper around ``paper_cpu.c``: the paper's level loop on host
threads, a parallel CPU baseline (test and benchmark infrastructure only; not
the oracle, which is ``kd_oracle.c``).  Records as for ``oracle.py``: a 2-D
array of 4-byte items, int32 and uint32 arrays have int32 and uint32
coordinates."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "paper_cpu.c")
_LIB = os.path.join(_HERE, "_build", "libpaper_cpu.so")
_lock = threading.Lock()
_lib = None

INT32 = 0x100
UINT32 = 0x200


def compile_lib(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-pthread", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(compile_lib())
            i64, i32, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
            lib.pc_build.argtypes = [vp, i64, i32, i32, i32, i32, vp]
            lib.pc_build.restype = i32
            _lib = lib
    return _lib


def build(points: np.ndarray, k: int, mode: int = 0, threads: int = 0) -> np.ndarray:
    """Original index of the point at each node (threads = 0: one per core)."""
    pts = np.ascontiguousarray(points)
    if pts.ndim != 2 or pts.dtype.itemsize != 4:
        raise ValueError("records must be a 2-D array of 4-byte items")
    n, w = pts.shape
    orig = np.empty(n, dtype=np.int32)
    m = mode | {np.dtype(np.int32): INT32, np.dtype(np.uint32): UINT32}.get(pts.dtype, 0)
    rc = _load().pc_build(pts.ctypes.data, n, k, 4 * w, m, threads, orig.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"pc_build returned {rc}")
    return orig


def cores() -> int:
    return os.cpu_count() or 1
