"""Build and load the oracle's C part (rb_oracle.c) with gcc.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Compiled with
-ffp-contract=off so that x86 and Arm builds round identically.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rb_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "librb_oracle.so")
_lock = threading.Lock()
_lib = None


class OrcGeom(ctypes.Structure):
    _fields_ = [
        ("n_elem", ctypes.c_int32),
        ("ring_radius", ctypes.c_double),
        ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32),
        ("h", ctypes.c_double),
        ("n_rays", ctypes.c_int32),
        ("ds", ctypes.c_double),
        ("max_steps", ctypes.c_int32),
        ("support_margin", ctypes.c_double),
        ("c_ref", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile rb_oracle.c into oracle/_build/librb_oracle.so (if stale)."""
    with _lock:
        os.makedirs(_OUT_DIR, exist_ok=True)
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC",
                   "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        L.orc_trace_fan.argtypes = [ctypes.POINTER(OrcGeom), P, ctypes.c_int, P, P]
        L.orc_trace_fan.restype = ctypes.c_int
        L.orc_trace_endpoints.argtypes = [ctypes.POINTER(OrcGeom), P, P, P, P]
        L.orc_trace_endpoints.restype = ctypes.c_int
        L.orc_grid.argtypes = [ctypes.POINTER(OrcGeom), P, ctypes.c_int64, P]
        L.orc_grid.restype = ctypes.c_int
        L.orc_grid_pixels.argtypes = [ctypes.POINTER(OrcGeom), P, ctypes.c_int64, P, ctypes.c_int64, P]
        L.orc_grid_pixels.restype = ctypes.c_int
        _lib = L
    return _lib
