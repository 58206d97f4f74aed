"""Fused multiply-add for the oracle (test infrastructure only).

numpy has no fused multiply-add, so the one primitive the oracle takes from
C is IEEE 754-2008 fusedMultiplyAdd: fma(a, b, c) = a * b + c computed
exactly and rounded once (C99 ``fma``, `oracle/fmath.c`).  The shared library
is compiled with gcc on first use into ``oracle/_build/`` (or by
``__graft_entry__.build()``).  Pinned against exact rational arithmetic in
``tests/test_oracle_detmath_rng.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmath.c")
_OUT = os.path.join(_HERE, "_build", "liboracle_fmath.so")
_lib = None
_lock = threading.Lock()


def build() -> str:
    """Compile fmath.c unless the library is newer than the source; return its path."""
    if os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = f"{_OUT}.{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                    "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            p = ctypes.POINTER(ctypes.c_double)
            lib.oracle_fma.argtypes = [p, p, p, p, ctypes.c_int64]
            lib.oracle_fma.restype = None
            _lib = lib
    return _lib


def fma(a, b, c):
    """Elementwise a * b + c with one rounding (numpy broadcasting)."""
    lib = _load()
    a, b, c = np.broadcast_arrays(np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64),
                                  np.asarray(c, dtype=np.float64))
    a, b, c = (np.ascontiguousarray(v) for v in (a, b, c))
    out = np.empty(a.shape, dtype=np.float64)
    if out.size:
        p = ctypes.POINTER(ctypes.c_double)
        lib.oracle_fma(a.ctypes.data_as(p), b.ctypes.data_as(p), c.ctypes.data_as(p), out.ctypes.data_as(p),
                       out.size)
    return out
