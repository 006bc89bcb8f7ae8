"""ctypes loader for the oracle's C primitives (oracle/ckks_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the GPU library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ckks_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libckks_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C file with gcc (-O2, OpenMP over limbs)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            I = ctypes.c_int
            U64 = ctypes.c_uint64
            L.orc_ntt.argtypes = [P, I, I, P, P]
            L.orc_intt.argtypes = [P, I, I, P, P]
            for f in (L.orc_mul, L.orc_add, L.orc_sub, L.orc_mul_const):
                f.argtypes = [P, P, P, I, I, P]
            L.orc_bconv.argtypes = [P, I, P, P, I, I, P]
            L.orc_auto_coeff.argtypes = [P, P, I, I, U64, P]
            L.orc_auto_ntt.argtypes = [P, P, I, I, U64]
            L.orc_bitrev.argtypes = [ctypes.c_uint32, I]
            L.orc_bitrev.restype = ctypes.c_uint32
            L.orc_mulmod.argtypes = [U64, U64, U64]
            L.orc_mulmod.restype = U64
            L.orc_powmod.argtypes = [U64, U64, U64]
            L.orc_powmod.restype = U64
            _lib = L
    return _lib


def ptr(a: np.ndarray) -> int:
    assert a.flags.c_contiguous and a.dtype == np.uint64, (a.dtype, a.flags)
    return a.ctypes.data


def u64arr(vals) -> np.ndarray:
    return np.ascontiguousarray(np.array([int(v) for v in vals], dtype=np.uint64))
