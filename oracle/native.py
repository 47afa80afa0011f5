"""The oracle's C brute force (bruteforce.c): compiled with gcc and OpenMP
into oracle/_build/libbrute.so when missing or older than its source, loaded
with ctypes.  Test infrastructure only (see the package header)."""
from __future__ import annotations

import ctypes
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "bruteforce.c")
OUT = os.path.join(HERE, "_build", "libbrute.so")
CMD = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", OUT, SRC, "-lm"]

_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(OUT) or os.path.getmtime(OUT) < os.path.getmtime(SRC):
        os.makedirs(os.path.dirname(OUT), exist_ok=True)
        subprocess.run(CMD, check=True, capture_output=True, text=True)
    return OUT


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        p32, p64 = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
        _lib.oracle_brute_force.restype = ctypes.c_int
        _lib.oracle_brute_force.argtypes = [ctypes.c_int, ctypes.c_int, p32, p32, p64, p64, ctypes.c_double, p64,
                                            p64, ctypes.POINTER(ctypes.c_double)]
    return _lib
