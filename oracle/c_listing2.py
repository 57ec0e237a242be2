"""ctypes loader and build step for the plain-C Listing 2 oracle
(``spmv_listing2.c``).  Test infrastructure only (see ``oracle/__init__.py``).

``build()`` compiles the C file with gcc into ``oracle/_build/``; the flags
keep every product and sum separately rounded (``-ffp-contract=off``) and
contain nothing machine-specific, so the result is the same on x86-64 and
AArch64 hosts."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "spmv_listing2.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libspmv_listing2.so")

_lib = None


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", LIB + ".tmp", SRC]
        subprocess.run(cmd, check=True)
        os.replace(LIB + ".tmp", LIB)
    return LIB


def load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(LIB)
        P = ctypes.c_void_p
        for name in ("oracle_spmv_csr32_f64", "oracle_spmv_dacsr16_f64"):
            f = getattr(lib, name)
            f.restype = None
            f.argtypes = [ctypes.c_int32, P, P, P, P, P, ctypes.c_double, ctypes.c_double,
                          ctypes.c_int]
        lib.oracle_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def max_threads() -> int:
    return int(load().oracle_max_threads())


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def spmv_csr32(nrows, rowptr, col, val, x, y=None, alpha=1.0, beta=0.0, nthreads=1, out=None):
    lib = load()
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    if out is None:
        out = np.zeros(nrows) if y is None else np.array(y, dtype=np.float64)
    lib.oracle_spmv_csr32_f64(nrows, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(x), _ptr(out),
                              alpha, beta, int(nthreads))
    return out


def spmv_dacsr16(nrows, rowptr, off, val, x, y=None, alpha=1.0, beta=0.0, nthreads=1, out=None):
    lib = load()
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    off = np.ascontiguousarray(off, dtype=np.int16)
    val = np.ascontiguousarray(val, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    if out is None:
        out = np.zeros(nrows) if y is None else np.array(y, dtype=np.float64)
    lib.oracle_spmv_dacsr16_f64(nrows, _ptr(rowptr), _ptr(off), _ptr(val), _ptr(x), _ptr(out),
                                alpha, beta, int(nthreads))
    return out
