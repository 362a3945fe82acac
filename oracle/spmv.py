"""CSR SpMV of the oracle's assembled SIPG matrix, timed on the host cores.

TEST INFRASTRUCTURE (see ``oracle/__init__``): the CPU baseline of the 8^3-cell
apply times y = A x with the matrix of ``sipg.assemble`` (Sec. 2, Eq. (2)),
once through SciPy (one core) and once through ``spmv_omp.c`` (plain C,
OpenMP over rows, all host cores). Both compute the plain definition
y_r = sum_p A[r, p] x[p]; ``tests/test_oracle_spmv.py`` pins the C routine
against the dense product of the same matrix.

The C library is compiled by ``build()`` below (gcc, -fopenmp) into
``oracle/libspmv_omp.so``; if it cannot be built or loaded, ``csr_spmv_omp``
raises.
"""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "spmv_omp.c")
LIB = os.path.join(HERE, "libspmv_omp.so")


def build():
    """Compile spmv_omp.c (returns the library path; raises on failure)."""
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", SRC, "-o", LIB]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"gcc failed for {SRC}:\n{r.stdout}\n{r.stderr}")
    return LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_csr_spmv.restype = None
        lib.oracle_csr_spmv.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        lib.oracle_csr_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def csr_arrays(A):
    """The CSR arrays of a scipy matrix in the C routine's types (int64 row pointers, int32 columns)."""
    A = A.tocsr()
    return (np.ascontiguousarray(A.indptr, dtype=np.int64), np.ascontiguousarray(A.indices, dtype=np.int32),
            np.ascontiguousarray(A.data, dtype=np.float64))


def csr_spmv_omp(arrays, x, threads=0):
    """y = A x with the C/OpenMP routine; threads = 0 keeps the OpenMP default."""
    lib = _load()
    indptr, indices, data = arrays
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(len(indptr) - 1, dtype=np.float64)
    lib.oracle_csr_spmv(len(y), indptr.ctypes.data, indices.ctypes.data, data.ctypes.data, x.ctypes.data,
                        y.ctypes.data, int(threads))
    return y


def omp_threads():
    """Threads the OpenMP runtime uses by default."""
    return int(_load().oracle_csr_threads())
