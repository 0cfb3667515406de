"""ctypes loader for the plain-C part of the oracle (oracle/oracle.c).

TEST INFRASTRUCTURE ONLY: see the package docstring.  The library is built
with gcc, -O2, OpenMP, and floating-point contraction switched off, so that
every product and sum is rounded exactly as written in the C source.
"""
import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force=False):
    """Compile oracle.c into liboracle.so next to it (atomic replace)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fcx-limited-range",
           "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(cmd, check=True, capture_output=True, text=True)
        os.replace(tmp, _LIB)
    finally:
        if os.path.exists(tmp):
            os.unlink(tmp)
    return _LIB


class Model(ctypes.Structure):
    """Parameters of the synthetic Eq. (1) Hamiltonian (energies in eV)."""
    _fields_ = [("band_gap", ctypes.c_double), ("w0", ctypes.c_double),
                ("x0", ctypes.c_double), ("jitter", ctypes.c_double),
                ("dispersion", ctypes.c_double), ("rank_x", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, u64, i32, dbl = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_int,
                              ctypes.c_double)
        L.or_splitmix64.argtypes = [u64]
        L.or_splitmix64.restype = u64
        L.or_uniform.argtypes = [u64, u64, u64]
        L.or_uniform.restype = dbl
        L.or_random_block.argtypes = [u64, u64, i64, i64, P, i64]
        L.or_random_block.restype = None
        L.or_bse_tables.argtypes = [u64, i32, i32, i32, ctypes.POINTER(Model),
                                    P, P, P]
        L.or_bse_tables.restype = None
        L.or_bse_build.argtypes = [u64, i32, i32, i32, ctypes.POINTER(Model),
                                   P, i64]
        L.or_bse_build.restype = None
        L.or_bse_elements.argtypes = [u64, i32, i32, i32, ctypes.POINTER(Model),
                                      i64, P, P, P]
        L.or_bse_elements.restype = None
        L.or_tridiag_eig.argtypes = [i32, P, P, P]
        L.or_tridiag_eig.restype = i32
        L.or_heev.argtypes = [i32, P, i64, P, P, i64, i32]
        L.or_heev.restype = i32
        L.or_cholesky.argtypes = [i32, P, i64]
        L.or_cholesky.restype = i32
        _lib = L
    return _lib


def ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def fortran(a, dtype):
    """A column-major (Fortran-ordered) copy of `a` with the given dtype."""
    return np.asfortranarray(np.asarray(a, dtype=dtype))
