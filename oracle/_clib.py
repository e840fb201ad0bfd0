"""Loader for the oracle's own C helpers (oracle/csrc), built with gcc.

Test infrastructure only (see the package docstring)."""
import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "oracle_geom.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_OUT = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared",
               "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            d = ctypes.c_double
            L.oracle_orient2d.argtypes = [d] * 6
            L.oracle_orient2d.restype = ctypes.c_int
            L.oracle_orient2d_exact.argtypes = [d] * 6
            L.oracle_orient2d_exact.restype = ctypes.c_int
            L.oracle_incircle.argtypes = [d] * 8
            L.oracle_incircle.restype = ctypes.c_int
            L.oracle_incircle_exact.argtypes = [d] * 8
            L.oracle_incircle_exact.restype = ctypes.c_int
            p = ctypes.c_void_p
            L.oracle_delaunay.argtypes = [ctypes.c_int, p, p, p, p]
            L.oracle_delaunay.restype = ctypes.c_int
            L.oracle_force_long.argtypes = [ctypes.c_int, p, p, p, p, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, p, p, ctypes.c_int]
            L.oracle_force_long.restype = None
            L.oracle_force_long_periodic.argtypes = [ctypes.c_int, p, p, p, p, ctypes.c_int,
                                                     ctypes.c_double, ctypes.c_int, ctypes.c_int, p, p,
                                                     ctypes.c_int]
            L.oracle_force_long_periodic.restype = None
            L.oracle_force_long_jvp.argtypes = [ctypes.c_int, p, p, p, p, ctypes.c_int, p, p, p, p,
                                                ctypes.c_int]
            L.oracle_force_long_jvp.restype = None
            L.oracle_force_long_dA.argtypes = [ctypes.c_int, p, p, p, p, ctypes.c_int]
            L.oracle_force_long_dA.restype = None
            L.oracle_has_openmp.restype = ctypes.c_int
            _lib = L
        return _lib
