"""Builds and loads the oracle's plain C helpers (TEST INFRASTRUCTURE ONLY).

The product library never imports this module.  The shared object is compiled
with the system C compiler into ``oracle/_build/`` on first use, or ahead of
time by ``build()``.
"""
import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "search.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle_search.so")
_lock = threading.Lock()
_handle = None


def build(force=False):
    """Compile search.c (gcc -O2, OpenMP when available).  Returns the .so path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:2] + ["-fopenmp"] + base[2:], check=True,
                       stdout=subprocess.PIPE, stderr=subprocess.PIPE)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _handle
    with _lock:
        if _handle is None:
            h = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            h.oracle_partition_search.argtypes = [dp, dp, ctypes.c_double, ctypes.c_int,
                                                  ctypes.c_int, ip, dp, dp]
            h.oracle_partition_search.restype = ctypes.c_int
            h.oracle_tuple_error.argtypes = [dp, dp, ctypes.c_double, ctypes.c_int,
                                             ctypes.c_int, ip, dp, dp]
            h.oracle_tuple_error.restype = ctypes.c_int
            _handle = h
    return _handle
