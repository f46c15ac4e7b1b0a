"""Builds and loads the oracle's plain C helpers (TEST INFRASTRUCTURE ONLY).

The product library never imports this module.  The shared objects are
compiled with the system C compiler into ``oracle/_build/`` on first use, or
ahead of time by ``build()``:

* search.c - the exhaustive partition search of the fit (Sec. 4.2)
* conv.c   - the filter's result definition on all host cores (FP64 separable
             direct convolution) and the running-sum method on the CPU (timing
             context for the benchmark)
"""
import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_OUT_DIR = os.path.join(_HERE, "_build")
_LIBS = {"search": ("search.c", "liboracle_search.so"), "conv": ("conv.c", "liboracle_conv.so")}
_lock = threading.Lock()
_handles = {}


def _build_one(name, force=False):
    src, so = _LIBS[name]
    src = os.path.join(_HERE, src)
    lib = os.path.join(_OUT_DIR, so)
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(src):
        return lib
    tmp = lib + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", src, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:2] + ["-fopenmp"] + base[2:], check=True,
                       stdout=subprocess.PIPE, stderr=subprocess.PIPE)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(tmp, lib)
    return lib


def build(force=False):
    """Compile every helper (gcc -O2, OpenMP when available).  Returns the .so paths."""
    return [_build_one(n, force) for n in sorted(_LIBS)]


def lib():
    """The partition-search helper."""
    with _lock:
        if "search" not in _handles:
            h = ctypes.CDLL(_build_one("search"))
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            h.oracle_partition_search.argtypes = [dp, dp, ctypes.c_double, ctypes.c_int,
                                                  ctypes.c_int, ip, dp, dp]
            h.oracle_partition_search.restype = ctypes.c_int
            h.oracle_tuple_error.argtypes = [dp, dp, ctypes.c_double, ctypes.c_int,
                                             ctypes.c_int, ip, dp, dp]
            h.oracle_tuple_error.restype = ctypes.c_int
            _handles["search"] = h
        return _handles["search"]


def conv_lib():
    """The convolution helper (all host cores)."""
    with _lock:
        if "conv" not in _handles:
            h = ctypes.CDLL(_build_one("conv"))
            dp = ctypes.POINTER(ctypes.c_double)
            fp = ctypes.POINTER(ctypes.c_float)
            ip = ctypes.POINTER(ctypes.c_int)
            h.oracle_threads.argtypes = []
            h.oracle_threads.restype = ctypes.c_int
            h.oracle_conv_separable.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, dp,
                                                ctypes.c_int, ctypes.c_int, dp]
            h.oracle_conv_separable.restype = ctypes.c_int
            h.oracle_boxsum_u8_f32.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ip,
                                               fp, ctypes.c_int, ctypes.c_int, fp]
            h.oracle_boxsum_u8_f32.restype = ctypes.c_int
            _handles["conv"] = h
        return _handles["conv"]
