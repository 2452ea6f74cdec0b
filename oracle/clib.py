"""Build and load the oracle's plain-C loops (quapi_oracle.c).  Test infrastructure only."""

from __future__ import annotations

import ctypes
import hashlib
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "quapi_oracle.c")
_LIB = os.path.join(_HERE, "libquapi_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile quapi_oracle.c with gcc (-O2, OpenMP) into oracle/libquapi_oracle.so.

    Rebuilt whenever the source, the command or the host machine type differ from the
    key stored beside the library (libquapi_oracle.so.buildkey), never by file times."""
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    h = hashlib.sha256()
    with open(_SRC, "rb") as fh:
        h.update(fh.read())
    h.update(" ".join(cmd[:6]).encode() + b"|" + platform.machine().encode())
    key = h.hexdigest()
    try:
        with open(_LIB + ".buildkey") as fh:
            stored = fh.read().strip()
    except OSError:
        stored = None
    if not force and os.path.exists(_LIB) and stored == key:
        return _LIB
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    with open(_LIB + ".buildkey", "w") as fh:
        fh.write(key + "\n")
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            for name in ("oracle_grow", "oracle_step", "oracle_readout"):
                fn = getattr(L, name)
                fn.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
                fn.restype = None
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.complex128 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def call(name: str, M2: int, n: int, A: np.ndarray, G: np.ndarray, g: np.ndarray, out: np.ndarray):
    A = np.ascontiguousarray(A, dtype=np.complex128)
    G = np.ascontiguousarray(G, dtype=np.complex128)
    g = np.ascontiguousarray(g, dtype=np.complex128)
    getattr(lib(), name)(M2, n, _ptr(A), _ptr(G), _ptr(g), _ptr(out))
    return out


def set_threads(n: int) -> None:
    """Threads for the oracle's OpenMP loops from now on (the OpenMP runtime's own setting)."""
    lib()
    gomp = ctypes.CDLL("libgomp.so.1")
    gomp.omp_set_num_threads.argtypes = [ctypes.c_int]
    gomp.omp_set_num_threads(int(max(1, n)))
