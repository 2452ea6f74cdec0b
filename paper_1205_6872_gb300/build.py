"""Build libquapi.so in-tree: nvcc for sm_103a, one object per .cu, compiled in parallel.

What to rebuild is decided by content, not by file times: every object carries a
key (sha256 over the compiler command, the compiler's version line, the host
machine type, the .cu source and every header of the library), stored beside it
as ``<object>.buildkey``; the library's key covers its objects' keys and the link
command.  A fresh checkout, a copy whose file times were reset, or binaries made
on another host type are therefore always compiled from the committed sources.
"""

from __future__ import annotations

import hashlib
import os
import platform
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libquapi.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers():
    hs = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh")))
    hs.append(os.path.join(ROOT, "include", "quapi.h"))
    return hs


_TOOL_ID = None


def _tool_id():
    """nvcc's version line and the host machine type (part of every key)."""
    global _TOOL_ID
    if _TOOL_ID is None:
        try:
            v = subprocess.run([NVCC, "--version"], capture_output=True, text=True).stdout.strip().splitlines()
            v = v[-1] if v else ""
        except OSError:
            v = ""
        _TOOL_ID = f"{v}|{platform.machine()}"
    return _TOOL_ID


def _key(parts):
    h = hashlib.sha256()
    for p in parts:
        h.update(p if isinstance(p, bytes) else str(p).encode())
        h.update(b"\0")
    return h.hexdigest()


def _read(path):
    with open(path, "rb") as fh:
        return fh.read()


def _stored_key(path):
    try:
        with open(path + ".buildkey") as fh:
            return fh.read().strip()
    except OSError:
        return None


def _write_key(path, key):
    with open(path + ".buildkey", "w") as fh:
        fh.write(key + "\n")


def _compile(src, extra, header_bytes):
    obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")
    cmd = [NVCC] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
    key = _key([" ".join(cmd), _tool_id(), _read(src)] + header_bytes)
    if os.path.exists(obj) and _stored_key(obj) == key:
        return obj, key
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}")
    _write_key(obj, key)
    return obj, key


def build(verbose: bool = False, extra=()) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    srcs = sources()
    header_bytes = [_read(h) for h in _headers()]
    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        done = list(ex.map(lambda s: _compile(s, list(extra), header_bytes), srcs))
    objs = [o for o, _ in done]
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs
    lib_key = _key([" ".join([NVCC] + ARCH + ["-shared"]), _tool_id()] + [k for _, k in done])
    lib_key_path = os.path.join(OUT_DIR, "libquapi")
    if os.path.exists(LIB) and _stored_key(lib_key_path) == lib_key:
        return LIB
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc link failed")
    os.replace(tmp, LIB)
    _write_key(lib_key_path, lib_key)
    if verbose:
        print(f"built {LIB}")
    return LIB


if __name__ == "__main__":
    build(verbose=True)
