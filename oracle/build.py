"""Compile the FP64 oracle (``tfs_oracle.cpp``) into ``oracle/_build/liboracle.so``.

Test infrastructure: see the package docstring.
"""
import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tfs_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_handle = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2, IEEE arithmetic, OpenMP). Returns the .so path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
           _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def load_library() -> ctypes.CDLL:
    global _handle
    with _lock:
        if _handle is None:
            _handle = ctypes.CDLL(build())
    return _handle
