"""CPU oracle for exact string matching (test infrastructure).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference leg of ``bench.py`` may import this package.  The
CUDA library never calls it and shares no code with it.

The oracle computes the set of all occurrences of p in t as defined in the
problem statement of Section 1 (every start position i in [0, n-m] with
t[i..i+m-1] = p, increasing, overlaps included).  ``oracle.c`` holds the
routines; this module compiles it with gcc and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_u64p = ctypes.POINTER(ctypes.c_uint64)
_u8p = ctypes.c_void_p


def compile_oracle(src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile ``src`` into a shared library at ``out`` (gcc -O2)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                    "-o", tmp, src], check=True)
    os.replace(tmp, out)
    return out


def build() -> str:
    """Build the oracle library if missing or older than its source."""
    with _lock:
        if (not os.path.exists(_LIB_PATH)
                or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
            compile_oracle()
    return _LIB_PATH


def _bind(lib):
    for name in ("oracle_naive", "oracle_kmp"):
        f = getattr(lib, name)
        f.restype = ctypes.c_uint64
        f.argtypes = [_u8p, ctypes.c_uint64, _u8p, ctypes.c_uint64, _u64p, ctypes.c_uint64]
    lib.oracle_naive_mt.restype = ctypes.c_uint64
    lib.oracle_naive_mt.argtypes = [_u8p, ctypes.c_uint64, _u8p, ctypes.c_uint64, _u64p,
                                    ctypes.c_uint64, ctypes.c_int]
    lib.oracle_binary_masks.restype = ctypes.c_int
    lib.oracle_binary_masks.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_uint32)]
    return lib


def load(path: str | None = None):
    """Load (building first if needed) and return the ctypes library."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _as_u8(x) -> np.ndarray:
    if isinstance(x, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(x), dtype=np.uint8)
    a = np.ascontiguousarray(x)
    if a.dtype != np.uint8:
        raise TypeError("oracle inputs are byte strings or uint8 arrays")
    return a


def _run(fn, text, pattern, *extra, lib=None):
    lib = lib or load()
    t = _as_u8(text)
    p = _as_u8(pattern)
    if len(p) == 0:
        raise ValueError("m = 0 is outside the problem statement")
    f = getattr(lib, fn)
    tp = t.ctypes.data if len(t) else None
    pp = p.ctypes.data
    cnt = f(tp, len(t), pp, len(p), None, 0, *extra)
    if cnt == 2**64 - 1:
        raise MemoryError(fn)
    out = np.empty(max(int(cnt), 1), dtype=np.uint64)
    cnt2 = f(tp, len(t), pp, len(p), out.ctypes.data_as(_u64p), int(cnt), *extra)
    assert cnt2 == cnt
    return out[: int(cnt)]


def naive(text, pattern, lib=None) -> np.ndarray:
    """All occurrences by the definition (sorted uint64 start positions)."""
    return _run("oracle_naive", text, pattern, lib=lib)


def kmp(text, pattern, lib=None) -> np.ndarray:
    """All occurrences by Knuth-Morris-Pratt (sorted uint64 positions)."""
    return _run("oracle_kmp", text, pattern, lib=lib)


def naive_mt(text, pattern, threads: int | None = None, lib=None) -> np.ndarray:
    """``naive`` split over host threads by start position."""
    threads = threads or os.cpu_count() or 1
    return _run("oracle_naive_mt", text, pattern, int(threads), lib=lib)


def count_mt(text, pattern, threads: int | None = None, lib=None) -> int:
    """|H| only, by the threaded naive routine."""
    lib = lib or load()
    t = _as_u8(text)
    p = _as_u8(pattern)
    if len(p) == 0:
        raise ValueError("m = 0 is outside the problem statement")
    threads = threads or os.cpu_count() or 1
    return int(lib.oracle_naive_mt(t.ctypes.data if len(t) else None, len(t), p.ctypes.data,
                                   len(p), None, 0, int(threads)))


def binary_masks(n: int, m: int, which: str = "naive", lib=None) -> np.ndarray:
    """Hit bitmasks for every binary (text, pattern) pair of lengths n, m."""
    lib = lib or load()
    out = np.zeros((1 << n) * (1 << m), dtype=np.uint32)
    rc = lib.oracle_binary_masks(n, m, 0 if which == "naive" else 1,
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    if rc != 0:
        raise ValueError((n, m))
    return out.reshape(1 << n, 1 << m)
