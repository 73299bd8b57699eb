"""CPU oracle for the segmented sieve of Eratosthenes (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the product library never does.  It is
a thin ctypes wrapper over ``oracle.c``, a plain byte-per-odd-integer sieve
written from the paper's Section 3.1 (mark the multiples of each prime,
starting from 2) and Section 1 (primes <= sqrt(n) decide n).  The arithmetic
lives only in ``oracle.c``; this file marshals arguments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_FAIL = (1 << 64) - 1
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with gcc into ``liboracle.so`` next to it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        u64, u32p, u64p = ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64)
        lib.oracle_isqrt.argtypes = [u64]
        lib.oracle_isqrt.restype = u64
        lib.oracle_base_primes.argtypes = [u64, u32p, u64]
        lib.oracle_base_primes.restype = u64
        lib.oracle_count.argtypes = [u64, u64, ctypes.c_int]
        lib.oracle_count.restype = u64
        lib.oracle_bitmap.argtypes = [u64, u64, u32p, u64]
        lib.oracle_bitmap.restype = u64
        lib.oracle_list.argtypes = [u64, u64, u64p, u64]
        lib.oracle_list.restype = u64
        lib.oracle_crossings.argtypes = [u64, u64, u64, u64]
        lib.oracle_crossings.restype = u64
        lib.oracle_default_threads.argtypes = []
        lib.oracle_default_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _check(v: int) -> int:
    if v == _FAIL:
        raise ValueError("oracle call failed (bad range or out of memory)")
    return v


def isqrt(n: int) -> int:
    return int(_load().oracle_isqrt(n))


def default_threads() -> int:
    return int(_load().oracle_default_threads())


def base_primes(limit: int) -> np.ndarray:
    """All primes <= limit as uint32 (plain sieve of Eratosthenes)."""
    lib = _load()
    n = _check(lib.oracle_base_primes(limit, None, 0))
    out = np.zeros(max(n, 1), dtype=np.uint32)
    lib.oracle_base_primes(limit, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), n)
    return out[:n]


def count(lo: int, hi: int, threads: int = 0) -> int:
    """#primes in [lo, hi)."""
    return _check(int(_load().oracle_count(lo, hi, threads)))


def bitmap_words(lo: int, hi: int) -> int:
    o0 = lo | 1
    if o0 >= hi:
        return 0
    return ((hi - o0 + 1) // 2 + 31) // 32


def bitmap(lo: int, hi: int) -> np.ndarray:
    """Odd-only bitmap of [lo, hi) as uint32 words (bit i <-> (lo|1) + 2i)."""
    nw = bitmap_words(lo, hi)
    out = np.zeros(max(nw, 1), dtype=np.uint32)
    if nw:
        _check(_load().oracle_bitmap(lo, hi, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), nw))
    return out[:nw]


def primes(lo: int, hi: int) -> np.ndarray:
    """The primes in [lo, hi) ascending, as uint64 (2 included)."""
    lib = _load()
    n = _check(int(lib.oracle_list(lo, hi, None, 0)))
    out = np.zeros(max(n, 1), dtype=np.uint64)
    m = _check(int(lib.oracle_list(lo, hi, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), n)))
    assert m == n
    return out[:n]


def crossings(lo: int, hi: int, pmin: int = 23, wheel: int = 30) -> int:
    """Bit-clears of the crossing-off step on a wheel of modulus `wheel`: the
    pairs (p, m), p prime >= pmin, m >= p, gcd(m, wheel) = 1, lo <= p m < hi."""
    return _check(int(_load().oracle_crossings(lo, hi, pmin, wheel)))
