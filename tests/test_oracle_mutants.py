"""Plants plausible mistakes in a copy of the oracle (on the CPU) and checks
that the pins catch every one: evidence that the pins are sharp enough to
trust the oracle."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from numtheory import load_golden, td_prime_mask, unpack_odd_bitmap

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "oracle.c")
PI = {int(x): int(v) for x, v in load_golden("pi_values.txt")}

# (name, text in oracle.c, replacement)
MUTANTS = [
    ("cross_from_p", "uint64_t start = p * p;", "uint64_t start = p;"),
    ("one_is_prime", "if (first_odd == 1) mark[0] = 1;", ""),
    ("step_p_not_2p", "m <= last; m += 2 * p)", "m <= last; m += p)"),
    ("even_start", "if ((m & 1) == 0) m += p;", ""),
    ("break_at_square", "if (p * p > last) break;", "if (p * p >= last) break;"),
    ("sqrt_of_hi", "oracle_isqrt(hi - 1)", "oracle_isqrt(hi) - 1"),
    ("two_inclusive", "uint64_t c = (lo <= 2 && 2 < hi) ? 1 : 0;", "uint64_t c = (lo <= 2 && 2 <= hi) ? 1 : 0;"),
    ("count_marked", "c += (mark[j] == 0);", "c += (mark[j] != 0);"),
    ("bit_index", "out[i >> 5] |= (uint32_t)1 << (i & 31);", "out[i >> 5] |= (uint32_t)1 << (i & 15);"),
    ("list_origin", "if (out && n < cap) out[n] = o0 + 2 * (j0 + j);", "if (out && n < cap) out[n] = o0 + 2 * j;"),
    ("isqrt_step", "r = (r >> 1) + bit;", "r = r + bit;"),
    ("base_sieve_from_2p", "for (uint64_t m = p * p; m <= limit; m += p)", "for (uint64_t m = 2 * p; m < limit; m += p)"),
    ("segment_stride", "sieve_odd_segment(job->o0 + 2 * j0, n", "sieve_odd_segment(job->o0 + j0, n"),
]


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-pthread", str(path), "-o", str(so)])
    lib = ctypes.CDLL(str(so))
    u64 = ctypes.c_uint64
    lib.oracle_count.argtypes = [u64, u64, ctypes.c_int]
    lib.oracle_count.restype = u64
    lib.oracle_bitmap.argtypes = [u64, u64, ctypes.POINTER(ctypes.c_uint32), u64]
    lib.oracle_bitmap.restype = u64
    lib.oracle_list.argtypes = [u64, u64, ctypes.POINTER(ctypes.c_uint64), u64]
    lib.oracle_list.restype = u64
    lib.oracle_isqrt.argtypes = [u64]
    lib.oracle_isqrt.restype = u64
    lib.oracle_base_primes.argtypes = [u64, ctypes.POINTER(ctypes.c_uint32), u64]
    lib.oracle_base_primes.restype = u64
    return lib


def _pins_pass(lib, td):
    """A quick subset of the oracle pins; False as soon as one fails."""
    for n in list(range(0, 3000)) + [2**32, 2**62, 2**64 - 1, 10**14 + 10**8]:
        r = lib.oracle_isqrt(n)
        if not (r * r <= n < (r + 1) * (r + 1)):
            return False
    for k in range(1, 8):
        if lib.oracle_count(0, 10**k, 2) != PI[10**k]:
            return False
    n = 10**5
    expect = np.nonzero(td[:n])[0].astype(np.uint64)
    out = np.zeros(len(expect) + 8, dtype=np.uint64)
    m = lib.oracle_list(0, n, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), len(out))
    if m != len(expect) or not np.array_equal(out[:m], expect):
        return False
    words = np.zeros((n // 2 + 31) // 32, dtype=np.uint32)
    lib.oracle_bitmap(0, n, words.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), len(words))
    if not np.array_equal(unpack_odd_bitmap(words, 0, n), expect[1:]):
        return False
    base = np.zeros(len(expect) + 8, dtype=np.uint32)
    m = lib.oracle_base_primes(n - 1, base.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), len(base))
    if m != len(expect) or not np.array_equal(base[:m].astype(np.uint64), expect):
        return False
    prefix = np.concatenate([[0], np.cumsum(td[:400])])
    for lo in range(0, 200):
        for hi in range(lo, 400, 7):
            if lib.oracle_count(lo, hi, 1) != prefix[hi] - prefix[lo]:
                return False
    # pi(10^7) single-threaded spans three oracle segments (2^21 odd integers each)
    if lib.oracle_count(0, 10**7, 1) != PI[10**7]:
        return False
    # the list over the same three segments: length, order and last element
    big = np.zeros(PI[10**7] + 8, dtype=np.uint64)
    m = lib.oracle_list(0, 10**7, big.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), len(big))
    if m != PI[10**7] or big[m - 1] != 9_999_991 or not np.all(np.diff(big[:m].astype(np.int64)) > 0):
        return False
    return True


@pytest.fixture(scope="module")
def td():
    return td_prime_mask(10**5 + 10)


def test_unmutated_copy_passes(tmp_path, td):
    lib = _build(tmp_path, "clean", "#include <stdint.h>", "#include <stdint.h>")
    assert _pins_pass(lib, td)


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, td, name, old, new):
    lib = _build(tmp_path, name, old, new)
    assert not _pins_pass(lib, td), f"planted mistake {name} was not caught by the pins"
