"""Pins for the oracle's count of the crossing-off work (the bit-clears of a
wheel sieve, Section 3.1's marking of multiples restricted to a wheel), which
is the numerator of the count kernel's roofline.  Checked against two
formulations that share nothing with it: a literal double loop over (p, m),
and a loop over the integers n that counts, for each, its prime factors p
with p^2 <= n and a cofactor coprime to the wheel.  Planted mistakes in a copy
of the oracle must each fail one of these.  CPU only."""
import ctypes
import math
import os
import subprocess

import pytest

import oracle
from numtheory import load_golden, td_is_prime

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "oracle.c")


def double_loop(lo, hi, pmin, w):
    """Every prime p with p^2 < hi, every m >= p: count p m in [lo, hi) with gcd(m, w) = 1."""
    n = 0
    for p in range(2, math.isqrt(max(hi - 1, 0)) + 1):
        if p < pmin or not td_is_prime(p):
            continue
        m = p
        while p * m < hi:
            if p * m >= lo and math.gcd(m, w) == 1:
                n += 1
            m += 1
    return n


def by_factors(lo, hi, pmin, w):
    """Sum over n in [lo, hi) of #{p prime : p | n, p >= pmin, p^2 <= n, gcd(n / p, w) = 1}."""
    total = 0
    for n in range(max(lo, 2), hi):
        x, d, factors = n, 2, set()
        while d * d <= x:
            while x % d == 0:
                factors.add(d)
                x //= d
            d += 1
        if x > 1:
            factors.add(x)
        total += sum(1 for p in factors if p >= pmin and p * p <= n and math.gcd(n // p, w) == 1)
    return total


CASES = [(0, 3000, 23, 30), (0, 3000, 7, 30), (0, 3000, 2, 1), (0, 3000, 11, 210), (500, 2600, 23, 30),
         (961, 962, 2, 1), (960, 1000, 23, 30), (0, 529, 23, 30), (0, 530, 23, 30), (1, 2, 2, 1),
         (5, 5, 2, 1), (12_345, 17_000, 61, 30), (12_345, 17_000, 23, 210), (0, 10_000, 3, 2)]


@pytest.mark.parametrize("lo,hi,pmin,w", CASES)
def test_crossings_equal_double_loop_and_factor_count(lo, hi, pmin, w):
    want = double_loop(lo, hi, pmin, w)
    assert by_factors(lo, hi, pmin, w) == want
    assert oracle.crossings(lo, hi, pmin, w) == want


def test_crossings_every_small_range():
    # all 0 <= lo <= hi <= 400 against the per-integer factor count (prefix sums)
    for pmin, w in ((2, 1), (7, 30), (23, 30)):
        per_n = [by_factors(n, n + 1, pmin, w) for n in range(401)]
        prefix = [0]
        for v in per_n:
            prefix.append(prefix[-1] + v)
        for lo in range(0, 401, 7):
            for hi in range(lo, 401, 3):
                assert oracle.crossings(lo, hi, pmin, w) == prefix[hi] - prefix[lo], (lo, hi, pmin, w)


def test_crossings_plain_sieve_marks_each_composite_once_per_small_factor():
    # with no wheel and pmin = 2 every composite n < N is cleared once per prime
    # factor p with p^2 <= n; so the number of distinct integers cleared is the
    # number of composites below N, which pi(N) fixes
    pi = {int(x): int(v) for x, v in load_golden("pi_values.txt")}
    N = 10**4
    distinct = sum(1 for n in range(4, N) if by_factors(n, n + 1, 2, 1) > 0)
    assert distinct == N - 2 - pi[N]
    assert oracle.crossings(0, N, 2, 1) >= distinct


def test_crossings_additive_and_rejects_bad_input():
    a, m, b = 10**9, 10**9 + 123_457, 10**9 + 10**6
    for pmin, w in ((23, 30), (61, 30), (23, 210)):
        assert oracle.crossings(a, m, pmin, w) + oracle.crossings(m, b, pmin, w) == oracle.crossings(a, b, pmin, w)
    with pytest.raises(ValueError):
        oracle.crossings(10, 5, 23, 30)
    with pytest.raises(ValueError):
        oracle.crossings(0, 10, 23, 0)


def test_crossings_golden_file_matches_the_oracle():
    # the stored values (written by tests/golden/make_crossings.py from the oracle)
    # are what the oracle still computes
    for lo, hi, pmin, w, v in load_golden("crossings.txt"):
        lo, hi, pmin, w, v = (int(x) for x in (lo, hi, pmin, w, v))
        if hi - lo <= 10**13:
            assert oracle.crossings(lo, hi, pmin, w) == v, (lo, hi, pmin, w)


# (name, text in oracle.c, replacement): plausible mistakes in oracle_crossings
MUTANTS = [
    ("start_at_lo_not_p2", "if (m_lo < p) m_lo = p;", ""),
    ("start_at_2p", "if (m_lo < p) m_lo = p;", "if (m_lo < 2) m_lo = 2;"),
    ("hi_inclusive", "uint64_t m_hi = (hi - 1) / p + 1;", "uint64_t m_hi = hi / p + 1;"),
    ("lo_floor", "uint64_t m_lo = (lo + p - 1) / p;", "uint64_t m_lo = lo / p;"),
    ("no_gcd", "n += (gcd_u64(m, w) == 1);", "n += 1;"),
    ("phi_odd_only", "phi += (gcd_u64(m, w) == 1);", "phi += (m & 1);"),
    ("pmin_exclusive", "if (p < pmin) continue;", "if (p <= pmin) continue;"),
    ("sqrt_bound", "uint64_t lim = oracle_isqrt(hi - 1);", "uint64_t lim = oracle_isqrt(hi) - 1;"),
    ("runs_floor", "uint64_t runs = (b - a) / w;", "uint64_t runs = (b - a + w - 1) / w;"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_crossing_mistakes_are_caught(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-pthread", str(path), "-o", str(so)])
    lib = ctypes.CDLL(str(so))
    u64 = ctypes.c_uint64
    lib.oracle_crossings.argtypes = [u64, u64, u64, u64]
    lib.oracle_crossings.restype = u64
    caught = False
    for lo, hi, pmin, w in CASES:
        if int(lib.oracle_crossings(lo, hi, pmin, w)) != double_loop(lo, hi, pmin, w):
            caught = True
            break
    assert caught, name
