"""Primality tests written independently of the oracle, used only to pin it.

* Trial division (paper, Section 1): n >= 2 is prime iff no prime <= sqrt(n)
  divides it.
* Miller-Rabin (the improved test the paper names after the Fermat test of
  Section 3.2, Algorithm 3).  With the first twelve primes as bases the test
  is deterministic for every n < 3.18e23 (Sorenson and Webster, "Strong
  pseudoprimes to twelve prime bases", Math. Comp. 86, 2017), which covers all
  64-bit n.  The modular exponentiation is exponentiation by squaring
  (Algorithm 2), here Python's exact three-argument pow.
"""
from __future__ import annotations

import math
from typing import List

import numpy as np

MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def td_is_prime(n: int) -> bool:
    if n < 2:
        return False
    for d in range(2, math.isqrt(n) + 1):
        if n % d == 0:
            return False
    return True


def td_primes_upto(limit: int) -> List[int]:
    """Primes <= limit by trial division of every integer (slow, small limits)."""
    return [n for n in range(2, limit + 1) if td_is_prime(n)]


def td_prime_mask(n: int) -> np.ndarray:
    """Boolean array a[0..n): a[v] iff v is prime, by trial division with all
    primes <= sqrt(n - 1) (vectorised over v)."""
    v = np.arange(n, dtype=np.int64)
    mask = v >= 2
    for p in td_primes_upto(math.isqrt(max(n - 1, 0))):
        mask &= ~((v % p == 0) & (v != p))
    return mask


def mr_is_prime(n: int) -> bool:
    if n < 2:
        return False
    for p in MR_BASES:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in MR_BASES:
        x = pow(a, d, n)
        if x == 1 or x == n - 1:
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def unpack_odd_bitmap(words: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """Integers whose bit is set in an odd-only bitmap of [lo, hi)."""
    o0 = lo | 1
    nbits = max(0, (hi - o0 + 1) // 2)
    bits = np.unpackbits(np.asarray(words, dtype="<u4").view(np.uint8), bitorder="little")[:nbits]
    return o0 + 2 * np.nonzero(bits)[0].astype(np.uint64)


def load_golden(name: str) -> List[List[str]]:
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows
