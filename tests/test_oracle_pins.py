"""Pins for the CPU oracle: checks against facts fixed by mathematics, not by
the oracle itself (trial division, closed values of pi(x), Miller-Rabin,
invariants).  CPU only."""
import numpy as np
import pytest

import oracle
from numtheory import (load_golden, mr_is_prime, td_is_prime, td_prime_mask,
                       unpack_odd_bitmap)

PI = {int(x): int(v) for x, v in load_golden("pi_values.txt")}
FACTS = {k: int(v) for k, v in load_golden("prime_facts.txt")}


@pytest.fixture(scope="module")
def td_1e6():
    return td_prime_mask(10**6)


def test_isqrt_exact():
    for n in list(range(0, 5000)) + [2**32 - 1, 2**32, 2**62, 2**64 - 1, 10**14 + 10**8,
                                     (2**31 - 1) ** 2, (2**31 - 1) ** 2 - 1]:
        r = oracle.isqrt(n)
        assert r * r <= n < (r + 1) * (r + 1), n


def test_trial_division_every_n_below_1e6(td_1e6):
    # Section 1: primality by divisibility by primes <= sqrt(n), for every n < 10^6.
    expect = np.nonzero(td_1e6)[0].astype(np.uint64)
    assert np.array_equal(oracle.primes(0, 10**6), expect)
    assert np.array_equal(unpack_odd_bitmap(oracle.bitmap(0, 10**6), 0, 10**6), expect[1:])
    assert oracle.count(0, 10**6) == len(expect)
    assert np.array_equal(oracle.base_primes(10**6 - 1).astype(np.uint64), expect)


def test_trial_division_windows(td_1e6):
    # Ranges starting mid-way, with odd and even ends, several segments long.
    prefix = np.concatenate([[0], np.cumsum(td_1e6)])
    for lo, hi in [(1, 999_999), (2, 3), (3, 4), (524_287, 999_983), (999_000, 10**6),
                   (17, 17), (101, 100_003), (4_194_303 // 8, 10**6)]:
        got = oracle.primes(lo, hi)
        assert np.array_equal(got, np.nonzero(td_1e6[lo:hi])[0].astype(np.uint64) + lo)
        assert oracle.count(lo, hi, 3) == prefix[hi] - prefix[lo]


def test_all_small_ranges_brute_force():
    # Every 0 <= lo <= hi <= 2000 against trial division.
    mask = np.array([td_is_prime(n) for n in range(2001)])
    prefix = np.concatenate([[0], np.cumsum(mask)])
    for lo in range(0, 2001):
        for hi in range(lo, 2001):
            assert oracle.count(lo, hi, 1) == prefix[hi] - prefix[lo], (lo, hi)


def test_small_range_lists_and_bitmaps():
    mask = np.array([td_is_prime(n) for n in range(700)])
    for lo in range(0, 260):
        for hi in range(lo, lo + 130):
            expect = np.nonzero(mask[lo:hi])[0] + lo
            assert np.array_equal(oracle.primes(lo, hi), expect.astype(np.uint64))
            words = oracle.bitmap(lo, hi)
            assert len(words) == oracle.bitmap_words(lo, hi)
            assert np.array_equal(unpack_odd_bitmap(words, lo, hi), expect[expect != 2].astype(np.uint64))
            # bits past the range in the last word are zero
            o0 = lo | 1
            nbits = max(0, (hi - o0 + 1) // 2)
            if nbits % 32:
                assert int(words[-1]) >> (nbits % 32) == 0


@pytest.mark.parametrize("x", [10**k for k in range(1, 11)] + [2**32])
def test_pi_closed_values(x):
    assert oracle.count(0, x) == PI[x]


@pytest.mark.slow
@pytest.mark.parametrize("x", [10**11, 10**12])
def test_pi_closed_values_slow(x):
    assert oracle.count(0, x) == PI[x]


def test_prime_facts():
    p = oracle.primes(10**7 - 100, 10**7 + 100)
    assert p[p < 10**7][-1] == FACTS["largest_prime_below_1e7"]
    assert p[p > 10**7][0] == FACTS["smallest_prime_above_1e7"]
    assert oracle.primes(2**32 - 100, 2**32)[-1] == FACTS["largest_prime_below_2p32"]
    assert oracle.primes(10**12 - 100, 10**12)[-1] == FACTS["largest_prime_below_1e12"]
    assert oracle.primes(10**12, 10**12 + 100)[0] == FACTS["smallest_prime_above_1e12"]
    assert oracle.primes(10**14, 10**14 + 100)[0] == FACTS["smallest_prime_above_1e14"]
    # the oracle's base-prime count at sqrt(10^12) is pi(10^6)
    assert len(oracle.base_primes(10**6)) == PI[10**6]


def test_list_across_oracle_segments():
    # [0, 10^7) spans three of the oracle's segments of 2^21 odd integers.
    lst = oracle.primes(0, 10**7)
    assert len(lst) == PI[10**7]
    assert lst[-1] == FACTS["largest_prime_below_1e7"]
    assert np.all(np.diff(lst.astype(np.int64)) > 0)
    rng = np.random.default_rng(3)
    for v in rng.choice(lst, 2000):
        assert mr_is_prime(int(v))
    # and far from 0: every odd gap interior fails Miller-Rabin
    lo, hi = 10**12, 10**12 + 4_500_000
    lst = [int(v) for v in oracle.primes(lo, hi)]
    assert len(lst) == oracle.count(lo, hi)
    for a, b in zip(lst[::97], lst[1::97]):
        assert mr_is_prime(a)
        assert not any(mr_is_prime(n) for n in range(a + 2, b, 2))


def test_mr_matches_trial_division(td_1e6):
    # The Miller-Rabin used below is itself pinned to trial division first.
    for n in range(0, 200_000):
        assert mr_is_prime(n) == bool(td_1e6[n]), n
    # strong pseudoprimes to small base sets and Carmichael numbers are composite
    for n in (561, 1105, 1729, 2047, 3215031751, 2152302898747, 3474749660383,
              341550071728321, 3825123056546413051):
        assert not mr_is_prime(n)


@pytest.mark.parametrize("lo,w", [(10**12 - 20_000, 40_000), (10**14, 30_000),
                                  (2**32 - 15_000, 30_000), (10**13 + 12345, 20_000)])
def test_large_lo_against_miller_rabin(lo, w):
    hi = lo + w
    got = [int(v) for v in oracle.primes(lo, hi)]
    expect = [n for n in range(lo, hi) if mr_is_prime(n)]
    assert got == expect
    assert oracle.count(lo, hi) == len(expect)


def test_invariants_random_ranges():
    from paper_1205_4883_gb300.workloads import random_ranges
    for lo, hi in random_ranges(40, seed=7, max_lo=10**9, max_w=3 * 10**6):
        c = oracle.count(lo, hi)
        words = oracle.bitmap(lo, hi)
        pop = int(np.unpackbits(words.view(np.uint8)).sum()) if len(words) else 0
        assert pop + (1 if lo <= 2 < hi else 0) == c
        lst = oracle.primes(lo, hi)
        assert len(lst) == c
        assert np.all(np.diff(lst.astype(np.int64)) > 0)
        mid = (lo + hi) // 2
        assert oracle.count(lo, mid) + oracle.count(mid, hi) == c
        # every listed odd value has its bit set
        assert np.array_equal(unpack_odd_bitmap(words, lo, hi), lst[lst != 2])


def test_special_cases():
    assert oracle.count(0, 0) == 0
    assert oracle.count(0, 1) == 0
    assert oracle.count(0, 2) == 0
    assert oracle.count(0, 3) == 1
    assert oracle.count(1, 2) == 0
    assert oracle.count(2, 3) == 1
    assert oracle.count(3, 3) == 0
    assert oracle.count(4, 5) == 0
    assert oracle.count(10**12, 10**12) == 0
    assert list(oracle.primes(0, 30)) == [2, 3, 5, 7, 11, 13, 17, 19, 23, 29]
    assert oracle.bitmap_words(4, 5) == 0
    with pytest.raises(ValueError):
        oracle.count(5, 4)


def test_threads_do_not_change_result():
    lo, hi = 123_456_789, 123_456_789 + 50_000_000
    ref = oracle.count(lo, hi, 1)
    for t in (2, 3, 7, 16):
        assert oracle.count(lo, hi, t) == ref
