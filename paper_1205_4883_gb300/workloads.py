"""Seeded synthetic inputs for the sieve: ranges, interval batches, request streams.

This module holds no sieve arithmetic.  It only turns a seed into integer
ranges, so that the CUDA path and the CPU oracle can be fed the same inputs.
Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written here from its
published definition.  Log-uniform values are computed with ``decimal`` at
fixed precision so that x86 and Arm hosts draw bit-identical integers.
"""
from __future__ import annotations

import decimal
import math
from dataclasses import dataclass
from typing import List, Tuple

_MASK = (1 << 64) - 1

# The paper's workloads are "disorder integers of scale n" split into blocks
# (Section 3.1); the named workloads below are the single-range, batched and
# served configurations measured by bench.py and the tests.
PI_1E7 = (0, 10**7)          # plain sieve, count + bitmap + u32 list
PI_1E12 = (0, 10**12)        # count only
RANGE_2P32 = (0, 1 << 32)    # odd-only bitmap + u32 list


class SplitMix64:
    """SplitMix64: a 64-bit counter advanced by the golden-ratio increment,
    then finalised by two xor-shift-multiply rounds."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform in [0, 1) with 53 random bits (exact in binary64)."""
        return (self.next() >> 11) * (2.0 ** -53)


def _pow10_floor(exponent: decimal.Decimal) -> int:
    with decimal.localcontext() as ctx:
        ctx.prec = 60
        v = decimal.Decimal(10) ** exponent
        return int(v.to_integral_value(rounding=decimal.ROUND_FLOOR))


def log_uniform_int(rng: SplitMix64, e_lo: int, e_hi: int) -> int:
    """floor(10 ** (e_lo + (e_hi - e_lo) * u)), u uniform in [0, 1)."""
    u = decimal.Decimal(rng.uniform())  # exact conversion of a binary64
    with decimal.localcontext() as ctx:
        ctx.prec = 60
        e = decimal.Decimal(e_lo) + decimal.Decimal(e_hi - e_lo) * u
    return _pow10_floor(e)


def batch_intervals(m: int = 4096, seed: int = 1205, lo_exp: Tuple[int, int] = (6, 14),
                    w_exp: Tuple[int, int] = (3, 8)) -> Tuple[List[int], List[int]]:
    """m intervals [lo_i, lo_i + w_i): lo_i log-uniform in [10^lo_exp[0], 10^lo_exp[1]),
    w_i log-uniform in [10^w_exp[0], 10^w_exp[1]).  Draw order per interval: lo, then w."""
    rng = SplitMix64(seed)
    los, his = [], []
    for _ in range(m):
        lo = log_uniform_int(rng, *lo_exp)
        w = log_uniform_int(rng, *w_exp)
        los.append(lo)
        his.append(lo + w)
    return los, his


@dataclass
class Request:
    arrival_s: float   # offset from the start of the stream
    lo: int
    hi: int
    kind: str          # "count" or "list"


def served_stream(rate: float, n: int, seed: int = 1205, list_frac: float = 0.2,
                  lo_exp: Tuple[int, int] = (0, 12), w_exp: Tuple[int, int] = (4, 9)) -> List[Request]:
    """A Poisson stream of n sieve requests at `rate` requests/s.

    Per request the draws are: inter-arrival gap (exponential), kind (list with
    probability list_frac), start offset lo = floor(10^(12 u)) - 1 clamped at 0,
    width w log-uniform in [10^w_exp[0], 10^w_exp[1])."""
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    for _ in range(n):
        t += -math.log(1.0 - rng.uniform()) / rate
        kind = "list" if rng.uniform() < list_frac else "count"
        lo = max(0, log_uniform_int(rng, *lo_exp) - 1)
        w = log_uniform_int(rng, *w_exp)
        out.append(Request(t, lo, lo + w, kind))
    return out


def rank_block(rank: int, units: int = PI_1E12[1]) -> Tuple[int, int]:
    """The block of integers rank `rank` sieves when several GPUs run the
    single-range workload side by side: [rank units, (rank + 1) units)
    (independent ranges, no exchange between ranks; weak scaling)."""
    return rank * units, (rank + 1) * units


def random_ranges(count: int, seed: int, max_lo: int, max_w: int) -> List[Tuple[int, int]]:
    """`count` ranges [lo, lo + w) with lo uniform in [0, max_lo] and w uniform in [0, max_w]."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        lo = rng.next() % (max_lo + 1)
        w = rng.next() % (max_w + 1)
        out.append((lo, lo + w))
    return out
