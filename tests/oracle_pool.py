"""The CPU oracle over many host threads, for the full-size parity tests.

oracle's ctypes calls release the GIL, so a thread pool runs them on every
core.  A range is cut into windows that tile it exactly; window k of an
odd-only bitmap starts at o0 + 64 w_k (o0 = lo | 1), so its own bitmap is
words [w_k, w_{k+1}) of the whole one.  Only the oracle is called here.
"""
from __future__ import annotations

from concurrent.futures import ThreadPoolExecutor
from typing import Callable, Iterable, List, Sequence, Tuple

import numpy as np

import oracle


def threads() -> int:
    return max(1, oracle.default_threads())


def pmap(fn: Callable, items: Iterable):
    with ThreadPoolExecutor(threads()) as ex:
        return list(ex.map(fn, items))


def counts(los: Sequence[int], his: Sequence[int]) -> List[int]:
    """oracle.count of every interval, one thread each."""
    return pmap(lambda lh: oracle.count(lh[0], lh[1], 1), list(zip(los, his)))


def bitmap_windows(lo: int, hi: int, window_words: int = 1 << 20) -> List[Tuple[int, int, int]]:
    """(first word, sub-range lo, sub-range hi) of windows tiling the bitmap of [lo, hi)."""
    o0 = lo | 1
    nw = oracle.bitmap_words(lo, hi)
    out = []
    for w0 in range(0, nw, window_words):
        a = o0 + 64 * w0
        b = min(hi, o0 + 64 * (w0 + window_words))
        out.append((w0, a, b))
    return out


def compare_bitmap(words: np.ndarray, lo: int, hi: int, window_words: int = 1 << 20) -> List[int]:
    """Indices of the first words of windows where `words` differs from the oracle's bitmap."""
    assert len(words) == oracle.bitmap_words(lo, hi)

    def check(win):
        w0, a, b = win
        ref = oracle.bitmap(a, b)
        return None if np.array_equal(words[w0:w0 + len(ref)], ref) else w0

    return [w for w in pmap(check, bitmap_windows(lo, hi, window_words)) if w is not None]


def compare_list(values: np.ndarray, lo: int, hi: int, window: int = 1 << 26) -> Tuple[int, List[int]]:
    """Compare an ascending prime list of [lo, hi) with the oracle window by
    window.  Returns (oracle's total count, starts of windows that differ)."""
    edges = list(range(lo, hi, window)) + [hi]
    spans = list(zip(edges[:-1], edges[1:]))
    lists = pmap(lambda ab: oracle.primes(ab[0], ab[1]), spans)
    bad, at = [], 0
    for (a, _), ref in zip(spans, lists):
        got = values[at:at + len(ref)].astype(np.uint64)
        if len(got) != len(ref) or not np.array_equal(got, ref):
            bad.append(a)
        at += len(ref)
    return at, bad
