"""GPU parity of the asynchronous entry points (sieve_count_dev, sieve_bitmap_dev,
sieve_compact_dev): the counts they leave on the device, the bitmaps and the lists
against the CPU oracle, bit-exact, with many calls enqueued before one
synchronisation.  Marked gpu."""
import numpy as np
import pytest

import oracle
from numtheory import load_golden

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only hosts
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1205_4883_gb300 as gb  # noqa: E402
from paper_1205_4883_gb300.workloads import random_ranges  # noqa: E402

PI = {int(x): int(v) for x, v in load_golden("pi_values.txt")}

# ragged and degenerate ranges below 2^32: empty, the list [2], one odd integer,
# a word edge, several segments and tiles of the compaction, the top of 2^32
RANGES = [(0, 0), (2, 2), (2, 3), (0, 3), (1, 2), (3, 4), (4, 5), (0, 64), (63, 129), (0, 10**7),
          (10**9 + 1, 10**9 + 10**6 + 17), (2**32 - 10**6 - 3, 2**32), (123_456_789, 123_456_789 + 4_194_303)]


@pytest.fixture(scope="module")
def sv():
    s = gb.Sieve(1 << 40)
    yield s
    s.close()


def _sync():
    # the context runs on torch's current stream; the test reads results only after this
    torch.cuda.synchronize()


def test_bitmap_dev_and_compact_dev_enqueued_together_match_the_oracle(sv):
    ranges = RANGES + random_ranges(10, seed=4242, max_lo=2**32 - 3 * 10**6, max_w=3 * 10**6)
    bufs = []
    for lo, hi in ranges:
        nw = gb.sieve_bitmap_words(lo, hi)
        bm = torch.full((max(nw, 1),), -1, dtype=torch.int32, device="cuda")
        lst = torch.full((oracle.count(lo, hi) + 5,), -7, dtype=torch.int32, device="cuda")
        cnt = torch.full((2,), -1, dtype=torch.int64, device="cuda")
        bufs.append((lo, hi, nw, bm, lst, cnt))
    _sync()
    for lo, hi, nw, bm, lst, cnt in bufs:  # every call enqueued before the one synchronisation
        gb.sieve_bitmap_dev(sv.ctx, lo, hi, bm, cnt[0:1])
        gb.sieve_compact_dev(sv.ctx, bm, lo, hi, lst, cnt[1:2])
    _sync()
    for lo, hi, nw, bm, lst, cnt in bufs:
        expect = oracle.count(lo, hi)
        c, n = (int(x) for x in cnt.cpu())
        assert c == expect and n == expect, (lo, hi)
        assert np.array_equal(bm[:nw].cpu().numpy().view(np.uint32), oracle.bitmap(lo, hi)), (lo, hi)
        got = lst.cpu().numpy().view(np.uint32)
        assert np.array_equal(got[:n].astype(np.uint64), oracle.primes(lo, hi)), (lo, hi)
        assert (got[n:].view(np.int32) == -7).all(), (lo, hi)  # nothing written past the list


def test_back_to_back_async_calls_behind_a_long_launch(sv):
    # A long count first: the calls after it are enqueued while it runs, so each
    # one's launch block must not be rewritten before its copy has run.
    cases = [(0, 10**11), (0, 10**7), (10**9, 10**9 + 10**6), (7, 8), (2, 3), (10**10, 10**10 + 3 * 10**6),
             (10**12 - 10**6, 10**12), (5 * 10**8, 5 * 10**8 + 10**5), (1, 10**6)]
    outs = torch.full((len(cases),), -1, dtype=torch.int64, device="cuda")
    lo, hi = 10**9 + 7, 10**9 + 7 + 10**6
    nw = gb.sieve_bitmap_words(lo, hi)
    bm = torch.zeros(nw, dtype=torch.int32, device="cuda")
    c = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    _sync()
    for i, (lo2, hi2) in enumerate(cases):
        sv.count_dev(lo2, hi2, outs[i:i + 1])
    gb.sieve_bitmap_dev(sv.ctx, lo, hi, bm, c)
    _sync()
    got = outs.cpu().tolist()
    assert got[0] == PI[10**11]
    for (lo2, hi2), g in zip(cases[1:], got[1:]):
        assert g == oracle.count(lo2, hi2), (lo2, hi2)
    assert int(c.item()) == oracle.count(lo, hi)
    assert np.array_equal(bm.cpu().numpy().view(np.uint32), oracle.bitmap(lo, hi))


def test_compact_dev_below_capacity_truncates(sv):
    # one pass: a list that does not fit is written up to cap (the prime 2 included),
    # nothing beyond it; cap = 0 without an output is the size query
    lo, hi = 0, 10**6
    want = oracle.primes(lo, hi)
    nw = gb.sieve_bitmap_words(lo, hi)
    bm = torch.zeros(nw, dtype=torch.int32, device="cuda")
    n = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    _sync()
    gb.sieve_bitmap_dev(sv.ctx, lo, hi, bm, n)
    for cap in (0, 1, 2, 2047, 40_000, PI[10**6] - 1):
        lst = torch.full((PI[10**6] + 1,), -3, dtype=torch.int32, device="cuda")
        _sync()
        gb.sieve_compact_dev(sv.ctx, bm, lo, hi, lst if cap else None, n, cap=cap)
        _sync()
        assert int(n.item()) == PI[10**6]
        got = lst.cpu().numpy()
        assert np.array_equal(got[:cap].view(np.uint32).astype(np.uint64), want[:cap]), cap
        assert (got[cap:] == -3).all(), cap
    lst = torch.full((PI[10**6],), -3, dtype=torch.int32, device="cuda")
    _sync()
    gb.sieve_compact_dev(sv.ctx, bm, lo, hi, lst, n)
    _sync()
    assert int(n.item()) == PI[10**6]
    assert np.array_equal(lst.cpu().numpy().view(np.uint32).astype(np.uint64), oracle.primes(lo, hi))


def test_async_argument_errors(sv):
    bm = torch.zeros(16, dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(gb.SieveError) as e:
        gb.sieve_bitmap_dev(sv.ctx, 0, 100, bm, None)
    assert e.value.code == gb.SIEVE_EINVAL
    with pytest.raises(gb.SieveError) as e:
        gb.sieve_bitmap_dev(sv.ctx, 0, 10**6, bm, n)  # 16 words are too few
    assert e.value.code == gb.SIEVE_ETRUNC
    with pytest.raises(gb.SieveError) as e:
        gb.sieve_compact_dev(sv.ctx, bm, 0, 100, bm, None)
    assert e.value.code == gb.SIEVE_EINVAL
    with pytest.raises(gb.SieveError) as e:
        gb.sieve_compact_dev(sv.ctx, bm, 2**32, 2**32 + 64, bm, n)
    assert e.value.code == gb.SIEVE_ERANGE
    with pytest.raises(gb.SieveError) as e:
        gb.sieve_compact_dev(sv.ctx, bm, 0, 100, None, n, cap=5)
    assert e.value.code == gb.SIEVE_EINVAL
    with pytest.raises(gb.SieveError) as e:
        gb.sieve_compact_dev(sv.ctx, bm, 200, 100, bm, n)
    assert e.value.code == gb.SIEVE_EINVAL
