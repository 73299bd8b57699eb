"""GPU parity: the CUDA sieve (through the C ABI) against the CPU oracle,
element by element, bit-exact.  Marked gpu."""
import math

import numpy as np
import pytest

import oracle
import oracle_pool
from numtheory import load_golden, mr_is_prime, td_is_prime

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only hosts
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1205_4883_gb300 as gb  # noqa: E402
from paper_1205_4883_gb300.workloads import batch_intervals, random_ranges  # noqa: E402

PI = {int(x): int(v) for x, v in load_golden("pi_values.txt")}
HI_MAX = 1 << 47  # covers 10^14 + 10^8 (batched) and 10^12 + 10^9 (served)


@pytest.fixture(scope="module")
def sv():
    s = gb.Sieve(HI_MAX)
    yield s
    s.close()


def gpu_bitmap(sv, lo, hi):
    words, c = sv.bitmap(lo, hi)
    return words.cpu().numpy().view(np.uint32), c


def test_base_primes_match_oracle(sv):
    info = sv.info()
    assert info.prime_limit == math.isqrt(HI_MAX - 1)
    assert np.array_equal(sv.base_primes(), oracle.base_primes(info.prime_limit))


def test_pi_1e7_count_bitmap_list(sv):
    lo, hi = 0, 10**7
    assert sv.count(lo, hi) == PI[10**7]
    words, c = gpu_bitmap(sv, lo, hi)
    assert c == PI[10**7]
    assert np.array_equal(words, oracle.bitmap(lo, hi))
    lst = sv.primes(lo, hi).cpu().numpy().view(np.uint32).astype(np.uint64)
    assert np.array_equal(lst, oracle.primes(lo, hi))
    assert lst[-1] == 9_999_991


def test_all_small_ranges_brute_force(sv):
    # every 0 <= lo <= hi <= 2000, batched, against trial division
    mask = np.array([td_is_prime(n) for n in range(2001)])
    prefix = np.concatenate([[0], np.cumsum(mask)])
    pairs = [(lo, hi) for lo in range(2001) for hi in range(lo, 2001)]
    for k in range(0, len(pairs), 250_000):
        chunk = pairs[k:k + 250_000]
        got = sv.batch_count([p[0] for p in chunk], [p[1] for p in chunk])
        expect = [int(prefix[hi] - prefix[lo]) for lo, hi in chunk]
        assert got == expect


@pytest.mark.parametrize("lo", [0, 1, 2, 3, 4, 5, 7, 8, 29, 30, 31, 959, 960, 961])
def test_low_starts_bitmap_and_list(sv, lo):
    for hi in (lo, lo + 1, lo + 2, lo + 31, lo + 64, lo + 1000, lo + 123_457, 7_000_000):
        if hi < lo:
            continue
        words, c = gpu_bitmap(sv, lo, hi)
        assert np.array_equal(words, oracle.bitmap(lo, hi)), (lo, hi)
        assert c == oracle.count(lo, hi)
        assert sv.count(lo, hi) == c
        lst = sv.primes(lo, hi, dtype64=True).cpu().numpy().view(np.uint64)
        assert np.array_equal(lst, oracle.primes(lo, hi)), (lo, hi)


def test_every_start_below_1000(sv):
    # exercises every phase of the segment grid origin (negative wheel bytes included)
    for lo in range(0, 1000):
        hi = lo + 3001
        words, c = gpu_bitmap(sv, lo, hi)
        assert np.array_equal(words, oracle.bitmap(lo, hi)), lo
        assert c == oracle.count(lo, hi)


@pytest.mark.parametrize("p", [2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 9_999_991, 4_294_967_291])
def test_prime_at_range_edges(sv, p):
    for lo, hi in ((p, p), (p, p + 1), (p - 1, p), (p - 1, p + 1), (p + 1, p + 2), (0, p), (0, p + 1)):
        if lo < 0:
            continue
        assert sv.count(lo, hi) == oracle.count(lo, hi), (lo, hi)
        words, _ = gpu_bitmap(sv, lo, hi)
        assert np.array_equal(words, oracle.bitmap(lo, hi)), (lo, hi)


def test_random_ranges_vs_oracle(sv):
    for lo, hi in random_ranges(60, seed=1205, max_lo=10**12, max_w=2 * 10**7):
        c = sv.count(lo, hi)
        assert c == oracle.count(lo, hi), (lo, hi)
        words, c2 = gpu_bitmap(sv, lo, hi)
        assert c2 == c
        assert np.array_equal(words, oracle.bitmap(lo, hi)), (lo, hi)


def test_lists_vs_oracle(sv):
    for lo, hi in random_ranges(12, seed=77, max_lo=2**32 - 10**7, max_w=10**7) + [(2**32 - 10**6, 2**32)]:
        got = sv.primes(lo, hi).cpu().numpy().view(np.uint32).astype(np.uint64)
        assert np.array_equal(got, oracle.primes(lo, hi)), (lo, hi)
    for lo, hi in random_ranges(8, seed=78, max_lo=10**14, max_w=3 * 10**6):
        got = sv.primes(lo, hi, dtype64=True).cpu().numpy().view(np.uint64)
        assert np.array_equal(got, oracle.primes(lo, hi)), (lo, hi)


def test_multi_segment_ranges_several_grid_phases(sv):
    # Ranges spanning many segments, with p^2 crossing segment edges; lo and hi
    # on and off multiples of 30 and 210, and straddling 2^32.
    S = sv.get_param(gb.SIEVE_PARAM_SEGMENT_BYTES)
    span = 30 * S
    for lo, hi in [(0, 9 * span + 17), (30 * 7, 210 * 100_000), (span - 1, 3 * span + 1),
                   (2**32 - 5 * span // 2, 2**32 + 5 * span // 2), (10**12 - span, 10**12 + span),
                   (210 * 10**9, 210 * 10**9 + 4 * span)]:
        assert sv.count(lo, hi) == oracle.count(lo, hi), (lo, hi)
        words, _ = gpu_bitmap(sv, lo, hi)
        assert np.array_equal(words, oracle.bitmap(lo, hi)), (lo, hi)


@pytest.mark.parametrize("seg,threads,small,ctas,chunk,blim", [
    (1024, 256, 23, 1, 1, 0), (4096 + 32, 512, 100, 2, 7, 0), (65536, 1024, 65536, 1, 64, 0),
    (229376, 1024, 7168, 1, 16, 0), (32 * 1001, 256, 2000, 3, 3, 0),
    # most primes through the bucket lists, several hits per list per prime
    (229376, 1024, 1792, 1, 16, 30), (8192, 512, 60, 1, 64, 100), (229376, 1024, 1792, 1, 1, 2000),
    # no bucket lists at all
    (229376, 1024, 1792, 1, 16, 1 << 40)])
def test_launch_parameters_do_not_change_results(seg, threads, small, ctas, chunk, blim):
    with gb.Sieve(10**13) as s:
        s.set_param(gb.SIEVE_PARAM_SEGMENT_BYTES, seg)
        s.set_param(gb.SIEVE_PARAM_THREADS, threads)
        s.set_param(gb.SIEVE_PARAM_SMALL_LIMIT, small)
        s.set_param(gb.SIEVE_PARAM_CTAS_PER_SM, ctas)
        s.set_param(gb.SIEVE_PARAM_CHUNK_SEGMENTS, chunk)
        s.set_param(gb.SIEVE_PARAM_BUCKET_LIMIT, blim)
        for lo, hi in [(0, 10**7), (123_456_789_012, 123_456_789_012 + 3 * 10**6), (5, 40_000),
                       (9 * 10**12, 9 * 10**12 + 2 * 10**7)]:
            assert s.count(lo, hi) == oracle.count(lo, hi)
            words, _ = s.bitmap(lo, hi)
            assert np.array_equal(words.cpu().numpy().view(np.uint32), oracle.bitmap(lo, hi))


@pytest.mark.parametrize("mid", [0, 2000, 400_000, 60])
def test_tier_limits_do_not_change_results(mid):
    # which primes go to the per-phase tier and which to the wheel walk; ranges around
    # the squares of primes near 10^6 (999983^2) start those primes mid-segment
    p2 = 999983 ** 2
    with gb.Sieve(10**13) as s:
        s.set_param(gb.SIEVE_PARAM_MID_LIMIT, mid)
        for lo, hi in [(0, 10**8), (123_456_789_012, 123_456_789_012 + 3 * 10**6), (5, 40_000),
                       (9 * 10**12, 9 * 10**12 + 2 * 10**7), (p2 - 5 * 10**6, p2 + 5 * 10**6)]:
            assert s.count(lo, hi) == oracle.count(lo, hi), (lo, hi)
            words, _ = s.bitmap(lo, hi)
            assert np.array_equal(words.cpu().numpy().view(np.uint32), oracle.bitmap(lo, hi)), (lo, hi)


@pytest.mark.parametrize("presieve", [19, 59, 71])
@pytest.mark.parametrize("small", [23, 61, 512])
def test_presieve_patterns_do_not_change_results(presieve, small):
    # primes 23..59 crossed one by one (19) or ANDed in as three patterns (59), with the
    # small tier starting below, at or above the first prime it crosses; wheel bytes
    # 0 and 1 (integers 1..59) hold primes the patterns clear
    with gb.Sieve(10**13) as s:
        s.set_param(gb.SIEVE_PARAM_PRESIEVE, presieve)
        s.set_param(gb.SIEVE_PARAM_SMALL_LIMIT, small)
        assert s.get_param(gb.SIEVE_PARAM_PRESIEVE) == presieve
        for lo, hi in [(0, 10**7), (0, 60), (1, 61), (30, 90), (31, 32), (47, 48), (49, 50), (53, 60),
                       (60, 90), (61, 62), (67, 68), (71, 72), (73, 74), (77, 78), (0, 100), (59, 200),
                       (5, 40_000), (10**12 - 10**6, 10**12 + 10**6), (9 * 10**12, 9 * 10**12 + 2 * 10**7)]:
            assert s.count(lo, hi) == oracle.count(lo, hi), (lo, hi)
            words, _ = s.bitmap(lo, hi)
            assert np.array_equal(words.cpu().numpy().view(np.uint32), oracle.bitmap(lo, hi)), (lo, hi)
        with pytest.raises(gb.SieveError):
            s.set_param(gb.SIEVE_PARAM_PRESIEVE, 47)


def test_bounded_device_wait_and_fault_hook(sv):
    # the bounded mbarrier wait of the bulk shared-memory copies: it completes when a copy
    # arrives, and when nothing ever completes the barrier it runs out after the limit and
    # returns (no trap, no hang); the context stays usable afterwards
    assert gb.sieve_selftest_wait(sv.ctx, True, 1 << 20) is False
    assert gb.sieve_selftest_wait(sv.ctx, False, 2000) is True
    assert sv.count(0, 10**6) == 78498
    # the host's handling of a device-side wait failure, injected on the host
    sv.set_param(gb.SIEVE_PARAM_FAULT_WAIT, 1)
    try:
        with pytest.raises(gb.SieveError) as e:
            sv.count(0, 10**6)
        assert e.value.code == gb.SIEVE_EDEVICE
    finally:
        sv.set_param(gb.SIEVE_PARAM_FAULT_WAIT, 0)
    assert sv.count(0, 10**6) == 78498


def test_large_lo_against_miller_rabin(sv):
    lo, hi = 10**14, 10**14 + 60_000
    got = [int(v) for v in sv.primes(lo, hi, dtype64=True).cpu().numpy().view(np.uint64)]
    assert got == [n for n in range(lo, hi) if mr_is_prime(n)]


def test_additivity_at_scale(sv):
    for lo, hi in random_ranges(10, seed=9, max_lo=10**14, max_w=10**9):
        mid = (lo + hi) // 2 + 13
        mid = min(mid, hi)
        assert sv.count(lo, mid) + sv.count(mid, hi) == sv.count(lo, hi)


def test_count_dev_matches_count(sv):
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    for lo, hi in [(0, 10**9), (10**12, 10**12 + 10**8), (7, 8), (100, 100)]:
        out.fill_(12345)
        sv.count_dev(lo, hi, out)
        assert int(out.item()) == sv.count(lo, hi) == oracle.count(lo, hi)


def test_errors_and_size_query(sv):
    with pytest.raises(gb.SieveError) as e:
        sv.count(10, 5)
    assert e.value.code == gb.SIEVE_EINVAL
    with pytest.raises(gb.SieveError) as e:
        sv.count(0, HI_MAX + 1)
    assert e.value.code == gb.SIEVE_ERANGE
    with pytest.raises(gb.SieveError) as e:
        gb.sieve_list(sv.ctx, 0, 2**32 + 2, None, 0)
    assert e.value.code == gb.SIEVE_ERANGE
    n, rc = gb.sieve_list(sv.ctx, 0, 10**6, None, 0)
    assert rc == gb.SIEVE_ETRUNC and n == PI[10**6]
    small = torch.zeros(10, dtype=torch.int32, device="cuda")
    n, rc = gb.sieve_list(sv.ctx, 0, 10**6, small)
    assert rc == gb.SIEVE_ETRUNC and n == PI[10**6]
    assert int(small.abs().sum().item()) == 0  # nothing written on ETRUNC
    bm = torch.zeros(3, dtype=torch.int32, device="cuda")
    with pytest.raises(gb.SieveError) as e:
        gb.sieve_bitmap(sv.ctx, 0, 10**4, bm)
    assert e.value.code == gb.SIEVE_ETRUNC
    assert sv.count(5, 5) == 0
    n, rc = gb.sieve_list(sv.ctx, 8, 8, None, 0)
    assert n == 0 and rc == gb.SIEVE_OK


def test_pi_1e12_full_size(sv):
    # the count-only workload at full size, default launch configuration
    assert sv.count(0, 10**12) == PI[10**12]


def test_range_2p32_bitmap_then_compaction(sv):
    # the [0, 2^32) workload at full size in the bench's launch shape (sieve_bitmap, then
    # sieve_compact): every word of the bitmap and every entry of the list against the oracle
    lo, hi = 0, 1 << 32
    nw = gb.sieve_bitmap_words(lo, hi)
    assert nw == 1 << 26
    bm = torch.empty(nw, dtype=torch.int32, device="cuda")
    c = gb.sieve_bitmap(sv.ctx, lo, hi, bm)
    assert c == PI[1 << 32]
    lst = torch.empty(PI[1 << 32], dtype=torch.int32, device="cuda")
    n, rc = gb.sieve_compact(sv.ctx, bm, lo, hi, lst)
    assert rc == gb.SIEVE_OK and n == PI[1 << 32]
    bmh = bm.cpu().numpy().view(np.uint32)
    assert oracle_pool.compare_bitmap(bmh, lo, hi) == []
    uh = lst.cpu().numpy().view(np.uint32)
    total, bad = oracle_pool.compare_list(uh, lo, hi)
    assert total == n and bad == []
    assert int(uh[0]) == 2 and int(uh[-1]) == 4_294_967_291


def test_batch_4096_intervals(sv):
    # the batched workload at full size: every one of the 4096 counts against the oracle,
    # and against the single-range call on the same GPU for a sample
    los, his = batch_intervals(4096, seed=1205)
    counts = sv.batch_count(los, his)
    assert counts == oracle_pool.counts(los, his)
    for i in range(0, 4096, 97):
        assert counts[i] == sv.count(los[i], his[i]), i


def test_batch_4096_intervals_with_bitmaps(sv):
    # the same 4096 intervals with a bitmap for every one, in one launch (bitmap mode):
    # each count and every word of each bitmap against the oracle
    los, his = batch_intervals(4096, seed=1205)
    nws = [gb.sieve_bitmap_words(a, b) for a, b in zip(los, his)]
    offs = np.concatenate([[0], np.cumsum(nws)]).astype(np.int64)
    store = torch.zeros(int(offs[-1]) + 1, dtype=torch.int32, device="cuda")
    base = store.data_ptr()
    ptrs = [base + 4 * int(offs[i]) for i in range(4096)]
    counts = sv.batch_count(los, his, ptrs)
    host = store.cpu().numpy().view(np.uint32)

    def check(i):
        ref = oracle.bitmap(los[i], his[i])
        ok = np.array_equal(host[offs[i]:offs[i + 1]], ref)
        return ok and counts[i] == int(np.unpackbits(ref.view(np.uint8)).sum()) + (los[i] <= 2 < his[i])

    bad = [i for i, ok in zip(range(4096), oracle_pool.pmap(check, range(4096))) if not ok]
    assert bad == []


def test_crossing_work_matches_the_oracle(sv):
    # the roofline numerator (sieve_crossing_work, host arithmetic in the library) against
    # the oracle's count of the same bit-clears: the stored golden values at full size,
    # then random ranges
    for lo, hi, pmin, w, v in load_golden("crossings.txt"):
        lo, hi, pmin, w, v = (int(x) for x in (lo, hi, pmin, w, v))
        if hi > HI_MAX:
            continue
        sv.set_param(gb.SIEVE_PARAM_WHEEL, w)
        try:
            assert sv.crossing_work(lo, hi, pmin) == v, (lo, hi, pmin, w)
            if pmin == 23:
                assert sv.crossing_work(lo, hi) == v
        finally:
            sv.set_param(gb.SIEVE_PARAM_WHEEL, 30)
    for lo, hi in random_ranges(20, seed=31, max_lo=10**14, max_w=10**9):
        for pmin in (23, 61, 1000):
            assert sv.crossing_work(lo, hi, pmin) == oracle.crossings(lo, hi, max(pmin, 23), 30), (lo, hi)


def test_batch_order_does_not_change_results(sv):
    los, his = batch_intervals(512, seed=77)
    assert sv.get_param(gb.SIEVE_PARAM_BATCH_ORDER) == 0
    as_given = sv.batch_count(los, his)
    try:
        for order in (1, 2):
            sv.set_param(gb.SIEVE_PARAM_BATCH_ORDER, order)
            assert sv.batch_count(los, his) == as_given, order
    finally:
        sv.set_param(gb.SIEVE_PARAM_BATCH_ORDER, 0)
    for i in range(0, 512, 61):
        assert as_given[i] == sv.count(los[i], his[i])


def test_batch_with_bitmaps(sv):
    los, his = batch_intervals(64, seed=11, lo_exp=(3, 13), w_exp=(1, 6))
    bms = [torch.zeros(max(gb.sieve_bitmap_words(a, b), 1), dtype=torch.int32, device="cuda") if i % 3 else None
           for i, (a, b) in enumerate(zip(los, his))]
    counts = sv.batch_count(los, his, bms)
    for i, (a, b) in enumerate(zip(los, his)):
        assert counts[i] == oracle.count(a, b), i
        if bms[i] is not None:
            nw = gb.sieve_bitmap_words(a, b)
            assert np.array_equal(bms[i][:nw].cpu().numpy().view(np.uint32), oracle.bitmap(a, b)), i


def _random_range_params(m, seed, bitmaps=False):
    from paper_1205_4883_gb300 import autotune
    from paper_1205_4883_gb300.workloads import SplitMix64
    rng = SplitMix64(seed)
    out = []
    for _ in range(m):
        q = {}
        for f, cands in autotune.CANDIDATES.items():
            q[f] = cands[rng.next() % len(cands)]
        if bitmaps:
            q["wheel"] = 30 if rng.next() % 2 else 0
        if rng.next() % 4 == 0:
            q["seg_bytes"] = 1024 + 32 * (rng.next() % 7000)
        out.append(q)
    return out


def test_batch_per_range_parameters_do_not_change_results(sv):
    # the 4096-interval batch with every range's segment bytes, wheel, bucket limit, tier
    # limit and Miller-Rabin threshold drawn at random, in one launch: every count
    # against the oracle
    los, his = batch_intervals(4096, seed=1205)
    params = _random_range_params(4096, seed=7)
    assert sv.batch_count_params(los, his, params) == oracle_pool.counts(los, his)


def test_batch_per_range_parameters_with_bitmaps(sv):
    # bitmap mode (mod-30 wheel only): counts and every word of every bitmap
    los, his = batch_intervals(512, seed=99, lo_exp=(3, 14), w_exp=(2, 7))
    params = _random_range_params(512, seed=8, bitmaps=True)
    nws = [gb.sieve_bitmap_words(a, b) for a, b in zip(los, his)]
    offs = np.concatenate([[0], np.cumsum(nws)]).astype(np.int64)
    store = torch.zeros(int(offs[-1]) + 1, dtype=torch.int32, device="cuda")
    ptrs = [store.data_ptr() + 4 * int(offs[i]) for i in range(512)]
    counts = sv.batch_count_params(los, his, params, ptrs)
    host = store.cpu().numpy().view(np.uint32)
    assert counts == oracle_pool.counts(los, his)
    bad = [i for i, ok in enumerate(oracle_pool.pmap(
        lambda i: np.array_equal(host[offs[i]:offs[i + 1]], oracle.bitmap(los[i], his[i])), range(512))) if not ok]
    assert bad == []


def test_batch_per_range_parameter_errors(sv):
    los, his = [10**9, 10**10], [10**9 + 1000, 10**10 + 1000]
    for bad in ({"seg_bytes": 1000}, {"seg_bytes": 229376 + 32}, {"wheel": 60}):
        with pytest.raises(gb.SieveError) as e:
            sv.batch_count_params(los, his, [bad, {}])
        assert e.value.code == gb.SIEVE_EINVAL
    bm = [torch.zeros(64, dtype=torch.int32, device="cuda") for _ in range(2)]
    with pytest.raises(gb.SieveError) as e:
        sv.batch_count_params(los, his, [{"wheel": 210}, {}], bm)
    assert e.value.code == gb.SIEVE_EINVAL
    # all fields 0: the context's parameters, as sieve_batch_count
    assert sv.batch_count_params(los, his, [{}, {}]) == sv.batch_count(los, his)


def test_batch_tuned_equals_untuned(sv):
    from paper_1205_4883_gb300 import autotune
    los, his = batch_intervals(600, seed=3, lo_exp=(2, 14), w_exp=(1, 7))
    table = {"classes": {"0/0": {"seg_bytes": 32768, "mid_limit": 4096},
                         "1/1": {"wheel": 210, "seg_bytes": 65536},
                         "2/2": {"bucket_limit": 229376},
                         "4/2": {"mr_percent": 100},
                         "3/1": {"wheel": 210}}}
    assert sv.batch_count_tuned(los, his, table) == sv.batch_count(los, his) == oracle_pool.counts(los, his)
    assert sv.get_param(gb.SIEVE_PARAM_SEGMENT_BYTES) == 229376  # the context is untouched
    assert {autotune.class_key(a, b) for a, b in zip(los, his)} >= {"0/0", "1/1", "2/2"}


@pytest.mark.parametrize("lo,hi", [(0, 10**10), (99 * 10**10, 10**12), (10**9 - 5, 10**9 + 4 * 10**9),
                                   (4 * 10**12, 4 * 10**12 + 10**10)])
def test_large_prime_cursors_match_recomputation(lo, hi):
    # chunks of consecutive segments carry the large primes' wheel cursors; primes
    # whose p^2 enters mid-chunk start fresh.  Same results as recomputing per segment.
    with gb.Sieve(5 * 10**12) as s:
        s.set_param(gb.SIEVE_PARAM_CHUNK_SEGMENTS, 64)
        with_cursors = s.count(lo, hi)
        wa, _ = s.bitmap(lo, min(hi, lo + 2 * 10**9))
        s.set_param(gb.SIEVE_PARAM_CURSOR_MB, 0)
        assert s.count(lo, hi) == with_cursors
        wb, _ = s.bitmap(lo, min(hi, lo + 2 * 10**9))
        assert torch.equal(wa, wb)
    if (lo, hi) == (0, 10**10):
        assert with_cursors == PI[10**10]
    else:
        assert with_cursors == oracle.count(lo, hi)


@pytest.mark.parametrize("lo,w", [(10**12 + 7, 10**5), (10**13 + 11, 3 * 10**4), (10**14, 10**5),
                                  (2**32 + 1, 5 * 10**5), (4295098369 - 500, 1000)])
def test_miller_rabin_path_matches(sv, lo, w):
    # narrow ranges high up: sieve with the primes below 2^16, then Miller-Rabin
    hi = lo + w
    s = sv
    s.set_param(gb.SIEVE_PARAM_MR_PERCENT, 10**6)  # force the path
    try:
        c_mr = s.count(lo, hi)
        bm_mr, _ = s.bitmap(lo, hi)
        lst_mr = s.primes(lo, hi, dtype64=True).cpu().numpy().view(np.uint64)
        counts_mr = s.batch_count([lo, lo + 17, lo + w // 2], [hi, hi - 3, hi])
    finally:
        s.set_param(gb.SIEVE_PARAM_MR_PERCENT, 0)
    assert c_mr == s.count(lo, hi) == oracle.count(lo, hi)
    bm_sieve, _ = s.bitmap(lo, hi)
    assert torch.equal(bm_mr, bm_sieve)
    assert np.array_equal(lst_mr, oracle.primes(lo, hi))
    assert counts_mr == [oracle.count(lo, hi), oracle.count(lo + 17, hi - 3), oracle.count(lo + w // 2, hi)]
    s.set_param(gb.SIEVE_PARAM_MR_PERCENT, 0)


def test_miller_rabin_path_rejects_strong_pseudoprimes():
    with gb.Sieve(4 * 10**14) as s:
        s.set_param(gb.SIEVE_PARAM_MR_PERCENT, 10**6)
        for n in (2152302898747, 3474749660383, 341550071728321):
            lo, hi = n - 2000, n + 2000
            got = [int(v) for v in s.primes(lo, hi, dtype64=True).cpu().numpy().view(np.uint64)]
            assert n not in got
            assert got == [x for x in range(lo, hi) if mr_is_prime(x)]


def test_roofline_probes_report_plausible_rates(sv):
    # measured denominators: lane-ops per SM clock (at most 32, one per lane) and GB/s
    cf = gb.sieve_probe(sv.ctx, gb.SIEVE_PROBE_SMEM_AND_CONFLICT_FREE)
    rnd = gb.sieve_probe(sv.ctx, gb.SIEVE_PROBE_SMEM_AND_RANDOM)
    st = gb.sieve_probe(sv.ctx, gb.SIEVE_PROBE_SMEM_STORE_CONFLICT_FREE)
    assert 4 < rnd < cf <= 32.5 and 4 < st <= 32.5
    buf = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")
    gbs = gb.sieve_probe(sv.ctx, gb.SIEVE_PROBE_HBM_WRITE, buf)
    assert 1000 < gbs < 20000
    with pytest.raises(gb.SieveError):
        gb.sieve_probe(sv.ctx, 99)


def test_compaction_into_unaligned_and_offset_outputs(sv):
    # list outputs at every 4-byte (u32) and 8-byte (u64) offset from a 16-byte boundary:
    # the emit's 16-byte stores apply only when the output is aligned, and neighbouring
    # entries outside the list are never written
    lo, hi = 10**9 - 12_345, 10**9 + 3_000_000
    want = oracle.primes(lo, hi)
    n = len(want)
    for off in range(4):
        buf = torch.full((n + 8,), -1, dtype=torch.int32, device="cuda")
        got_n, rc = gb.sieve_list(sv.ctx, lo, hi, buf[off:], n)
        assert rc == gb.SIEVE_OK and got_n == n
        h = buf.cpu().numpy()
        assert np.array_equal(h[off:off + n].view(np.uint32).astype(np.uint64), want), off
        assert (h[:off] == -1).all() and (h[off + n:] == -1).all(), off
    for off in range(2):
        buf = torch.full((n + 4,), -1, dtype=torch.int64, device="cuda")
        got_n, rc = gb.sieve_list64(sv.ctx, lo, hi, buf[off:], n)
        assert rc == gb.SIEVE_OK and got_n == n
        h = buf.cpu().numpy()
        assert np.array_equal(h[off:off + n].view(np.uint64), want), off
        assert (h[:off] == -1).all() and (h[off + n:] == -1).all(), off
