"""The request server (continuous batching): every result is the same alone and
in the mix (exact), short requests are not held behind long ones, and
admission and errors behave as declared.  Marked gpu."""
import time

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only hosts
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1205_4883_gb300 as gb  # noqa: E402
from paper_1205_4883_gb300.workloads import served_stream  # noqa: E402


@pytest.fixture(scope="module")
def sv():
    s = gb.Sieve(10**12 + 2 * 10**9)
    yield s
    s.close()


@pytest.mark.parametrize("serial", [False, True])
def test_mixed_stream_equals_alone(sv, serial):
    # ticks on two streams (overlapping) or on one: the same results
    reqs = served_stream(rate=1000.0, n=120, seed=1205, w_exp=(4, 8))
    with gb.Server(sv, tick_segments=300, serial_ticks=serial) as srv:
        tickets = []
        for r in reqs:
            kind = gb.SIEVE_REQ_LIST if r.kind == "list" else gb.SIEVE_REQ_COUNT
            rc, t = srv.submit(r.lo, r.hi, kind)
            assert rc == gb.SIEVE_OK
            tickets.append(t)
        results = []
        for t in tickets:
            rc, res = srv.poll(t, timeout_us=60_000_000)
            assert rc == gb.SIEVE_OK and res["status"] == gb.SIEVE_OK
            results.append(res)
            assert srv.release(t) == gb.SIEVE_OK
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["in_flight"] == 0
        assert st["segments"] >= len(reqs) and st["tick_gpu_ms"] > 0 and st["ticks"] > 0
    for r, res in zip(reqs, results):
        alone = sv.count(r.lo, r.hi)
        assert res["count"] == alone, (r.lo, r.hi)
        if r.kind == "list":
            lst = sv.primes(r.lo, r.hi, dtype64=True).cpu().numpy().view(np.uint64)
            assert np.array_equal(res["primes"], lst)
    # a seeded subset against the oracle
    for r, res in list(zip(reqs, results))[:25]:
        assert res["count"] == oracle.count(r.lo, r.hi)
        if r.kind == "list":
            assert np.array_equal(res["primes"], oracle.primes(r.lo, r.hi))


def test_short_requests_overtake_a_long_one(sv):
    # a long request advances a few segments per tick; short ones that arrive
    # meanwhile join the next tick and finish long before it
    with gb.Server(sv, tick_segments=152) as srv:
        rc, long_t = srv.submit(0, 10**12)
        assert rc == gb.SIEVE_OK
        time.sleep(0.01)
        shorts = []
        for k in range(8):
            lo = 10**11 + k * 10**7
            rc, t = srv.submit(lo, lo + 10**6, gb.SIEVE_REQ_LIST if k % 2 else gb.SIEVE_REQ_COUNT)
            assert rc == gb.SIEVE_OK
            shorts.append((lo, t))
        for lo, t in shorts:
            rc, res = srv.poll(t, timeout_us=30_000_000)
            assert rc == gb.SIEVE_OK
            assert res["count"] == oracle.count(lo, lo + 10**6)
            # the long request is still running when the short ones are done
            rc_long, _ = srv.poll(long_t, timeout_us=0)
            assert rc_long == gb.SIEVE_ETIMEOUT
        rc, res = srv.poll(long_t, timeout_us=120_000_000)
        assert rc == gb.SIEVE_OK and res["count"] == 37607912018


def test_admission_and_errors(sv):
    with gb.Server(sv, max_requests=4, max_device_bytes=64 << 20) as srv:
        tickets = [srv.submit(10**12, 10**12 + 10**9)[1] for _ in range(4)]
        rc, _ = srv.submit(0, 100)
        assert rc == gb.SIEVE_EBUSY  # no free slot
        with pytest.raises(gb.SieveError) as e:
            gb.sieve_server_submit(srv.srv, 5, 4)
        assert e.value.code == gb.SIEVE_EINVAL
        for t in tickets:
            assert srv.poll(t, timeout_us=60_000_000)[0] == gb.SIEVE_OK
            assert srv.release(t) == gb.SIEVE_OK
        assert srv.release(tickets[0]) == gb.SIEVE_ENOENT
        # a list request whose bitmap + bound exceed the memory budget is refused
        rc, _ = srv.submit(0, 10**9, gb.SIEVE_REQ_LIST)
        assert rc == gb.SIEVE_EBUSY
        st = srv.stats()
        assert st["rejected"] == 2 and st["device_bytes_reserved"] == 0
        # empty ranges complete at once
        rc, t = srv.submit(7, 7, gb.SIEVE_REQ_LIST)
        rc, res = srv.poll(t, timeout_us=1_000_000)
        assert rc == gb.SIEVE_OK and res["count"] == 0
    with pytest.raises(gb.SieveError) as e:
        with gb.Server(sv) as srv2:
            gb.sieve_server_poll(srv2.srv, 12345, 0)
    assert e.value.code == gb.SIEVE_ENOENT


def test_offset_lists_match_the_oracle(sv):
    # SIEVE_REQ_LIST_OFFSETS: uint32 offsets p - lo; the same primes as a uint64 list of the
    # same range, submitted in the same stream; ranges around 2, ragged ends, one at the top
    # of the context's range and a 3e8-wide one (many tiles of the compaction)
    ranges = [(0, 100), (1, 3), (2, 3), (3, 4), (0, 2), (10**12 - 10**6, 10**12),
              (10**12 + 2 * 10**9 - 10**6 - 7, 10**12 + 2 * 10**9), (10**9 + 1, 10**9 + 3 * 10**8)]
    ranges += [(r.lo, r.hi) for r in served_stream(rate=1000.0, n=20, seed=77, w_exp=(3, 7))]
    with gb.Server(sv, max_device_bytes=4 << 30) as srv:
        tickets = []
        for lo, hi in ranges:
            pair = []
            for kind in (gb.SIEVE_REQ_LIST_OFFSETS, gb.SIEVE_REQ_LIST):
                rc, t = srv.submit(lo, hi, kind)
                assert rc == gb.SIEVE_OK
                pair.append(t)
            tickets.append(pair)
        for (lo, hi), (t_off, t_list) in zip(ranges, tickets):
            rc, off = srv.poll(t_off, timeout_us=60_000_000)
            assert rc == gb.SIEVE_OK and off["status"] == gb.SIEVE_OK
            rc, lst = srv.poll(t_list, timeout_us=60_000_000)
            assert rc == gb.SIEVE_OK and lst["status"] == gb.SIEVE_OK
            want = oracle.primes(lo, hi)
            assert off["count"] == lst["count"] == len(want), (lo, hi)
            assert off["primes"] is None and off["offsets"].dtype == np.uint32
            assert np.array_equal(off["offsets"].astype(np.uint64) + np.uint64(lo), want), (lo, hi)
            assert np.array_equal(lst["primes"], want), (lo, hi)
            assert srv.release(t_off) == gb.SIEVE_OK and srv.release(t_list) == gb.SIEVE_OK
        # offsets must fit in 32 bits: a range wider than 2^32 is refused at submit
        with pytest.raises(gb.SieveError) as e:
            srv.submit(0, 2**32 + 1, gb.SIEVE_REQ_LIST_OFFSETS)
        assert e.value.code == gb.SIEVE_ERANGE
        with pytest.raises(gb.SieveError) as e:
            srv.submit(0, 10, 3)
        assert e.value.code == gb.SIEVE_EINVAL


def test_list_results_beyond_the_pinned_arena(sv):
    # four list results of ~48M primes (~385 MB each) held at once: the first ones land in
    # the 1 GiB pinned arena, the last one on the heap (bounce-buffer path); all exact
    ranges = [(10**9 * k, 10**9 * (k + 1)) for k in range(1, 5)]
    with gb.Server(sv, max_device_bytes=6 << 30) as srv:
        tickets = []
        for lo, hi in ranges:
            rc, t = srv.submit(lo, hi, gb.SIEVE_REQ_LIST)
            assert rc == gb.SIEVE_OK
            tickets.append(t)
        results = []
        for t in tickets:
            rc, res = srv.poll(t, timeout_us=120_000_000)
            assert rc == gb.SIEVE_OK and res["status"] == gb.SIEVE_OK
            results.append(res)
        for (lo, hi), res in zip(ranges, results):
            want = sv.primes(lo, hi, dtype64=True).cpu().numpy().view(np.uint64)
            assert res["count"] == len(want) == oracle.count(lo, hi)
            assert np.array_equal(res["primes"], want), (lo, hi)
        for t in tickets:
            assert srv.release(t) == gb.SIEVE_OK


def test_offset_results_beyond_the_pinned_arena(sv):
    # six offset lists of ~48M primes (~190 MB each, 1.15 GB in all) held at once: the last
    # ones overflow the 1 GiB pinned arena onto the heap (bounce buffer, 4-byte elements)
    ranges = [(10**9 * k + 7, 10**9 * (k + 1) + 7) for k in range(1, 7)]
    with gb.Server(sv, max_device_bytes=6 << 30) as srv:
        tickets = []
        for lo, hi in ranges:
            rc, t = srv.submit(lo, hi, gb.SIEVE_REQ_LIST_OFFSETS)
            assert rc == gb.SIEVE_OK
            tickets.append(t)
        results = []
        for t in tickets:  # every result held before any is released: they overflow the arena
            rc, res = srv.poll(t, timeout_us=120_000_000)
            assert rc == gb.SIEVE_OK and res["status"] == gb.SIEVE_OK
            results.append(res)
        assert 4 * sum(r["count"] for r in results) > 1 << 30
        for (lo, hi), res in zip(ranges, results):
            want = sv.primes(lo, hi, dtype64=True).cpu().numpy().view(np.uint64)
            assert res["count"] == len(want)
            assert np.array_equal(res["offsets"].astype(np.uint64) + np.uint64(lo), want), (lo, hi)
        for t in tickets:
            assert srv.release(t) == gb.SIEVE_OK
    lo, hi = ranges[-1]
    assert len(want) == oracle.count(lo, hi)


def test_completion_queue_reports_each_request_once(sv):
    # sieve_server_wait_any: every admitted request is reported exactly once, whether or
    # not it was polled first, and results read after it are the requests' own
    reqs = served_stream(rate=5000.0, n=200, seed=4, w_exp=(4, 7))
    with gb.Server(sv, tick_segments=200) as srv:
        want = {}
        for i, r in enumerate(reqs):
            kind = gb.SIEVE_REQ_LIST if r.kind == "list" else gb.SIEVE_REQ_COUNT
            rc, t = srv.submit(r.lo, r.hi, kind)
            assert rc == gb.SIEVE_OK
            want[t] = r
            if i == 10:  # one request polled before it is collected
                rc, _ = srv.poll(t, timeout_us=60_000_000)
                assert rc == gb.SIEVE_OK
        seen = []
        deadline = time.time() + 120
        while len(seen) < len(reqs) and time.time() < deadline:
            seen += srv.wait_any(64, timeout_us=100_000)
        assert sorted(seen) == sorted(want)
        assert srv.wait_any(8, timeout_us=1000) == []  # nothing left to report
        for t in seen:
            rc, res = srv.poll(t, timeout_us=0, copy_primes=False)
            assert rc == gb.SIEVE_OK and res["count"] == oracle.count(want[t].lo, want[t].hi)
            assert srv.release(t) == gb.SIEVE_OK
