"""GPU parity of the count path on the mod-210 wheel (SIEVE_PARAM_WHEEL = 210):
counts against the CPU oracle, trial division and the published pi(x) values,
bit-exact, through the C ABI.  Marked gpu."""
import numpy as np
import pytest

import oracle
from numtheory import load_golden, td_is_prime

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only hosts
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1205_4883_gb300 as gb  # noqa: E402
from paper_1205_4883_gb300.workloads import batch_intervals, random_ranges  # noqa: E402

PI = {int(x): int(v) for x, v in load_golden("pi_values.txt")}
HI_MAX = 1 << 47


@pytest.fixture(scope="module")
def sv210():
    s = gb.Sieve(HI_MAX)
    s.set_param(gb.SIEVE_PARAM_WHEEL, 210)
    yield s
    s.close()


def test_wheel_parameter(sv210):
    assert sv210.get_param(gb.SIEVE_PARAM_WHEEL) == 210
    with pytest.raises(gb.SieveError) as e:
        sv210.set_param(gb.SIEVE_PARAM_WHEEL, 6)
    assert e.value.code == gb.SIEVE_EINVAL


def test_w210_all_small_ranges_brute_force(sv210):
    # every 0 <= lo <= hi <= 1500 (group 0 with 11..19 and 1, the primes 2, 3, 5, 7 outside
    # the wheel), batched, against trial division
    mask = np.array([td_is_prime(n) for n in range(1501)])
    prefix = np.concatenate([[0], np.cumsum(mask)])
    pairs = [(lo, hi) for lo in range(1501) for hi in range(lo, 1501)]
    for k in range(0, len(pairs), 250_000):
        chunk = pairs[k:k + 250_000]
        got = sv210.batch_count([p[0] for p in chunk], [p[1] for p in chunk])
        assert got == [int(prefix[hi] - prefix[lo]) for lo, hi in chunk]


def test_w210_pi_values(sv210):
    for x in [10**k for k in range(1, 11)] + [1 << 32]:
        assert sv210.count(0, x) == PI[x], x


def test_w210_every_start_below_1000(sv210):
    los = list(range(1000))
    his = [lo + 10**6 + 7 * lo for lo in los]
    got = sv210.batch_count(los, his)
    for lo, hi, c in zip(los, his, got):
        assert c == oracle.count(lo, hi), (lo, hi)


def test_w210_random_ranges_vs_oracle(sv210):
    for lo, hi in random_ranges(30, seed=210, max_lo=10**14, max_w=3 * 10**7):
        assert sv210.count(lo, hi) == oracle.count(lo, hi), (lo, hi)


def test_w210_multi_segment_ranges_and_pattern_phases(sv210):
    # several segments, edges on and off multiples of 210, the pattern period
    # (46189 groups) and 2^32; squares of primes near 10^6 inside the range
    span = 210 * (57342 // 3 * 2)
    p2 = 999983 ** 2
    for lo, hi in [(0, 7 * span + 13), (210 * 46189 - 5, 210 * 46189 * 3 + 11), (span - 1, 3 * span + 1),
                   (2**32 - 5 * span // 2, 2**32 + 5 * span // 2), (10**12 - span, 10**12 + span),
                   (p2 - span, p2 + 2 * span)]:
        assert sv210.count(lo, hi) == oracle.count(lo, hi), (lo, hi)


@pytest.mark.parametrize("seg,small,mid,chunk,cursor_mb", [
    (1024, 23, 0, 1, 64), (4096 + 32, 60, 300, 7, 64), (65536, 1000, 5000, 64, 64),
    (229376, 128, 0, 16, 0), (229344, 23, 1 << 20, 16, 64), (229376, 512, 24, 3, 64)])
def test_w210_launch_parameters_do_not_change_results(seg, small, mid, chunk, cursor_mb):
    with gb.Sieve(10**13) as s:
        s.set_param(gb.SIEVE_PARAM_WHEEL, 210)
        s.set_param(gb.SIEVE_PARAM_SEGMENT_BYTES, seg)
        s.set_param(gb.SIEVE_PARAM_SMALL_LIMIT_210, small)
        s.set_param(gb.SIEVE_PARAM_MID_LIMIT_210, mid)
        s.set_param(gb.SIEVE_PARAM_CHUNK_SEGMENTS, chunk)
        s.set_param(gb.SIEVE_PARAM_CURSOR_MB, cursor_mb)
        for lo, hi in [(0, 10**7), (123_456_789_012, 123_456_789_012 + 3 * 10**6), (5, 40_000),
                       (9 * 10**12, 9 * 10**12 + 2 * 10**7), (0, 3 * 10**8)]:
            assert s.count(lo, hi) == oracle.count(lo, hi), (lo, hi)


def test_w210_count_dev_and_batch_match_the_mod30_path(sv210):
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    for lo, hi in [(0, 10**9), (10**12, 10**12 + 10**8), (7, 8), (100, 100)]:
        out.fill_(12345)
        sv210.count_dev(lo, hi, out)
        assert int(out.item()) == oracle.count(lo, hi)
    los, his = batch_intervals(4096, seed=1205)
    got = sv210.batch_count(los, his)
    with gb.Sieve(HI_MAX) as s30:
        assert got == s30.batch_count(los, his)


def test_w210_crossing_work_counts_multiples_coprime_to_210(sv210):
    # brute force of the definition on a small range
    lo, hi = 10**6, 10**6 + 5000
    primes = [p for p in range(23, 1001) if td_is_prime(p)]
    want = sum(1 for p in primes for m in range(max(p, -(-lo // p)), -(-hi // p))
               if m % 2 and m % 3 and m % 5 and m % 7)
    assert sv210.crossing_work(lo, hi) == want


def test_w210_pi_1e12_full_size(sv210):
    assert sv210.count(0, 10**12) == PI[10**12]
