"""sieve_compact_static: the compaction for callers that cannot allocate device
memory (its scratch is a fixed array inside the library).  Its output must
equal sieve_compact's, call after call, even though every call reuses the same
array.  This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only hosts
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import oracle_pool  # noqa: E402
import paper_1205_4883_gb300 as gb  # noqa: E402


def _compare(sv, lo, hi):
    nw = gb.sieve_bitmap_words(lo, hi)
    bm = torch.zeros(max(nw, 1), dtype=torch.int32, device="cuda")
    gb.sieve_bitmap(sv.ctx, lo, hi, bm)
    n_ref, rc = gb.sieve_compact(sv.ctx, bm, lo, hi, None, 0)
    ref = torch.zeros(max(n_ref, 1), dtype=torch.int32, device="cuda")
    n_ref2, rc = gb.sieve_compact(sv.ctx, bm, lo, hi, ref)
    assert rc == gb.SIEVE_OK and n_ref2 == n_ref
    stream = gb.torch_stream_handle()
    # size query, then the real call into a buffer pre-filled with junk
    n_q, rc = gb.sieve_compact_static(bm, lo, hi, None, 0, stream=stream)
    assert n_q == n_ref and (rc == gb.SIEVE_ETRUNC or n_ref == 0)
    out = torch.full((max(n_ref, 1),), -7, dtype=torch.int32, device="cuda")
    n, rc = gb.sieve_compact_static(bm, lo, hi, out, stream=stream)
    assert rc == gb.SIEVE_OK and n == n_ref
    assert torch.equal(out[:n], ref[:n_ref])
    return out[:n]


def test_static_compaction_equals_sieve_compact_twice_in_a_row():
    with gb.Sieve(1 << 33) as sv:
        # two different ranges back to back: the second reuses the first's scratch contents
        for lo, hi in ((0, 10**7), (2**32 - 3 * 10**6 - 1, 2**32), (0, 10**7)):
            got = _compare(sv, lo, hi).cpu().numpy().view(np.uint32).astype(np.uint64)
            assert np.array_equal(got, oracle.primes(lo, hi)), (lo, hi)


def test_static_compaction_at_its_maximum_size():
    # [0, 2^32): the documented maximum, where every byte of the fixed scratch is written;
    # the list against sieve_compact and, entry by entry, against the oracle
    lo, hi = 0, 1 << 32
    with gb.Sieve(1 << 33) as sv:
        got = _compare(sv, lo, hi).cpu().numpy().view(np.uint32)
    assert len(got) == 203_280_221
    total, bad = oracle_pool.compare_list(got, lo, hi)
    assert total == len(got) and bad == []


def test_static_compaction_limits():
    # beyond the fixed scratch (more than [0, 2^32) of bitmap) -> ERANGE before any GPU work
    with pytest.raises(gb.SieveError) as e:
        gb.sieve_compact_static(None, 0, (1 << 32) + 64, None, 0)
    assert e.value.code == gb.SIEVE_ERANGE
    with pytest.raises(gb.SieveError) as e:
        gb.sieve_compact_static(None, 10, 5, None, 0)
    assert e.value.code == gb.SIEVE_EINVAL
    # a null output with a nonzero capacity, and a null bitmap for a nonempty range:
    # EINVAL before any GPU work (as sieve_compact)
    with pytest.raises(gb.SieveError) as e:
        gb.sieve_compact_static(None, 0, 10**6, None, 10)
    assert e.value.code == gb.SIEVE_EINVAL
    out1 = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(gb.SieveError) as e:
        gb.sieve_compact_static(None, 0, 10**6, out1, 4)
    assert e.value.code == gb.SIEVE_EINVAL
    with gb.Sieve(1 << 20) as sv:
        bm = torch.zeros(gb.sieve_bitmap_words(0, 10**6), dtype=torch.int32, device="cuda")
        with pytest.raises(gb.SieveError) as e:
            gb.sieve_compact(sv.ctx, bm, 0, 10**6, None, 10)
        assert e.value.code == gb.SIEVE_EINVAL
    # ranges with no odd integer still report 2 correctly
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    n, rc = gb.sieve_compact_static(None, 2, 3, out, stream=gb.torch_stream_handle())
    assert rc == gb.SIEVE_OK and n == 1 and int(out[0].item()) == 2
    assert np.array_equal(out[1:].cpu().numpy(), np.zeros(3, dtype=np.int32))
