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


def test_static_compaction_equals_sieve_compact_twice_in_a_row():
    with gb.Sieve(1 << 33) as sv:
        # two different ranges back to back: the second reuses the first's scratch contents
        _compare(sv, 0, 10**7)
        _compare(sv, 2**32 - 3 * 10**6 - 1, 2**32)
        _compare(sv, 0, 10**7)


def test_static_compaction_limits():
    # beyond the fixed scratch (more than [0, 2^32) of bitmap) -> ERANGE before any GPU work
    with pytest.raises(gb.SieveError) as e:
        gb.sieve_compact_static(None, 0, (1 << 32) + 64, None, 0)
    assert e.value.code == gb.SIEVE_ERANGE
    with pytest.raises(gb.SieveError) as e:
        gb.sieve_compact_static(None, 10, 5, None, 0)
    assert e.value.code == gb.SIEVE_EINVAL
    # ranges with no odd integer still report 2 correctly
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    n, rc = gb.sieve_compact_static(None, 2, 3, out, stream=gb.torch_stream_handle())
    assert rc == gb.SIEVE_OK and n == 1 and int(out[0].item()) == 2
    assert np.array_equal(out[1:].cpu().numpy(), np.zeros(3, dtype=np.int32))
