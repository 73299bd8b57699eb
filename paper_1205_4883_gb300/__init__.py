"""gbsieve: the segmented sieve of Eratosthenes on one GB300 (sm_103a).

A thin ctypes binding over ``libgbsieve.so`` (the C ABI in
``include/gbsieve.h``).  Functions keep the C names and only marshal
arguments: every step of the sieve runs in the library's CUDA kernels.
PyTorch supplies device memory (output tensors) and streams.  There is no CPU
fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgbsieve.so")

SIEVE_OK = 0
SIEVE_EINVAL = -1
SIEVE_ERANGE = -2
SIEVE_ETRUNC = -3
SIEVE_ENOMEM = -4
SIEVE_ECUDA = -5
SIEVE_ETIMEOUT = -6
SIEVE_EBUSY = -7
SIEVE_ENOENT = -8
SIEVE_EDEVICE = -9

SIEVE_PARAM_SEGMENT_BYTES = 1
SIEVE_PARAM_THREADS = 2
SIEVE_PARAM_SMALL_LIMIT = 3
SIEVE_PARAM_CTAS_PER_SM = 4
SIEVE_PARAM_CHUNK_SEGMENTS = 5
SIEVE_PARAM_BUCKET_LIMIT = 6
SIEVE_PARAM_CURSOR_MB = 7
SIEVE_PARAM_MR_PERCENT = 8
SIEVE_PARAM_MID_LIMIT = 9
SIEVE_PARAM_WHEEL = 10
SIEVE_PARAM_SMALL_LIMIT_210 = 11
SIEVE_PARAM_MID_LIMIT_210 = 12
SIEVE_PARAM_BATCH_ORDER = 13
SIEVE_PARAM_FAULT_WAIT = 14
SIEVE_PARAM_PRESIEVE = 15

SIEVE_PROBE_SMEM_AND_CONFLICT_FREE = 1
SIEVE_PROBE_SMEM_AND_RANDOM = 2
SIEVE_PROBE_SMEM_STORE_CONFLICT_FREE = 3
SIEVE_PROBE_HBM_WRITE = 4

_u64 = ctypes.c_uint64
_i64 = ctypes.c_int64
_vp = ctypes.c_void_p
_int = ctypes.c_int
_sz = ctypes.c_size_t
_pu64 = ctypes.POINTER(ctypes.c_uint64)
_pu32 = ctypes.POINTER(ctypes.c_uint32)


class sieve_info(ctypes.Structure):
    _fields_ = [("hi_max", _u64), ("prime_limit", _u64), ("n_base_primes", _u64),
                ("device", ctypes.c_int32), ("num_sms", ctypes.c_int32), ("device_bytes", _u64)]


class sieve_server_cfg(ctypes.Structure):
    _fields_ = [("max_requests", ctypes.c_uint32), ("tick_segments", ctypes.c_uint32),
                ("max_device_bytes", _u64), ("serial_ticks", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("host_arena_bytes", _u64)]


class sieve_req(ctypes.Structure):
    _fields_ = [("lo", _u64), ("hi", _u64), ("kind", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class sieve_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("kind", ctypes.c_int32), ("count", _u64),
                ("primes", ctypes.POINTER(_u64)), ("latency_us", ctypes.c_double),
                ("offsets", ctypes.POINTER(ctypes.c_uint32))]


class sieve_server_counters(ctypes.Structure):
    _fields_ = [("submitted", _u64), ("completed", _u64), ("rejected", _u64), ("ticks", _u64),
                ("integers", _u64), ("in_flight", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("device_bytes_reserved", _u64), ("segments", _u64), ("tick_gpu_ms", ctypes.c_double)]


class sieve_range_params(ctypes.Structure):
    _fields_ = [("seg_bytes", ctypes.c_uint32), ("wheel", ctypes.c_uint32), ("bucket_limit", _u64),
                ("mid_limit", ctypes.c_uint32), ("mr_percent", ctypes.c_uint32)]


SIEVE_REQ_COUNT = 0
SIEVE_REQ_LIST = 1
SIEVE_REQ_LIST_OFFSETS = 2
MR_NEVER = 0xFFFFFFFF

# name -> (restype, argtypes)
_SIGS = {
    "sieve_create": (_int, [ctypes.POINTER(_vp), _u64, _int, _vp]),
    "sieve_destroy": (None, [_vp]),
    "sieve_count": (_int, [_vp, _u64, _u64, _pu64]),
    "sieve_count_dev": (_int, [_vp, _u64, _u64, _vp]),
    "sieve_bitmap": (_int, [_vp, _u64, _u64, _vp, _sz, _pu64]),
    "sieve_bitmap_words": (_u64, [_u64, _u64]),
    "sieve_list": (_int, [_vp, _u64, _u64, _vp, _sz, _pu64]),
    "sieve_list64": (_int, [_vp, _u64, _u64, _vp, _sz, _pu64]),
    "sieve_compact": (_int, [_vp, _vp, _u64, _u64, _vp, _sz, _pu64]),
    "sieve_bitmap_dev": (_int, [_vp, _u64, _u64, _vp, _sz, _vp]),
    "sieve_compact_dev": (_int, [_vp, _vp, _u64, _u64, _vp, _sz, _vp]),
    "sieve_batch_count": (_int, [_vp, _pu64, _pu64, _sz, _pu64, ctypes.POINTER(_vp)]),
    "sieve_batch_count_params": (_int, [_vp, _pu64, _pu64, _sz, ctypes.POINTER(sieve_range_params), _pu64,
                                        ctypes.POINTER(_vp)]),
    "sieve_set_param": (_int, [_vp, _int, _i64]),
    "sieve_get_param": (_int, [_vp, _int, ctypes.POINTER(_i64)]),
    "sieve_get_info": (_int, [_vp, ctypes.POINTER(sieve_info)]),
    "sieve_base_primes": (_int, [_vp, _pu32, _sz, _pu64]),
    "sieve_crossing_work": (_int, [_vp, _u64, _u64, _pu64]),
    "sieve_crossing_work_ge": (_int, [_vp, _u64, _u64, _u64, _pu64]),
    "sieve_stream": (_vp, [_vp]),
    "sieve_strerror": (ctypes.c_char_p, [_int]),
    "sieve_last_error": (ctypes.c_char_p, [_vp]),
    "sieve_compact_static": (_int, [_vp, _u64, _u64, _vp, _sz, _pu64, _vp]),
    "sieve_server_create": (_int, [_vp, ctypes.POINTER(sieve_server_cfg), ctypes.POINTER(_vp)]),
    "sieve_server_submit": (_int, [_vp, ctypes.POINTER(sieve_req), _pu64]),
    "sieve_server_poll": (_int, [_vp, _u64, ctypes.POINTER(sieve_result), _i64]),
    "sieve_server_release": (_int, [_vp, _u64]),
    "sieve_server_wait_any": (_int, [_vp, _pu64, _sz, ctypes.POINTER(_sz), _i64]),
    "sieve_server_stats": (_int, [_vp, ctypes.POINTER(sieve_server_counters)]),
    "sieve_server_destroy": (None, [_vp]),
    "sieve_selftest_wait": (_int, [_vp, _int, ctypes.c_uint32, ctypes.POINTER(_int)]),
    "sieve_probe": (_int, [_vp, _int, _vp, _u64, ctypes.POINTER(ctypes.c_double)]),
}

_lib = None


def load_library(path: Optional[str] = None) -> ctypes.CDLL:
    """Load libgbsieve.so (building it first if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        from . import build as _build
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols() -> Sequence[str]:
    return tuple(_SIGS)


class SieveError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


def sieve_strerror(code: int) -> str:
    return load_library().sieve_strerror(code).decode()


def sieve_last_error(ctx: int) -> str:
    return load_library().sieve_last_error(ctx).decode()


def _check(ctx, rc: int, allow=()):
    if rc != SIEVE_OK and rc not in allow:
        lib = load_library()
        detail = lib.sieve_last_error(ctx).decode() if ctx else ""
        raise SieveError(rc, f"{lib.sieve_strerror(rc).decode()}: {detail}")
    return rc


def _ptr(t) -> int:
    """Device pointer of a CUDA tensor (or an int address / None)."""
    if t is None:
        return 0
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def sieve_create(hi_max: int, device: int = 0, stream: Optional[int] = None) -> int:
    lib = load_library()
    h = _vp()
    rc = lib.sieve_create(ctypes.byref(h), hi_max, device, stream or None)
    if rc != SIEVE_OK:
        raise SieveError(rc, f"sieve_create failed: {lib.sieve_strerror(rc).decode()}")
    return h.value


def sieve_destroy(ctx: int) -> None:
    load_library().sieve_destroy(ctx)


def sieve_count(ctx: int, lo: int, hi: int) -> int:
    c = _u64()
    _check(ctx, load_library().sieve_count(ctx, lo, hi, ctypes.byref(c)))
    return c.value


def sieve_count_dev(ctx: int, lo: int, hi: int, count_dev) -> None:
    _check(ctx, load_library().sieve_count_dev(ctx, lo, hi, _ptr(count_dev)))


def sieve_bitmap_words(lo: int, hi: int) -> int:
    return int(load_library().sieve_bitmap_words(lo, hi))


def sieve_bitmap(ctx: int, lo: int, hi: int, out, out_words: Optional[int] = None) -> int:
    """Odd-only bitmap into `out` (a CUDA int32/uint32 tensor or a device address); returns the count."""
    if out_words is None:
        out_words = out.numel() * out.element_size() // 4 if out is not None and not isinstance(out, int) else 0
    c = _u64()
    _check(ctx, load_library().sieve_bitmap(ctx, lo, hi, _ptr(out), out_words, ctypes.byref(c)))
    return c.value


def _list(fn, ctx, lo, hi, out, cap, elem):
    if cap is None:
        cap = out.numel() * out.element_size() // elem if out is not None and not isinstance(out, int) else 0
    n = _u64()
    rc = fn(ctx, lo, hi, _ptr(out), cap, ctypes.byref(n))
    _check(ctx, rc, allow=(SIEVE_ETRUNC,))
    return n.value, rc


def sieve_list(ctx: int, lo: int, hi: int, out, cap: Optional[int] = None):
    """uint32 prime list into `out`; returns (n, rc) with rc SIEVE_OK or SIEVE_ETRUNC."""
    return _list(load_library().sieve_list, ctx, lo, hi, out, cap, 4)


def sieve_list64(ctx: int, lo: int, hi: int, out, cap: Optional[int] = None):
    return _list(load_library().sieve_list64, ctx, lo, hi, out, cap, 8)


def sieve_compact(ctx: int, bitmap, lo: int, hi: int, out, cap: Optional[int] = None):
    if cap is None:
        cap = out.numel() * out.element_size() // 4 if out is not None and not isinstance(out, int) else 0
    n = _u64()
    rc = load_library().sieve_compact(ctx, _ptr(bitmap), lo, hi, _ptr(out), cap, ctypes.byref(n))
    _check(ctx, rc, allow=(SIEVE_ETRUNC,))
    return n.value, rc


def sieve_bitmap_dev(ctx: int, lo: int, hi: int, out, count_dev, out_words: Optional[int] = None) -> None:
    """Asynchronous sieve_bitmap: the count goes to the device integer `count_dev`
    (a one-element CUDA int64 tensor or a device address); nothing waits for the stream."""
    if out_words is None:
        out_words = out.numel() * out.element_size() // 4 if out is not None and not isinstance(out, int) else 0
    _check(ctx, load_library().sieve_bitmap_dev(ctx, lo, hi, _ptr(out), out_words, _ptr(count_dev)))


def sieve_compact_dev(ctx: int, bitmap, lo: int, hi: int, out, n_dev, cap: Optional[int] = None) -> None:
    """Asynchronous sieve_compact: the prime count goes to the device integer `n_dev`; the
    list is written only if it fits in `cap` (read n_dev after synchronising)."""
    if cap is None:
        cap = out.numel() * out.element_size() // 4 if out is not None and not isinstance(out, int) else 0
    _check(ctx, load_library().sieve_compact_dev(ctx, _ptr(bitmap), lo, hi, _ptr(out), cap, _ptr(n_dev)))


def sieve_compact_static(bitmap, lo: int, hi: int, out, cap: Optional[int] = None, stream: Optional[int] = None):
    """Compaction with the library's fixed scratch array (no device allocation).
    Returns (n, rc) with rc SIEVE_OK or SIEVE_ETRUNC; other codes raise."""
    if cap is None:
        cap = out.numel() * out.element_size() // 4 if out is not None and not isinstance(out, int) else 0
    n = _u64()
    rc = load_library().sieve_compact_static(_ptr(bitmap), lo, hi, _ptr(out), cap, ctypes.byref(n), stream or None)
    _check(0, rc, allow=(SIEVE_ETRUNC,))
    return n.value, rc


def sieve_selftest_wait(ctx: int, arm: bool, limit: int) -> bool:
    """Run the bounded device-wait self-test; True if the wait ran out."""
    out = _int()
    _check(ctx, load_library().sieve_selftest_wait(ctx, 1 if arm else 0, limit, ctypes.byref(out)))
    return bool(out.value)


def sieve_probe(ctx: int, kind: int, buf=None, nbytes: int = 0) -> float:
    """A roofline probe (SIEVE_PROBE_*): lane-ops per SM clock, or GB/s for the HBM write."""
    v = ctypes.c_double()
    if buf is not None and not isinstance(buf, int) and not nbytes:
        nbytes = buf.numel() * buf.element_size()
    _check(ctx, load_library().sieve_probe(ctx, kind, _ptr(buf), nbytes, ctypes.byref(v)))
    return v.value


def sieve_batch_count(ctx: int, lo: Sequence[int], hi: Sequence[int], bitmaps=None):
    """Counts of m ranges in one launch; `bitmaps` optionally a list of CUDA tensors (or None)."""
    import numpy as np
    m = len(lo)
    if len(hi) != m:
        raise ValueError("lo and hi differ in length")
    # contiguous uint64 arrays passed by pointer (no per-element ctypes conversion)
    lo_a = np.ascontiguousarray(lo, dtype=np.uint64) if m else np.zeros(1, np.uint64)
    hi_a = np.ascontiguousarray(hi, dtype=np.uint64) if m else np.zeros(1, np.uint64)
    cnt = np.zeros(max(m, 1), dtype=np.uint64)
    bm = None
    if bitmaps is not None:
        bm = (_vp * max(m, 1))(*[(_ptr(b) or None) for b in bitmaps])
    as_u64 = lambda a: a.ctypes.data_as(_pu64)  # noqa: E731
    _check(ctx, load_library().sieve_batch_count(ctx, as_u64(lo_a), as_u64(hi_a), m, as_u64(cnt), bm))
    return cnt[:m].tolist()


_RANGE_FIELDS = ("seg_bytes", "wheel", "bucket_limit", "mid_limit", "mr_percent")


def range_params_dtype():
    """numpy dtype with the layout of sieve_range_params."""
    import numpy as np
    dt = np.dtype([("seg_bytes", "<u4"), ("wheel", "<u4"), ("bucket_limit", "<u8"),
                   ("mid_limit", "<u4"), ("mr_percent", "<u4")])
    assert dt.itemsize == ctypes.sizeof(sieve_range_params)
    return dt


def range_params_array(params):
    """A sieve_range_params array from a sequence of dicts (missing fields: 0)."""
    import numpy as np
    pa = np.zeros(max(len(params), 1), dtype=range_params_dtype())
    for f in _RANGE_FIELDS:
        pa[f][:len(params)] = [int(p.get(f, 0) or 0) for p in params]
    return pa


def sieve_batch_count_params(ctx: int, lo: Sequence[int], hi: Sequence[int], params, bitmaps=None):
    """Counts of m ranges with per-range launch parameters, one graph launch.
    params: a sieve_range_params array (range_params_array) or a sequence of m
    dicts with any of seg_bytes, wheel, bucket_limit, mid_limit, mr_percent
    (missing or 0: the context's value)."""
    import numpy as np
    m = len(lo)
    if len(hi) != m or len(params) < m:
        raise ValueError("lo, hi and params differ in length")
    lo_a = np.ascontiguousarray(lo, dtype=np.uint64) if m else np.zeros(1, np.uint64)
    hi_a = np.ascontiguousarray(hi, dtype=np.uint64) if m else np.zeros(1, np.uint64)
    cnt = np.zeros(max(m, 1), dtype=np.uint64)
    if isinstance(params, np.ndarray) and params.dtype == range_params_dtype():
        pa = np.ascontiguousarray(params)
    else:
        pa = range_params_array(params)
    bm = None
    if bitmaps is not None:
        bm = (_vp * max(m, 1))(*[(_ptr(b) or None) for b in bitmaps])
    as_u64 = lambda a: a.ctypes.data_as(_pu64)  # noqa: E731
    _check(ctx, load_library().sieve_batch_count_params(
        ctx, as_u64(lo_a), as_u64(hi_a), m, pa.ctypes.data_as(ctypes.POINTER(sieve_range_params)),
        as_u64(cnt), bm))
    return cnt[:m].tolist()


def sieve_set_param(ctx: int, param: int, value: int) -> None:
    _check(ctx, load_library().sieve_set_param(ctx, param, value))


def sieve_get_param(ctx: int, param: int) -> int:
    v = _i64()
    _check(ctx, load_library().sieve_get_param(ctx, param, ctypes.byref(v)))
    return v.value


def sieve_get_info(ctx: int) -> sieve_info:
    info = sieve_info()
    _check(ctx, load_library().sieve_get_info(ctx, ctypes.byref(info)))
    return info


def sieve_base_primes(ctx: int):
    import numpy as np
    n = _u64()
    lib = load_library()
    _check(ctx, lib.sieve_base_primes(ctx, None, 0, ctypes.byref(n)))
    out = np.zeros(max(n.value, 1), dtype=np.uint32)
    _check(ctx, lib.sieve_base_primes(ctx, out.ctypes.data_as(_pu32), n.value, ctypes.byref(n)))
    return out[:n.value]


def sieve_crossing_work(ctx: int, lo: int, hi: int) -> int:
    c = _u64()
    _check(ctx, load_library().sieve_crossing_work(ctx, lo, hi, ctypes.byref(c)))
    return c.value


def sieve_crossing_work_ge(ctx: int, lo: int, hi: int, pmin: int) -> int:
    c = _u64()
    _check(ctx, load_library().sieve_crossing_work_ge(ctx, lo, hi, pmin, ctypes.byref(c)))
    return c.value


def sieve_stream(ctx: int) -> int:
    return load_library().sieve_stream(ctx) or 0


def sieve_server_create(ctx: int, max_requests: int = 0, tick_segments: int = 0, max_device_bytes: int = 0,
                        serial_ticks: bool = False, host_arena_bytes: int = 0) -> int:
    cfg = sieve_server_cfg(max_requests, tick_segments, max_device_bytes, 1 if serial_ticks else 0, 0,
                           host_arena_bytes)
    h = _vp()
    rc = load_library().sieve_server_create(ctx, ctypes.byref(cfg), ctypes.byref(h))
    _check(ctx, rc)
    return h.value


def sieve_server_submit(srv: int, lo: int, hi: int, kind: int = SIEVE_REQ_COUNT):
    """Returns (rc, ticket); rc is SIEVE_OK or SIEVE_EBUSY (other codes raise)."""
    req = sieve_req(lo, hi, kind, 0)
    t = _u64()
    rc = load_library().sieve_server_submit(srv, ctypes.byref(req), ctypes.byref(t))
    _check(0, rc, allow=(SIEVE_EBUSY,))
    return rc, t.value


def sieve_server_poll(srv: int, ticket: int, timeout_us: int = -1, copy_primes: bool = True):
    """Returns (rc, result dict or None); rc SIEVE_OK or SIEVE_ETIMEOUT (others raise).
    A list result's primes (or, for SIEVE_REQ_LIST_OFFSETS, their uint32 offsets from lo,
    under "offsets") are copied out of the server's memory (unless copy_primes is False,
    when only the count is returned)."""
    res = sieve_result()
    rc = load_library().sieve_server_poll(srv, ticket, ctypes.byref(res), timeout_us)
    _check(0, rc, allow=(SIEVE_ETIMEOUT,))
    if rc != SIEVE_OK:
        return rc, None
    out = {"status": res.status, "kind": res.kind, "count": int(res.count), "latency_us": res.latency_us,
           "primes": None, "offsets": None}
    if copy_primes and res.kind == SIEVE_REQ_LIST and res.status == SIEVE_OK:
        import numpy as np
        n = int(res.count)
        out["primes"] = (np.ctypeslib.as_array(res.primes, shape=(n,)).copy() if n
                         else np.zeros(0, dtype=np.uint64))
    if copy_primes and res.kind == SIEVE_REQ_LIST_OFFSETS and res.status == SIEVE_OK:
        import numpy as np
        n = int(res.count)
        out["offsets"] = (np.ctypeslib.as_array(res.offsets, shape=(n,)).copy() if n
                          else np.zeros(0, dtype=np.uint32))
    return rc, out


def sieve_server_wait_any(srv: int, cap: int = 1024, timeout_us: int = -1):
    """Tickets of requests completed since the last call (up to cap); [] on timeout."""
    import numpy as np
    out = np.zeros(max(cap, 1), dtype=np.uint64)
    n = _sz()
    rc = load_library().sieve_server_wait_any(srv, out.ctypes.data_as(_pu64), cap, ctypes.byref(n), timeout_us)
    _check(0, rc, allow=(SIEVE_ETIMEOUT,))
    return out[:n.value].tolist()


def sieve_server_release(srv: int, ticket: int) -> int:
    rc = load_library().sieve_server_release(srv, ticket)
    _check(0, rc, allow=(SIEVE_EBUSY, SIEVE_ENOENT))
    return rc


def sieve_server_stats(srv: int) -> dict:
    c = sieve_server_counters()
    _check(0, load_library().sieve_server_stats(srv, ctypes.byref(c)))
    return {k: getattr(c, k) for k, _ in sieve_server_counters._fields_ if k != "reserved"}


def sieve_server_destroy(srv: int) -> None:
    load_library().sieve_server_destroy(srv)


class Server:
    """A continuous-batching request server on a Sieve context."""

    def __init__(self, sieve: "Sieve", max_requests: int = 0, tick_segments: int = 0, max_device_bytes: int = 0,
                 serial_ticks: bool = False, host_arena_bytes: int = 0):
        self.sieve = sieve  # keeps the context alive
        self.srv = sieve_server_create(sieve.ctx, max_requests, tick_segments, max_device_bytes, serial_ticks,
                                       host_arena_bytes)

    def submit(self, lo, hi, kind=SIEVE_REQ_COUNT):
        return sieve_server_submit(self.srv, lo, hi, kind)

    def poll(self, ticket, timeout_us=-1, copy_primes=True):
        return sieve_server_poll(self.srv, ticket, timeout_us, copy_primes)

    def release(self, ticket):
        return sieve_server_release(self.srv, ticket)

    def wait_any(self, cap=1024, timeout_us=-1):
        return sieve_server_wait_any(self.srv, cap, timeout_us)

    def stats(self):
        return sieve_server_stats(self.srv)

    def close(self):
        if self.srv:
            sieve_server_destroy(self.srv)
            self.srv = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# cudaStreamLegacy: the device's legacy default stream, shared with torch.
CUDA_STREAM_LEGACY = 1


def torch_stream_handle() -> int:
    """torch's current stream as a cudaStream_t value (legacy default -> 1)."""
    import torch
    h = torch.cuda.current_stream().cuda_stream
    return h if h else CUDA_STREAM_LEGACY


class Sieve:
    """Owns a sieve context; methods mirror the C calls without the ctx argument.

    By default the context runs on torch's current stream, so tensors torch
    fills or reads are ordered with the sieve's kernels."""

    def __init__(self, hi_max: int, device: int = 0, stream: Optional[int] = None):
        if stream is None:
            import torch
            with torch.cuda.device(device):
                stream = torch_stream_handle()
        self.ctx = sieve_create(hi_max, device, stream)

    def close(self):
        if self.ctx:
            sieve_destroy(self.ctx)
            self.ctx = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def count(self, lo, hi):
        return sieve_count(self.ctx, lo, hi)

    def count_dev(self, lo, hi, out):
        return sieve_count_dev(self.ctx, lo, hi, out)

    def bitmap(self, lo, hi, out=None):
        import torch
        if out is None:
            out = torch.zeros(max(sieve_bitmap_words(lo, hi), 1), dtype=torch.int32, device="cuda")
        c = sieve_bitmap(self.ctx, lo, hi, out)
        return out[:sieve_bitmap_words(lo, hi)], c

    def primes(self, lo, hi, dtype64: bool = False):
        import torch
        fn = sieve_list64 if dtype64 else sieve_list
        n, _ = fn(self.ctx, lo, hi, None, 0)
        out = torch.empty(max(n, 1), dtype=torch.int64 if dtype64 else torch.int32, device="cuda")
        n2, rc = fn(self.ctx, lo, hi, out)
        assert rc == SIEVE_OK and n2 == n
        return out[:n]

    def batch_count(self, lo, hi, bitmaps=None):
        return sieve_batch_count(self.ctx, lo, hi, bitmaps)

    _PARAM_IDS = {"segment_bytes": SIEVE_PARAM_SEGMENT_BYTES, "threads": SIEVE_PARAM_THREADS,
                  "small_limit": SIEVE_PARAM_SMALL_LIMIT, "ctas_per_sm": SIEVE_PARAM_CTAS_PER_SM,
                  "chunk_segments": SIEVE_PARAM_CHUNK_SEGMENTS, "bucket_limit": SIEVE_PARAM_BUCKET_LIMIT,
                  "cursor_mb": SIEVE_PARAM_CURSOR_MB, "mr_percent": SIEVE_PARAM_MR_PERCENT,
                  "mid_limit": SIEVE_PARAM_MID_LIMIT, "wheel": SIEVE_PARAM_WHEEL,
                  "small_limit_210": SIEVE_PARAM_SMALL_LIMIT_210, "mid_limit_210": SIEVE_PARAM_MID_LIMIT_210,
                  "batch_order": SIEVE_PARAM_BATCH_ORDER, "presieve": SIEVE_PARAM_PRESIEVE}

    def apply_plan(self, plan: dict) -> None:
        """Set the launch parameters of an autotuned plan (see autotune.py)."""
        for k, v in plan.items():
            if k in self._PARAM_IDS:
                sieve_set_param(self.ctx, self._PARAM_IDS[k], int(v))

    def batch_count_params(self, lo, hi, params, bitmaps=None):
        return sieve_batch_count_params(self.ctx, lo, hi, params, bitmaps)

    def batch_count_tuned(self, lo, hi, table=None, bitmaps=None):
        """Counts of many ranges, each sieved with the launch parameters the
        autotuner chose for its size class, all in one graph launch."""
        from . import autotune
        table = table if table is not None else autotune.load_table()
        return sieve_batch_count_params(self.ctx, lo, hi, autotune.range_params_array(table, lo, hi), bitmaps)

    def set_param(self, param, value):
        sieve_set_param(self.ctx, param, value)

    def get_param(self, param):
        return sieve_get_param(self.ctx, param)

    def info(self):
        return sieve_get_info(self.ctx)

    def base_primes(self):
        return sieve_base_primes(self.ctx)

    def crossing_work(self, lo, hi, pmin=None):
        if pmin is None:
            return sieve_crossing_work(self.ctx, lo, hi)
        return sieve_crossing_work_ge(self.ctx, lo, hi, pmin)

    def stream(self):
        return sieve_stream(self.ctx)
