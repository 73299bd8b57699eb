"""The C-ABI library builds, loads, and exports every symbol include/*.h
declares; the Python binding names the same calls.  No GPU needed (no compute
calls are made)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_ \*]*?)\b(sieve_[a-z0-9_]+)\s*\(", text):
            names.append(m.group(2))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1205_4883_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("sieve_create", "sieve_destroy", "sieve_count", "sieve_bitmap", "sieve_list",
              "sieve_list64", "sieve_batch_count", "sieve_strerror"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(sieve_\w+)", out))
    assert set(declared_functions()) <= exported


def test_binding_covers_the_header():
    import paper_1205_4883_gb300 as g
    assert set(declared_functions()) <= set(g.exported_symbols())
    for n in declared_functions():
        if n in g.exported_symbols():
            assert hasattr(g, n), n


def test_host_only_calls_without_gpu(lib):
    import paper_1205_4883_gb300 as g
    g.load_library()
    assert g.sieve_strerror(0) == "ok"
    assert g.sieve_strerror(-3) == "output truncated"
    assert g.sieve_bitmap_words(0, 10**7) == (5 * 10**6 + 31) // 32
    assert g.sieve_bitmap_words(4, 5) == 0
    assert g.sieve_bitmap_words(0, 3) == 1
    # invalid arguments are rejected before any device work
    h = ctypes.c_void_p()
    assert g.load_library().sieve_create(ctypes.byref(h), 1, 0, None) == g.SIEVE_ERANGE
    assert g.load_library().sieve_create(ctypes.byref(h), (1 << 62) + 1, 0, None) == g.SIEVE_ERANGE
    assert g.load_library().sieve_create(None, 100, 0, None) == g.SIEVE_EINVAL


def test_kernels_are_built_for_sm103a():
    from paper_1205_4883_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
