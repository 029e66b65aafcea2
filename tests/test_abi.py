"""C-ABI library: loads, exports every declared symbol, host-side checks.

No GPU work: only calls that return before touching the device.
"""
import ctypes
import os
import re

import pytest

import paper_1012_2547_gb300 as smg
from paper_1012_2547_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(inc, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for mt in re.finditer(r"\b(sm_\w+)\s*\(", src):
            names.add(mt.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_lib.LIB_PATH):
        from paper_1012_2547_gb300 import build
        build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 19
    for name in names:
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"


def test_binding_declares_nothing_undeclared():
    assert set(_lib.SIGNATURES) <= declared_functions()


def test_strerror(lib):
    assert lib.sm_strerror(0) == b"success"
    assert lib.sm_strerror(5).startswith(b"more occurrences")
    assert lib.sm_strerror(99) == b"unknown status"


def test_host_argument_checks(lib):
    h = ctypes.c_void_p()
    assert lib.sm_prepare(None, 4, 0, None, ctypes.byref(h)) == _lib.SM_EINVAL
    assert lib.sm_prepare(b"abcd", 0, 0, None, ctypes.byref(h)) == _lib.SM_EINVAL
    assert lib.sm_search(None, 10, b"ab", 2, None, 0, None, None) == _lib.SM_EINVAL
    assert lib.sm_search(None, 0, b"", 0, None, 0, 8, None) == _lib.SM_EINVAL
    # misaligned count pointer
    assert lib.sm_search(None, 0, b"ab", 2, None, 0, 12, None) == _lib.SM_EINVAL
    # cap > 0 without an output array
    assert lib.sm_search(None, 0, b"ab", 2, None, 5, 16, None) == _lib.SM_EINVAL
    assert lib.sm_search_plan(None, None, 0, None, 0, 16, None) == _lib.SM_EINVAL
    assert lib.sm_plan_info(None, None) == _lib.SM_EINVAL
    assert lib.sm_batch_launch(None, None) == _lib.SM_EINVAL
    assert lib.sm_search_batch(None, 0, None) == _lib.SM_OK
    assert lib.sm_plan_free(None) == _lib.SM_OK
    assert lib.sm_batch_free(None) == _lib.SM_OK
    assert lib.sm_plan_free_many(None, 0) == _lib.SM_OK
    assert lib.sm_plan_free_many(None, 3) == _lib.SM_EINVAL
    nulls = (ctypes.c_void_p * 3)()
    assert lib.sm_plan_free_many(nulls, 3) == _lib.SM_OK  # null entries are skipped


def test_noalloc_host_checks(lib):
    """sm_search_noalloc rejects what it cannot serve before any CUDA call
    (on this CPU-only host any later step would fail with SM_ECUDA)."""
    f = lib.sm_search_noalloc
    fake = 1 << 20  # never dereferenced: the argument checks come first
    assert f(fake, 1000, bytes(65), 65, fake, 8, fake, None) == _lib.SM_EINVAL
    assert f(fake, 1000, b"", 0, fake, 8, fake, None) == _lib.SM_EINVAL
    assert f(None, 1000, b"ab", 2, fake, 8, fake, None) == _lib.SM_EINVAL
    assert f(fake, 1000, b"ab", 2, fake, 8, fake + 4, None) == _lib.SM_EINVAL
    longest = 65536 * 64 * 4608 - 16
    assert f(fake, longest + 1, b"ab", 2, fake, 8, fake, None) == _lib.SM_EINVAL
    assert f(fake, 1 << 62, b"ab", 2, fake, 8, fake, None) == _lib.SM_EINVAL
    # within limits the call proceeds to the device, which this host lacks
    assert f(fake, longest, b"ab", 2, fake, 8, fake, None) == _lib.SM_ECUDA


def test_tuning_table_roundtrip(lib):
    smg.tuning_reset()
    cells = smg.tuning_get()
    assert len(cells) == 12 * 9 and all(c["variant"] == 0 for c in cells)
    cells[3 * 9 + 2] = dict(variant=2, q=3, word_bits=0, tile=12)
    smg.tuning_set(cells)
    assert smg.tuning_get()[3 * 9 + 2] == dict(variant=2, q=3, word_bits=0, tile=12)
    smg.tuning_reset()
    assert smg.tuning_get()[3 * 9 + 2]["variant"] == 0
    with pytest.raises(ValueError):
        smg.tuning_set(cells[:5])
