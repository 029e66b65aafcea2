"""Host logic of the plan builder, on the CPU: every table of a plan's
device image (sm_plan_image, no CUDA call) against its definition --
Shift-And masks (Section 1), the Knuth-Morris-Pratt border table, the
exact q-gram table, and the string-matching automaton (its transitions by
brute force, and its matches against the oracle)."""
import itertools

import numpy as np
import pytest

import oracle

from _helpers import DFA_MAX_TABLE

smg = pytest.importorskip("paper_1012_2547_gb300")


@pytest.fixture(scope="module", autouse=True)
def built_library():
    import os
    if not os.path.exists(smg._lib.LIB_PATH):
        from paper_1012_2547_gb300 import build
        build.build()


def image(p, **kw):
    return smg.plan_image(p, **kw)


def u16(img, off, count):
    return np.frombuffer(img[off: off + 2 * count].tobytes(), dtype="<u2")


def u32(img, off, count):
    return np.frombuffer(img[off: off + 4 * count].tobytes(), dtype="<u4")


def patterns(rng, m, sigma, k=3):
    out = [bytes(rng.integers(0, sigma, m, dtype=np.uint8)) for _ in range(k)]
    out.append(bytes(m))                                       # a^m
    out.append((b"ab" * m)[:m])                                # period 2
    return out


def brute_border(p):
    """fail[q] = length of the longest proper border of p[:q], by trying every length."""
    return [0] + [max(k for k in range(q) if p[:k] == p[q - k: q]) for q in range(1, len(p) + 1)]


def brute_delta(p, q, c):
    """Longest prefix of p that is a suffix of p[:q] + c (at most m)."""
    s = p[:q] + bytes([c])
    for k in range(min(len(s), len(p)), -1, -1):
        if s.endswith(p[:k]):
            return k
    return 0


def test_image_size_query_and_capacity():
    lib = smg._lib.load()
    import ctypes
    lay = smg._lib.sm_plan_layout()
    assert lib.sm_plan_image(b"abc", 3, 0, None, None, 0, ctypes.byref(lay)) == 0
    assert lay.bytes > 0 and lay.bytes % 256 == 0
    buf = (ctypes.c_uint8 * (lay.bytes - 1))()
    assert lib.sm_plan_image(b"abc", 3, 0, None, buf, lay.bytes - 1, ctypes.byref(lay)) == 1  # SM_EINVAL
    assert lib.sm_plan_image(b"abc", 0, 0, None, None, 0, ctypes.byref(lay)) == 1
    assert lib.sm_plan_image(b"abc", 3, 0, None, None, 0, None) == 1


@pytest.mark.parametrize("m", [1, 2, 5, 8, 9, 16, 17, 31, 32, 33, 49, 50, 64])
def test_shiftand_masks_are_the_definition(m):
    """bit j (j < m) of mask c is [p[j] == c]; every bit >= m is 1."""
    rng = np.random.default_rng(m)
    for p in patterns(rng, m, 4):
        for wb in ((32, 64) if m <= 32 else (64,)):
            img, lay = image(p, variant="shiftor", word_bits=wb)
            assert lay["variant"] == "shiftor" and lay["word_bits"] == wb
            esz = lay["entry_bytes"]
            full = (1 << (8 * esz)) - 1
            raw = img[lay["off_masks"]: lay["off_masks"] + 256 * esz].reshape(256, esz)
            got = [int.from_bytes(bytes(row), "little") for row in raw]
            low = (1 << m) - 1
            for c in range(256):
                bits = sum(1 << j for j in range(m) if p[j] == c)
                assert got[c] == full & (~low | bits), (p, wb, c)
            assert bytes(img[lay["off_pattern"]: lay["off_pattern"] + m]) == p


def test_border_table_is_the_longest_proper_border():
    rng = np.random.default_rng(2)
    cases = [bytes(x) for n in range(1, 9) for x in itertools.product(b"ab", repeat=n)]
    cases += [p for m in (20, 65, 130) for p in patterns(rng, m, 3)]
    for p in cases:
        img, lay = image(p)
        assert list(u32(img, lay["off_border"], len(p) + 1)) == brute_border(p), p


@pytest.mark.parametrize("m,q", [(17, 3), (40, 8), (65, 5), (300, 8), (1024, 4)])
def test_qgram_table_is_exact(m, q):
    """Every key's offsets are exactly the j with p[j:j+q] = key, in
    decreasing order; every q-gram of p is a key; the bitmap has each key's bit."""
    rng = np.random.default_rng(m * 10 + q)
    for p in patterns(rng, m, 4) + patterns(rng, m, 200, k=1)[:1]:
        img, lay = image(p, variant="qgram", q=q)
        assert lay["variant"] == "qgram" and lay["q"] == q and lay["s"] == m - q + 1
        want = {}
        for j in range(m - q + 1):
            want.setdefault(int.from_bytes(p[j: j + q], "little"), []).append(j)
        nslots = 1 << lay["slot_bits"]
        assert nslots >= 2 * len(want)
        slots = np.frombuffer(img[lay["off_qgram_slots"]: lay["off_qgram_slots"] + 16 * nslots].tobytes(),
                              dtype=np.dtype([("key", "<u8"), ("first", "<u4"), ("count", "<u4")]))
        offs = u32(img, lay["off_qgram_offsets"], m - q + 1)
        bitmap = u32(img, lay["off_qgram_bitmap"], (1 << lay["bitmap_bits"]) // 32)
        got = {}
        bits = set()
        for sl in slots[slots["count"] > 0]:
            key = int(sl["key"])
            assert key not in got
            got[key] = list(offs[sl["first"]: sl["first"] + sl["count"]])
            h = (((key & 0xFFFFFFFF) * 0x9E3779B1) ^ ((key >> 32) * 0x85EBCA77)) & 0xFFFFFFFF
            b = h >> (32 - lay["bitmap_bits"])
            assert (int(bitmap[b >> 5]) >> (b & 31)) & 1
            bits.add(b)
        assert got == {k: sorted(v, reverse=True) for k, v in want.items()}
        assert sum(bin(int(w)).count("1") for w in bitmap) == len(bits)   # no other bit set


def simulate(img, lay, text):
    """Run the image's automaton over text from state 0; positions where it
    reaches state m are ends of occurrences."""
    cls = u16(img, lay["off_classes_tab"], 256)
    C, m = lay["classes"], lay["m"]
    tab = u16(img, lay["off_automaton"], (m + 1) * C)
    fin, r, out = 2 * C * m, 0, []
    for e, c in enumerate(text):
        r = int(tab[(r + int(cls[c])) // 2])
        if r == fin:
            out.append(e - m + 1)
    return np.array(out, dtype=np.uint64)


def test_automaton_transitions_by_brute_force():
    """delta(q, c) = longest prefix of p that is a suffix of p[:q] c, for
    every state and byte; bytes absent from p form class 0 (to state 0)."""
    rng = np.random.default_rng(4)
    cases = [bytes(x) for n in range(1, 7) for x in itertools.product(b"ab", repeat=n)]
    cases += [p for m in (7, 12) for p in patterns(rng, m, 3)] + [b"abcabcab", b"aabaabaaab"]
    for p in cases:
        img, lay = image(p, variant="dfa")
        assert lay["variant"] == "dfa"
        m, C = len(p), lay["classes"]
        assert C == len(set(p)) + 1
        cls = u16(img, lay["off_classes_tab"], 256)
        tab = u16(img, lay["off_automaton"], (m + 1) * C)
        for c in range(256):
            assert (cls[c] == 0) == (c not in p)
        for q in range(m + 1):
            for c in sorted(set(p)) + [next(x for x in range(256) if x not in p)]:
                got = int(tab[q * C + int(cls[c]) // 2])
                assert got == 2 * C * brute_delta(p, q, c), (p, q, c)


def test_automaton_matches_the_oracle():
    rng = np.random.default_rng(5)
    for sigma in (2, 3, 4):
        t = rng.integers(0, sigma, 20_000, dtype=np.uint8)
        t[5000:6000] = 0
        for m in (1, 2, 5, 13, 40):
            for p in patterns(rng, m, sigma, k=2) + [bytes(t[100: 100 + m])]:
                img, lay = image(p, variant="dfa")
                assert np.array_equal(simulate(img, lay, t), oracle.naive(t, p)), (sigma, p)


def test_automaton_rules():
    """DFA plans need (m+1) x C x 2 <= 32,512 bytes; q-gram plans carry the
    automaton exactly for periodic patterns (period <= m/2) that fit."""
    big = bytes(range(256)) * 4
    with pytest.raises(smg.SmError):
        image(big, variant="dfa")
    assert (len(big) + 1) * 257 * 2 > DFA_MAX_TABLE
    m = 8127
    assert (m + 1) * 2 * 2 <= DFA_MAX_TABLE
    _, lay = image(bytes(m), variant="dfa")
    assert lay["classes"] == 2
    with pytest.raises(smg.SmError):
        image(bytes(m + 1), variant="dfa")
    _, lay = image(bytes(300), variant="qgram", q=8)
    assert lay["off_automaton"] and lay["classes"] == 2                 # period 1
    _, lay = image(b"ab" * 150, variant="qgram", q=8)
    assert lay["off_automaton"] and lay["classes"] == 3                 # period 2
    _, lay = image(bytes(299) + b"\x01", variant="qgram", q=8)
    assert lay["off_automaton"] == 0                                    # period 300 > 150
    _, lay = image(bytes(range(200)) * 2, variant="qgram", q=8)
    assert lay["off_automaton"] == 0                                    # periodic, table too big
    _, lay = image(bytes(300), variant="linear")
    assert lay["off_automaton"] == 0                                    # KMP plans: none


def test_tile_sizes():
    for m in (1, 100, 1024, 3000):
        _, lay = image(bytes(m), variant="dfa")
        assert lay["tile_starts"] == 128 * ((max(1024, m) + 15) // 16 * 16)
    _, lay = image(bytes(10), variant="dfa", tile=14)
    assert lay["tile_starts"] == 128 * (1 << 14)
    _, lay = image(bytes(10), variant="shiftor")
    assert lay["tile_starts"] == 32 * 144
