"""Pins for the CPU oracle (no GPU).

The oracle is the problem statement of Section 1 written out (all start
positions i with t[i..i+m-1] = p).  These tests tie it to things other than
itself: an exhaustive integer-window formulation over every binary pair with
n <= 12, closed forms, Python's own substring search routines, hand-derived
fixtures, and planted mutations that each pin must catch.
"""
import os
import re
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_1012_2547_gb300 import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def find_all_bytes(text: bytes, pat: bytes) -> list[int]:
    """Overlapping occurrences by repeated bytes.find (library routine)."""
    out, i = [], text.find(pat)
    while i >= 0:
        out.append(i)
        i = text.find(pat, i + 1)
    return out


def find_all_re(text: bytes, pat: bytes) -> list[int]:
    """Overlapping occurrences by a zero-width lookahead regex."""
    return [mt.start() for mt in re.finditer(b"(?=" + re.escape(pat) + b")", text)]


def windows_equal(text: np.ndarray, pat: np.ndarray) -> list[int]:
    """Sliding-window equality with numpy (vectorised formulation)."""
    m = len(pat)
    if m > len(text):
        return []
    w = np.lib.stride_tricks.sliding_window_view(text, m)
    return np.flatnonzero(np.all(w == pat[None, :], axis=1)).tolist()


def read_handworked():
    rows = []
    with open(os.path.join(GOLDEN, "handworked.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            t, p, pos = line.rstrip("\n").split("\t")
            exp = [] if pos == "-" else [int(x) for x in pos.split(",")]
            rows.append((t.encode(), p.encode(), exp))
    return rows


def expected_binary_masks(n: int, m: int) -> np.ndarray:
    """Hit bitmask for every (text, pattern) over {0,1} from integer windows.

    Text and pattern are integers whose bit j is symbol j.  Position i is a
    hit iff bits i..i+m-1 of the text, read as an integer, equal the pattern.
    """
    tv = np.arange(1 << n, dtype=np.int64)
    out = np.zeros((1 << n, 1 << m), dtype=np.uint32)
    mask = (1 << m) - 1
    for i in range(n - m + 1):
        win = (tv >> i) & mask
        out[tv, win] |= np.uint32(1 << i)
    return out


# ---------------------------------------------------------------- pins


def pin_handworked(lib):
    for t, p, exp in read_handworked():
        for fn in (oracle.naive, oracle.kmp):
            got = fn(t, p, lib=lib).tolist()
            if got != exp:
                return f"{fn.__name__}({t!r}, {p!r}) = {got} != {exp}"
    return None


def pin_exhaustive_binary(lib, nmax):
    for n in range(1, nmax + 1):
        for m in range(1, n + 1):
            exp = expected_binary_masks(n, m)
            for which in ("naive", "kmp"):
                got = oracle.binary_masks(n, m, which, lib=lib)
                if not np.array_equal(got, exp):
                    bad = np.argwhere(got != exp)[0]
                    return f"{which} n={n} m={m} text={bad[0]:b} pat={bad[1]:b}"
    return None


def pin_closed_forms(lib):
    for n in (1, 2, 7, 64, 257):
        for m in (1, 2, 5, 64, 300):
            t = bytes(n) if n else b""
            p = bytes(m)
            exp = list(range(n - m + 1)) if m <= n else []
            for fn in (oracle.naive, oracle.kmp):
                if fn(t, p, lib=lib).tolist() != exp:
                    return f"a^{m} in a^{n} via {fn.__name__}"
    rng = np.random.default_rng(5)
    t = rng.integers(0, 4, 5000, dtype=np.uint8)
    for c in range(5):
        exp = np.flatnonzero(t == c).tolist()
        for fn in (oracle.naive, oracle.kmp):
            if fn(t, bytes([c]), lib=lib).tolist() != exp:
                return f"m=1 symbol {c} via {fn.__name__}"
    # A pattern holding a byte absent from the text has no occurrence.
    for fn in (oracle.naive, oracle.kmp):
        if fn(t, bytes([0, 1, 9, 2]), lib=lib).size:
            return "absent symbol"
    return None


def pin_library_routines(lib, cases=300, seed=3):
    rng = np.random.default_rng(seed)
    for k in range(cases):
        sigma = int(rng.choice([2, 3, 4, 26, 256]))
        n = int(rng.integers(0, 400))
        m = int(rng.integers(1, 12))
        t = rng.integers(0, sigma, n, dtype=np.uint8)
        if n >= m and rng.random() < 0.5:
            o = int(rng.integers(0, n - m + 1))
            p = t[o : o + m].copy()
        else:
            p = rng.integers(0, sigma, m, dtype=np.uint8)
        exp = find_all_bytes(t.tobytes(), p.tobytes())
        if exp != find_all_re(t.tobytes(), p.tobytes()) or exp != windows_equal(t, p):
            return "library routines disagree (test bug)"
        for fn in (oracle.naive, oracle.kmp):
            if fn(t, p, lib=lib).tolist() != exp:
                return f"{fn.__name__} case {k} sigma={sigma} n={n} m={m}"
        if oracle.naive_mt(t, p, threads=3, lib=lib).tolist() != exp:
            return f"naive_mt case {k}"
    return None


# ---------------------------------------------------------------- tests


def test_handworked_fixtures():
    assert pin_handworked(oracle.load()) is None


def test_exhaustive_binary_pairs_n_le_12():
    """Every binary text of length n <= 12 with every pattern of length m <= n."""
    assert pin_exhaustive_binary(oracle.load(), 12) is None


def test_closed_forms():
    assert pin_closed_forms(oracle.load()) is None


def test_library_routines():
    assert pin_library_routines(oracle.load()) is None


def test_threaded_matches_single_on_sweep_text():
    spec = gen.uniform_text(1 << 18, 2, seed=1)
    t = spec.host()
    for m in (1, 2, 3, 8, 17):
        p = gen.substring_patterns(t, m, 1, seed=m)[0]
        a = oracle.naive(t, p)
        for th in (1, 2, 7, 16):
            assert np.array_equal(oracle.naive_mt(t, p, threads=th), a)
        assert np.array_equal(oracle.kmp(t, p), a)
        assert oracle.count_mt(t, p, threads=4) == a.size


def test_planted_occurrences_found():
    rng = np.random.default_rng(9)
    t = rng.integers(0, 128, 100_000, dtype=np.uint8)
    p = rng.integers(128, 256, 40, dtype=np.uint8)  # bytes absent from t
    offs = sorted(set(int(x) for x in rng.integers(0, len(t) - 40, 50)))
    keep = []
    for o in offs:  # plant non-overlapping copies
        if not keep or o >= keep[-1] + 40:
            t[o : o + 40] = p
            keep.append(o)
    assert oracle.naive(t, p).tolist() == keep
    assert oracle.kmp(t, p).tolist() == keep


def test_expected_count_random_pattern():
    """E|H| = (n-m+1)/sigma^m for an i.i.d. uniform text (statistical)."""
    spec = gen.uniform_text(1 << 20, 4, seed=2)
    t = spec.host()
    pats = gen.random_patterns(np.arange(4, dtype=np.uint8), 6, 40, seed=4)
    total = sum(oracle.count_mt(t, p) for p in pats)
    mean = ((1 << 20) - 5) / 4 ** 6 * 40
    assert abs(total - mean) < 6 * mean ** 0.5


def test_m_zero_rejected():
    with pytest.raises(ValueError):
        oracle.naive(b"abc", b"")


MUTANTS = [
    # (description, original text, mutated text)
    ("drop last alignment", "return naive_range(t, 0, n - m + 1,", "return naive_range(t, 0, n - m,"),
    ("ignore last pattern byte", "while (j < m && t[i + j] == p[j]) ++j;",
     "while (j + 1 < m && t[i + j] == p[j]) ++j;"),
    ("skip first alignment", "for (uint64_t i = lo; i < hi; ++i) {", "for (uint64_t i = lo + 1; i < hi; ++i) {"),
    ("off-by-one compare", "t[i + j] == p[j]", "t[i + j + 1] == p[j]"),
    ("kmp forgets overlaps", "q = fail[q];\n        }", "q = 0;\n        }"),
    ("kmp wrong start", "emit(out, cap, &cnt, i + 1 - m);", "emit(out, cap, &cnt, i - m);"),
    ("kmp border off by one", "fail[q + 1] = k;", "fail[q + 1] = k ? k - 1 : 0;"),
    ("threaded chunk overlap", "jobs[c].hi = starts * (uint64_t)(c + 1) / (uint64_t)threads;",
     "jobs[c].hi = starts * (uint64_t)(c + 1) / (uint64_t)threads + (c + 1 < threads);"),
]


@pytest.mark.parametrize("desc,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mutation_is_caught(desc, old, new, tmp_path):
    """A plausible mistake planted in a copy of the oracle fails some pin."""
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    assert old in src, desc
    mut = tmp_path / "oracle_mut.c"
    mut.write_text(src.replace(old, new, 1))
    so = oracle.compile_oracle(str(mut), str(tmp_path / "libmut.so"))
    lib = oracle.load(so)
    failures = [
        pin_handworked(lib),
        pin_exhaustive_binary(lib, 7),
        pin_closed_forms(lib),
        pin_library_routines(lib, cases=60),
    ]
    assert any(f is not None for f in failures), f"mutation '{desc}' not caught"
