"""GPU parity of the string-matching automaton (DFA kernel family, and the
q-gram kernel's dense fallback through the automaton), bit-exact with the
CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_1012_2547_gb300 import gen

from _helpers import DFA_MAX_TABLE, dfa_fits, gpu_search, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m", [1000, 4000, 8127])
def test_dfa_long_a_power(m):
    """a^m in a^n: the n-m+1 positions 0..n-m, for m up to the table bound
    ((m+1) x 2 classes x 2 bytes <= 32,512)."""
    assert dfa_fits(bytes(m))
    for n in (m, m + 1, 300_001):
        dev = to_dev(np.zeros(n, dtype=np.uint8), 5)
        got, total, plan = gpu_search(dev, bytes(m), "dfa")
        assert plan.info().variant == "dfa"
        assert total == n - m + 1
        assert np.array_equal(got, np.arange(n - m + 1, dtype=np.uint64))


def test_dfa_periodic_with_defects():
    """(abc)^k patterns on a periodic text with a few corrupted bytes: runs
    of overlapping occurrences broken at the defects."""
    rng = np.random.default_rng(11)
    t = np.frombuffer(b"abc" * 200_000, dtype=np.uint8).copy()
    t[rng.integers(0, len(t), 40)] = ord("x")
    for r in (1, 7, 300, 1300):
        p = b"abc" * r + b"ab"
        assert dfa_fits(p)
        exp = oracle.kmp(t, p)
        for off in (0, 9):
            dev = to_dev(t, off)
            for variant, q in (("dfa", 0), ("qgram", min(8, len(p))), ("qgram", 3)):
                got, total, _ = gpu_search(dev, p, variant, q)
                assert total == len(exp) and np.array_equal(got, exp), (r, off, variant, q)


@pytest.mark.parametrize("sigma,m", [(2, 64), (4, 1024), (4, 3000), (20, 700), (256, 60)])
def test_dfa_random_texts(sigma, m):
    """Sparse hits on random texts, text pointers at all alignments 0..15
    (the 16-byte loads start at the first aligned address)."""
    rng = np.random.default_rng(sigma * 10_000 + m)
    n = 500_000 + 77
    t = rng.integers(0, sigma, n, dtype=np.uint8)
    pats = gen.substring_patterns(t, m, 2, seed=m)
    pats = [p for p in pats if dfa_fits(p)]
    assert pats
    exps = [oracle.kmp(t, p) for p in pats]
    for off in range(16):
        dev = to_dev(t, off)
        for p, exp in zip(pats, exps):
            got, total, _ = gpu_search(dev, p, "dfa")
            assert total == len(exp) and np.array_equal(got, exp), (off, len(p))


def test_dfa_ranges_and_truncation():
    """Thread ranges of several sizes (config tile), hits at range and tile
    boundaries, and truncation with the true count."""
    rng = np.random.default_rng(3)
    n = 1 << 20
    t = rng.integers(0, 4, n, dtype=np.uint8)
    p = bytes([0, 1, 2, 3, 0, 1, 2])
    for x in list(range(0, n - 7, 4093)):
        t[x: x + 7] = np.frombuffer(p, dtype=np.uint8)
    exp = oracle.naive(t, p)
    dev = to_dev(t, 3)
    for tile in (0, 10, 12, 16):
        got, total, _ = gpu_search(dev, p, "dfa", tile=tile)
        assert total == len(exp) and np.array_equal(got, exp), tile
    got, total, _ = gpu_search(dev, p, "dfa", cap=100)
    assert total == len(exp) and np.array_equal(got, exp[:100])


def test_dfa_table_bound():
    """A pattern whose automaton exceeds the bound: an explicit DFA config is
    rejected (SM_EINVAL); the automatic choice still serves it."""
    import paper_1012_2547_gb300 as smg
    p = bytes(range(256)) * 4  # m = 1024, C = 257
    assert not dfa_fits(p)
    with pytest.raises(smg.SmError):
        smg.prepare(p, variant="dfa")
    t = np.frombuffer(p * 50, dtype=np.uint8)
    got, total, plan = gpu_search(to_dev(t), p)
    assert plan.info().variant != "dfa"
    assert np.array_equal(got, oracle.kmp(t, p))
    assert (len(p) + 1) * 257 * 2 > DFA_MAX_TABLE


def test_qgram_dense_fallback_periodic_and_aperiodic():
    """The q-gram density guard on a^n-like text: a periodic pattern (a^m,
    whose plan carries the automaton) and an aperiodic one (a^(m-1) b, whose
    dense tiles run Knuth-Morris-Pratt), both exact."""
    n = 400_000
    t = np.zeros(n, dtype=np.uint8)
    rng = np.random.default_rng(8)
    for m in (100, 1000):
        tt = t.copy()
        for x in rng.integers(0, n - m, 30):
            tt[x + m - 1] = 1  # a^(m-1) b ends here
        dev = to_dev(tt, 1)
        per, aper = bytes(m), bytes(m - 1) + b"\x01"
        for p in (per, aper):
            exp = oracle.kmp(tt, p)
            for q in (3, 8):
                got, total, _ = gpu_search(dev, p, "qgram", q)
                assert total == len(exp) and np.array_equal(got, exp), (m, p == per, q)
        import paper_1012_2547_gb300 as smg
        # The periodic pattern's plan is larger by its automaton's tables.
        b_per = smg.prepare(per, variant="qgram", q=8).info().device_bytes
        b_aper = smg.prepare(aper, variant="qgram", q=8).info().device_bytes
        assert b_per > b_aper


def test_mixed_batch_with_dfa():
    """One batch mixing automaton, q-gram and bit-parallel plans over several
    texts (one launch per kernel family), every result exact."""
    import paper_1012_2547_gb300 as smg
    tt = torch()
    rng = np.random.default_rng(21)
    texts = [rng.integers(0, s, n, dtype=np.uint8) for s, n in ((4, 300_000), (2, 123_457), (20, 65_536))]
    texts.append(np.zeros(100_000, dtype=np.uint8))
    devs = [to_dev(t, i) for i, t in enumerate(texts)]
    jobs = []
    for ti, t in enumerate(texts):
        for m in (5, 40, 300):
            p = bytes(m) if ti == 3 else gen.substring_patterns(t, m, 1, seed=ti * 100 + m)[0]
            for variant in ("dfa", "auto"):
                jobs.append((ti, p, variant))
    plans = [smg.prepare(p, variant=v) for _, p, v in jobs]
    exps = [oracle.kmp(texts[ti], p) for ti, p, _ in jobs]
    outs = [tt.full((max(len(e), 1),), -1, dtype=tt.int64, device="cuda") for e in exps]
    cnts = tt.zeros(len(jobs), dtype=tt.int64, device="cuda")
    items = [(devs[ti], plans[i], outs[i], cnts[i: i + 1]) for i, (ti, _, _) in enumerate(jobs)]
    smg.search_batch(items)
    smg.sync()
    c = cnts.cpu().numpy()
    for i, e in enumerate(exps):
        assert c[i] == len(e), jobs[i][1:]
        assert np.array_equal(outs[i][: len(e)].cpu().numpy().astype(np.uint64), e), jobs[i][1:]
