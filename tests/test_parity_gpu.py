"""GPU parity: sorted positions bit-exact with the CPU oracle.

All searches go through the C ABI (libsmgpu.so).  Each kernel family is
forced in turn on the same inputs, so every family is checked on its own.
"""
import numpy as np
import pytest

import oracle
from paper_1012_2547_gb300 import gen

from _helpers import expect, gpu_search, to_dev, torch, variants_for

pytestmark = pytest.mark.gpu


def test_single_search_1mib_sigma4_m8():
    """Single search: n = 1,048,576, uniform sigma = 4, m = 8 substring."""
    spec = gen.uniform_text(1 << 20, 4, seed=1)
    t = spec.host()
    p = gen.substring_patterns(t, 8, 1, seed=2)[0]
    exp = oracle.naive(t, p)
    dev = to_dev(t)
    for variant, q, wb in variants_for(8, p):
        got, total, _ = gpu_search(dev, p, variant, q, wb)
        assert total == len(exp), (variant, q, wb)
        assert np.array_equal(got, exp), (variant, q, wb)


@pytest.mark.parametrize("m", [1, 2, 3, 5, 8, 15, 16, 17, 18, 24, 31, 32, 33, 40, 48, 49, 50, 57,
                               63, 64, 65, 100, 255, 256, 700, 1024])
def test_random_texts_all_variants(m):
    rng = np.random.default_rng(1000 + m)
    for sigma, n in ((2, 200_003), (4, 123_457), (20, 77_777), (256, 65_536 + 13)):
        t = rng.integers(0, sigma, n, dtype=np.uint8)
        pats = gen.substring_patterns(t, m, 2, seed=m * 7 + sigma)
        pats.append(bytes(rng.integers(0, sigma, m, dtype=np.uint8)))
        for off in (0, 5):
            dev = to_dev(t, off)
            for p in pats:
                exp = expect(t, p)
                for variant, q, wb in variants_for(m, p):
                    got, total, _ = gpu_search(dev, p, variant, q, wb)
                    assert total == len(exp), (sigma, n, off, variant, q, wb)
                    assert np.array_equal(got, exp), (sigma, n, off, variant, q, wb)


@pytest.mark.parametrize("m", [1, 2, 4, 17, 32, 64, 65, 300, 1024])
def test_dense_a_power(m):
    """a^m in a^n: exactly the n-m+1 positions 0..n-m (closed form)."""
    for n in (m, m + 1, 70_001, 250_000):
        t = np.zeros(n, dtype=np.uint8)
        dev = to_dev(t, 3)
        p = bytes(m)
        for variant, q, wb in variants_for(m, p):
            got, total, _ = gpu_search(dev, p, variant, q, wb)
            assert total == n - m + 1, (n, variant, q, wb)
            assert np.array_equal(got, np.arange(n - m + 1, dtype=np.uint64)), (n, variant)


def test_periodic_patterns_on_periodic_text():
    """(ab)^k and (aab)^k style inputs: many overlapping occurrences."""
    for unit, reps, mreps in ((b"ab", 60_000, (1, 8, 40, 300)), (b"aab", 40_000, (2, 11, 22, 111))):
        t = np.frombuffer(unit * reps, dtype=np.uint8)
        dev = to_dev(t, 1)
        for r in mreps:
            p = unit * r
            exp = oracle.kmp(t, p)
            for variant, q, wb in variants_for(len(p), p):
                got, total, _ = gpu_search(dev, p, variant, q, wb)
                assert total == len(exp) and np.array_equal(got, exp), (unit, r, variant, q)


def test_edges_m_gt_n_empty_text_and_ends():
    t = np.frombuffer(b"abcdefghij" * 3, dtype=np.uint8)
    dev = to_dev(t)
    got, total, _ = gpu_search(dev, b"x" * 31)
    assert total == 0
    got, total, _ = gpu_search(dev[:0], b"ab")
    assert total == 0
    for p in (b"ab", b"ij", b"abcdefghij" * 3, b"j", b"a"):
        exp = oracle.naive(t, p)
        for variant, q, wb in variants_for(len(p), p):
            got, total, _ = gpu_search(dev, p, variant, q, wb)
            assert np.array_equal(got, exp), (p, variant, q, wb)


def test_every_offset_and_tile_boundary():
    """Planted occurrences at every position of a window around tile
    boundaries and at both ends; text pointer at all 16 alignments."""
    rng = np.random.default_rng(7)
    n = 4 * 30720 + 777
    base = rng.integers(0, 200, n, dtype=np.uint8)
    for m in (3, 16, 40, 64, 90):
        p = bytes(rng.integers(200, 256, m, dtype=np.uint8))
        t = base.copy()
        plant = [0, n - m] + [b + d for b in (30720, 61440, 92160) for d in (-m, -1, 0, 1, 7)]
        plant = sorted(set(x for x in plant if 0 <= x <= n - m))
        keep = []
        for x in plant:
            if not keep or x >= keep[-1] + m:
                t[x: x + m] = np.frombuffer(p, dtype=np.uint8)
                keep.append(x)
        exp = np.array(keep, dtype=np.uint64)
        assert np.array_equal(oracle.naive(t, p), exp)
        for off in range(16):
            dev = to_dev(t, off)
            for variant, q, wb in variants_for(m, p):
                got, total, _ = gpu_search(dev, p, variant, q, wb)
                assert np.array_equal(got, exp), (m, off, variant, q, wb)


def test_truncation_reports_true_count():
    t = np.zeros(100_000, dtype=np.uint8)
    dev = to_dev(t)
    for variant, q, wb in variants_for(4, bytes(4)):
        got, total, _ = gpu_search(dev, bytes(4), variant, q, wb, cap=1000)
        assert total == 100_000 - 3
        assert np.array_equal(got, np.arange(1000, dtype=np.uint64))


def test_exhaustive_binary_pairs_n_le_12():
    """Every binary text of length n <= 12 against every binary pattern of
    length m <= n, each kernel family forced in turn.  Texts of one length
    are concatenated with a separator byte (2) that no pattern contains."""
    import paper_1012_2547_gb300 as smg
    tt = torch()
    for n in range(1, 13):
        texts = ((np.arange(1 << n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)
        cat = np.concatenate([texts, np.full((1 << n, 1), 2, np.uint8)], axis=1).ravel()
        dev = to_dev(cat)
        for m in range(1, n + 1):
            exp = oracle.binary_masks(n, m)  # [text, pattern] -> hit bitmask
            pats = [bytes(((pv >> np.arange(m)) & 1).astype(np.uint8)) for pv in range(1 << m)]
            for variant, q, wb in variants_for(m, pats[-1]):
                plans = smg.prepare_many(pats, variant=variant, q=q, word_bits=wb)
                cap = (1 << n) * (n - m + 1)
                outs = tt.full((len(pats), cap), -1, dtype=tt.int64, device="cuda")
                cnts = tt.zeros(len(pats), dtype=tt.int64, device="cuda")
                items = [(dev, plans[i], outs[i], cnts[i: i + 1]) for i in range(len(pats))]
                smg.search_batch(items)
                smg.sync()
                outs_h = outs.cpu().numpy()
                cnts_h = cnts.cpu().numpy()
                for pv in range(1 << m):
                    pos = outs_h[pv, : cnts_h[pv]]
                    tv, off = np.divmod(pos, n + 1)
                    got = np.zeros(1 << n, dtype=np.uint32)
                    np.bitwise_or.at(got, tv, (1 << off).astype(np.uint32))
                    assert np.array_equal(got, exp[:, pv]), (n, m, pv, variant, q, wb)


def test_device_generator_matches_host():
    import paper_1012_2547_gb300 as smg
    tt = torch()
    for spec in (gen.uniform_text(1 << 20, 4, 3), gen.uniform_text(300_001, 128, 4),
                 gen.protein_text(200_000, 5), gen.english_text(200_000, 6)):
        out = tt.empty(spec.n - 1000, dtype=tt.uint8, device="cuda")
        thr = bmap = None
        sigma = spec.sigma
        if spec.kind == "skewed":
            thr = tt.tensor(np.asarray(spec.thresholds, dtype=np.uint32).view(np.int32), device="cuda")
            bmap = tt.tensor(np.asarray(spec.byte_map, dtype=np.uint8), device="cuda")
            sigma = 0
        smg.gen_text(out, 1000, spec.key, sigma, thr, bmap)
        smg.sync()
        assert np.array_equal(out.cpu().numpy(), spec.window(1000, spec.n - 1000))


@pytest.mark.parametrize("m", [1, 2, 3, 4, 6, 9, 20])
def test_long_work_items_hit_storage(m):
    """Bit-parallel work items of many sub-tiles (config tile): hits kept in
    shared memory, in the spill position list, and as spilled flag words
    (densities 1/4 .. 1/4^9 on sigma = 4), bit-exact with the oracle."""
    spec = gen.uniform_text((8 << 20) + 12_345, 4, seed=40 + m)
    t = spec.host()
    pats = gen.substring_patterns(t, m, 2, seed=m)
    for off in (0, 7):
        dev = to_dev(t, off)
        for p in pats:
            exp = oracle.naive_mt(t, p)
            for wb in ((32, 64) if m <= 32 else (64,)):
                for tile in (17, 22):
                    got, total, _ = gpu_search(dev, p, "shiftor", 0, wb, tile=tile)
                    assert total == len(exp), (off, wb, tile)
                    assert np.array_equal(got, exp), (off, wb, tile)
