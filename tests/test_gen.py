"""Seeded input generators (no GPU): determinism and published vectors."""
import numpy as np

from paper_1012_2547_gb300 import gen


def test_splitmix64_published_vector():
    # splitmix64 seeded with 1234567 (Vigna's reference splitmix64.c).
    got = [gen.mix64_int(1234567 + (i + 1) * gen.GAMMA) for i in range(3)]
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423]
    arr = gen.draws(1234567, 0, 3).tolist()
    assert arr == got


def test_window_is_position_indexed():
    for spec in (gen.uniform_text(100_000, 4, 3), gen.protein_text(100_000, 4),
                 gen.english_text(100_000, 5)):
        full = spec.host()
        for s, c in ((0, 10), (777, 5000), (99_990, 50)):
            assert np.array_equal(spec.window(s, c), full[s : s + c])


def test_symbol_ranges_and_skew():
    t = gen.uniform_text(1 << 18, 8, 1).host()
    assert t.max() == 7 and t.min() == 0
    pr = gen.protein_text(1 << 18, 2).host()
    h = np.bincount(pr, minlength=20)
    assert pr.max() < 20 and h[0] > 10 * h[19]
    en = gen.english_text(1 << 18, 3).host()
    assert en.min() >= 0x21 and en.max() <= 0x7A
    ge = gen.genome_text(1 << 16, 4).host()
    assert ge.max() <= 3


def test_deterministic_and_seed_sensitive():
    a = gen.uniform_text(4096, 4, 1).host()
    b = gen.uniform_text(4096, 4, 1).host()
    c = gen.uniform_text(4096, 4, 2).host()
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    g1 = gen.genome_text(5000, 7).host()
    assert np.array_equal(g1, gen.genome_text(5000, 7).host())


def test_pattern_offsets_in_range():
    offs = gen.pattern_offsets(1000, 10, 500, 3)
    assert min(offs) >= 0 and max(offs) <= 990
    spec = gen.uniform_text(1 << 16, 4, 9)
    t = spec.host()
    assert gen.substring_patterns(t, 8, 20, 5) == gen.substring_patterns_spec(spec, 8, 20, 5)


def test_plant_prefix():
    t = gen.uniform_text(1 << 16, 4, 1).host().copy()
    gen.plant_prefix(t, 1 << 14, 4096, seed=3)
    pos, val = gen.planted_positions(1 << 14, 4096, seed=3)
    assert len(pos) == 4
    assert np.all(t[pos] == val) and np.all(val != 0)
    mask = np.ones(1 << 14, bool)
    mask[pos] = False
    assert np.all(t[: 1 << 14][mask] == 0)
