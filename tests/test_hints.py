"""Effective alphabet size (plan-time hint) from a sample of a text."""
import numpy as np

from paper_1012_2547_gb300 import gen
from paper_1012_2547_gb300.hints import effective_sigma


def test_uniform_texts_give_their_alphabet_size():
    for sigma in (2, 4, 16, 64):
        t = gen.uniform_text(1 << 20, sigma, 3).host()
        assert abs(effective_sigma(t) - sigma) <= max(1, sigma // 32)


def test_skewed_and_correlated_texts_give_less():
    assert effective_sigma(gen.protein_text(1 << 20, 5).window(0, 1 << 20)) < 20
    assert effective_sigma(gen.english_text(1 << 20, 6).window(0, 1 << 20)) < 90
    assert effective_sigma(gen.genome_text(1 << 20, 7).host()) < 4


def test_periodic_and_constant_texts():
    assert effective_sigma(np.zeros(10_000, np.uint8)) == 1
    t = np.tile(np.arange(8, dtype=np.uint8), 5000)        # every 2- and 4-gram determined by its start
    assert effective_sigma(t) <= 3
