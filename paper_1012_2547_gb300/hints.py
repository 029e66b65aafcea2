"""Alphabet-size hints from a sample of a text.

The library takes an alphabet-size hint (sigma) at plan time: it picks the
tuning cell and decides whether a short pattern may share a packed
Shift-And state with others (its occurrences must be expected sparse).
The count of distinct symbols overstates how varied a skewed or
correlated text is, so the hint used here is an effective alphabet size
from collision probabilities of the sample's k-grams: with c_k = sum over
k-grams g of p(g)^2 (estimated without bias as sum n(n-1) / (N(N-1))), a
substring of the text of length k occurs about c_k times per position,
which is sigma^-k for a uniform text of sigma symbols.  The hint is
min(c_2^(-1/2), c_4^(-1/4)): 4-grams catch correlations between
neighbouring symbols that pairs miss.
"""
from __future__ import annotations

import numpy as np


def _collision(keys: np.ndarray) -> float:
    _, n = np.unique(keys, return_counts=True)
    n = n.astype(np.float64)
    total = float(n.sum())
    if total < 2:
        return 1.0
    return max(float(np.dot(n, n - 1.0)) / (total * (total - 1.0)), 1e-300)


def effective_sigma(sample: np.ndarray) -> int:
    """Effective alphabet size of a byte sample (at least 1)."""
    a = np.asarray(sample, dtype=np.uint8)
    if a.size < 4:
        return 1
    a32 = a.astype(np.uint32)
    c2 = _collision(a32[:-1] * 256 + a32[1:])
    c4 = _collision(a32[:-3] | (a32[1:-2] << 8) | (a32[2:-1] << 16) | (a32[3:] << 24))
    return max(1, int(round(min(c2 ** -0.5, c4 ** -0.25))))
