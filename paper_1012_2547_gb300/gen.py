"""Seeded synthetic inputs for exact string matching.

This module only makes inputs: texts and patterns with the shapes and symbol
distributions of the workloads the paper times (Section 2: random texts of
alphabet size sigma with a uniform distribution, a genome, a protein sequence
and natural-language text; patterns of length m extracted from the text at
random offsets).  It holds no part of the matching method, so both the CUDA
path (through its tests and the benchmark) and the CPU oracle can be fed from
it without sharing any matching arithmetic.

Random numbers come from one counter-based generator: the splitmix64 output
function (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014, as published in Vigna's splitmix64.c) applied to
``key + (i + 1) * GAMMA``.  Byte ``i`` of a counter-based text depends only on
``(seed, i)``, so a device kernel written from the same definition produces the
same bytes (``sm_gen_text`` in ``include/smgen.h``), and the host can rebuild
any window of a device-resident text without reading it back.

Symbol mapping from a 64-bit draw ``r``:
  * uniform over sigma symbols: ``((r >> 32) * sigma) >> 32``;
  * a skewed distribution: ``u = r >> 32`` and the symbol index is the number
    of 32-bit cumulative thresholds ``<= u`` (thresholds are
    ``floor(cdf_k * 2**32)`` of the distribution, computed once in float64);
then the symbol index goes through a 256-entry byte map (identity, or
``0x21 + rank`` for the English-like text).
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_STREAM = 0xD1B54A32D192ED03
MASK64 = (1 << 64) - 1

# Named streams: one per kind of draw, so that e.g. pattern offsets never
# reuse the text's numbers.
STREAM_TEXT = 1
STREAM_OFFSETS = 2
STREAM_RANDPAT = 3
STREAM_MARKOV_ROWS = 4
STREAM_PLANT = 5
STREAM_LENGTHS = 6
STREAM_SIZES = 7


def mix64_int(z: int) -> int:
    """splitmix64 output function on a Python int (exact, mod 2**64)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * _M1) & MASK64
    z = ((z ^ (z >> 27)) * _M2) & MASK64
    return z ^ (z >> 31)


def _mix64_np(z: np.ndarray) -> np.ndarray:
    z = z ^ (z >> np.uint64(30))
    z = z * np.uint64(_M1)
    z = z ^ (z >> np.uint64(27))
    z = z * np.uint64(_M2)
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> int:
    """64-bit key of the draw sequence ``stream`` under ``seed``."""
    return mix64_int((seed * GAMMA + stream * _STREAM + 1) & MASK64)


def draws(key: int, start: int, count: int) -> np.ndarray:
    """Draws ``start .. start+count-1`` of the sequence with ``key`` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(key) + i * np.uint64(GAMMA)
        return _mix64_np(z)


def draw_int(key: int, i: int) -> int:
    return mix64_int(key + (i + 1) * GAMMA)


def thresholds_from_probs(p) -> np.ndarray:
    """32-bit cumulative thresholds (K-1 of them) for probabilities p."""
    p = np.asarray(p, dtype=np.float64)
    p = p / p.sum()
    cdf = np.cumsum(p)[:-1]
    return np.floor(cdf * 4294967296.0).astype(np.uint64)


def protein_probs() -> np.ndarray:
    """Protein-like skew: p_k proportional to 0.85**k over 20 symbols."""
    return 0.85 ** np.arange(20, dtype=np.float64)


def zipf_probs(count: int = 90, s: float = 1.1) -> np.ndarray:
    """Zipf(s) over ``count`` ranks: p_r proportional to 1/(r+1)**s."""
    return 1.0 / np.arange(1, count + 1, dtype=np.float64) ** s


_BLOCK = 1 << 20


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


@dataclass(frozen=True)
class TextSpec:
    """A seeded synthetic text.

    kind: "uniform" (sigma symbols 0..sigma-1), "skewed" (thresholds +
    byte map), "markov3" (order-3 Markov chain over {0,1,2,3}, host only).
    """

    kind: str
    n: int
    seed: int
    sigma: int = 4
    name: str = ""
    thresholds: tuple = field(default=())
    byte_map: tuple = field(default=())

    @property
    def key(self) -> int:
        return stream_key(self.seed, STREAM_TEXT)

    @property
    def counter_based(self) -> bool:
        return self.kind in ("uniform", "skewed")

    def alphabet(self) -> np.ndarray:
        if self.kind == "uniform":
            return np.arange(self.sigma, dtype=np.uint8)
        if self.kind == "markov3":
            return np.arange(4, dtype=np.uint8)
        return np.asarray(self.byte_map[: len(self.thresholds) + 1], dtype=np.uint8)

    def window(self, start: int, count: int) -> np.ndarray:
        """Bytes [start, start+count) of a counter-based text.  Long windows
        are built in 1 MiB blocks on a pool of host threads (numpy's array
        loops run without the interpreter lock)."""
        if not self.counter_based:
            raise ValueError("window() needs a counter-based text kind")
        count = max(0, min(count, self.n - start))
        if count > _BLOCK:
            out = np.empty(count, dtype=np.uint8)

            def fill(off):
                out[off:off + _BLOCK] = self._block(start + off, min(_BLOCK, count - off))
            with ThreadPoolExecutor(_threads()) as ex:
                list(ex.map(fill, range(0, count, _BLOCK)))
            return out
        return self._block(start, count)

    def _block(self, start: int, count: int) -> np.ndarray:
        r = draws(self.key, start, count)
        u = (r >> np.uint64(32))
        if self.kind == "uniform":
            return ((u * np.uint64(self.sigma)) >> np.uint64(32)).astype(np.uint8)
        thr = np.asarray(self.thresholds, dtype=np.uint64)
        idx = np.searchsorted(thr, u, side="right")
        return np.asarray(self.byte_map, dtype=np.uint8)[idx]

    def host(self) -> np.ndarray:
        """The whole text as a host uint8 array."""
        if self.counter_based:
            return self.window(0, self.n)
        if self.kind == "markov3":
            return markov3_text(self.n, self.seed)
        raise ValueError(self.kind)


def uniform_text(n: int, sigma: int, seed: int) -> TextSpec:
    return TextSpec("uniform", n, seed, sigma=sigma, name=f"rand{sigma}")


def protein_text(n: int, seed: int) -> TextSpec:
    thr = tuple(int(x) for x in thresholds_from_probs(protein_probs()))
    return TextSpec("skewed", n, seed, sigma=20, name="protein20",
                    thresholds=thr, byte_map=tuple(range(256)))


def english_text(n: int, seed: int) -> TextSpec:
    thr = tuple(int(x) for x in thresholds_from_probs(zipf_probs(90, 1.1)))
    bm = tuple((0x21 + r) if r < 90 else 0 for r in range(256))
    return TextSpec("skewed", n, seed, sigma=90, name="english90",
                    thresholds=thr, byte_map=bm)


def genome_text(n: int, seed: int) -> TextSpec:
    return TextSpec("markov3", n, seed, sigma=4, name="genome4")


def markov3_rows(seed: int) -> np.ndarray:
    """64 context rows of 3 thresholds: Dirichlet(1) rows from the seed.

    A Dirichlet(1,1,1,1) row is four Exp(1) variates normalised to sum 1;
    each Exp(1) variate is -log of a uniform in (0, 1).
    """
    key = stream_key(seed, STREAM_MARKOV_ROWS)
    r = draws(key, 0, 64 * 4)
    u = ((r >> np.uint64(11)).astype(np.float64) + 0.5) / 9007199254740992.0
    e = -np.log(u).reshape(64, 4)
    rows = np.stack([thresholds_from_probs(row) for row in e])
    return rows.astype(np.uint64)


def markov3_text(n: int, seed: int) -> np.ndarray:
    """Order-3 Markov chain over {0,1,2,3} (genome-like), host only."""
    rows = markov3_rows(seed).tolist()
    key = stream_key(seed, STREAM_TEXT)
    out = bytearray(n)
    ctx = 0
    step = 1 << 20
    for s in range(0, n, step):
        u = (draws(key, s, min(step, n - s)) >> np.uint64(32)).tolist()
        for k, uk in enumerate(u):
            t0, t1, t2 = rows[ctx]
            sym = (uk >= t0) + (uk >= t1) + (uk >= t2)
            out[s + k] = sym
            ctx = ((ctx << 2) | sym) & 63
    return np.frombuffer(out, dtype=np.uint8)  # a writable view of the bytearray


def sweep_texts(n: int = 4_194_304, seed: int = 11) -> list[TextSpec]:
    """The ten texts of the paper-shaped sweep (Section 2 text buffers)."""
    out = [uniform_text(n, s, seed + i) for i, s in enumerate((2, 4, 8, 16, 32, 64, 128))]
    out.append(genome_text(n, seed + 7))
    out.append(protein_text(n, seed + 8))
    out.append(english_text(n, seed + 9))
    return out


SWEEP_M = (2, 4, 8, 16, 32, 64, 128, 256, 512, 1024)


def pattern_offsets(n: int, m: int, count: int, seed: int) -> list[int]:
    """Uniform offsets in [0, n-m] (exact 64-bit multiply-high)."""
    if m > n:
        return []
    key = stream_key(seed, STREAM_OFFSETS)
    span = n - m + 1
    return [(draw_int(key, k) * span) >> 64 for k in range(count)]


def substring_patterns(text: np.ndarray, m: int, count: int, seed: int) -> list[bytes]:
    offs = pattern_offsets(len(text), m, count, seed)
    return [bytes(text[o : o + m]) for o in offs]


def substring_patterns_spec(spec: TextSpec, m: int, count: int, seed: int) -> list[bytes]:
    """Substrings of a counter-based text, rebuilt from the generator."""
    offs = pattern_offsets(spec.n, m, count, seed)
    return [bytes(spec.window(o, m)) for o in offs]


def random_patterns(alphabet, m: int, count: int, seed: int, thresholds=None) -> list[bytes]:
    """i.i.d. patterns over ``alphabet`` (uniform, or by ``thresholds``)."""
    alphabet = np.asarray(alphabet, dtype=np.uint8)
    key = stream_key(seed, STREAM_RANDPAT)
    r = draws(key, 0, m * count) >> np.uint64(32)
    if thresholds is None:
        idx = (r * np.uint64(len(alphabet))) >> np.uint64(32)
    else:
        idx = np.searchsorted(np.asarray(thresholds, dtype=np.uint64), r, side="right")
    sym = alphabet[idx.astype(np.int64)]
    return [bytes(sym[k * m : (k + 1) * m]) for k in range(count)]


def plant_prefix(text: np.ndarray, prefix: int, block: int, seed: int, a: int = 0,
                 sigma: int = 4) -> np.ndarray:
    """Overwrite text[0:prefix) with symbol ``a`` except one random non-``a``
    byte per ``block`` bytes (the a^n-dominated region of the dense stress)."""
    text[:prefix] = a
    key = stream_key(seed, STREAM_PLANT)
    nb = prefix // block
    r = draws(key, 0, nb)
    pos = (np.arange(nb, dtype=np.uint64) * np.uint64(block)
           + (r & np.uint64(block - 1)))
    val = (((r >> np.uint64(32)) * np.uint64(sigma - 1)) >> np.uint64(32)) + np.uint64(1)
    text[pos.astype(np.int64)] = ((val.astype(np.int64) + a) % sigma).astype(np.uint8)
    return text


def planted_positions(prefix: int, block: int, seed: int, a: int = 0, sigma: int = 4):
    """Positions and byte values ``plant_prefix`` writes."""
    key = stream_key(seed, STREAM_PLANT)
    nb = prefix // block
    r = draws(key, 0, nb)
    pos = (np.arange(nb, dtype=np.uint64) * np.uint64(block)
           + (r & np.uint64(block - 1)))
    val = (((r >> np.uint64(32)) * np.uint64(sigma - 1)) >> np.uint64(32)) + np.uint64(1)
    return pos.astype(np.int64), ((val.astype(np.int64) + a) % sigma).astype(np.uint8)


def log_uniform_int(key: int, k: int, lo: int, hi: int) -> int:
    """floor(lo * (hi/lo)**u) with u from draw k (float64, deterministic)."""
    u = (draw_int(key, k) >> 11) / 9007199254740992.0
    return int(math.floor(lo * (hi / lo) ** u))
