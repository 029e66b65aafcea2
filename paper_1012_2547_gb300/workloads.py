"""Synthetic workloads shaped like the paper's experiments (Section 2).

Input construction only (texts, patterns, sizes); no matching arithmetic.
  single    : n = 1,048,576 uniform sigma = 4 text, one m = 8 substring.
  sweep     : ten 4 MiB texts (uniform sigma in {2,..,128}, order-3 Markov
              genome-like, skewed protein-like sigma = 20, Zipf English-like
              over 90 printable bytes); m in {2, 4, ..., 1024}; 100 substring
              patterns per (text, m) at seeded offsets (Section 2 extracts
              its patterns from the text at random).
  bandwidth : one 8 GiB uniform sigma = 4 text built on the device,
              m in {4, 32, 256, 1024}, 20 substring + 20 random patterns per
              m, and a^m on an a^n-dominated 64 MiB prefix.
  batched   : (i) 4096 patterns, m log-uniform in [2, 1024], half
              substrings and half i.i.d. uniform over the 20 symbols, on one
              shared 1 GiB protein-like (sigma = 20, skewed) text; (ii) 10,000
              (pattern, text) pairs, text lengths log-uniform in [4 KiB,
              64 MiB], sigma alternating 4 / 64, m log-uniform in [2, 1024],
              substring patterns.  Device-built texts.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import gen
from .hints import effective_sigma

SWEEP_N = 4_194_304
SWEEP_PER_M = 100


@dataclass
class Query:
    text_id: int
    pattern: bytes
    sigma_hint: int
    n: int | None = None  # None = the whole text
    offset: int = 0       # first byte of the query's text within texts[text_id]


@dataclass
class Workload:
    name: str
    texts: list          # host uint8 arrays (or TextSpec for device-built texts)
    specs: list
    queries: list = field(default_factory=list)

    @property
    def scanned_bytes(self) -> int:
        tot = 0
        for q in self.queries:
            tot += q.n if q.n is not None else self.specs[q.text_id].n
        return tot


def sigma_hint(spec: gen.TextSpec, sample=None) -> int:
    """Alphabet-size hint of a text: sigma for a uniform text, else the
    effective alphabet size of a sample of it (hints.effective_sigma)."""
    if spec.kind == "uniform":
        return spec.sigma
    if sample is None:
        sample = spec.host()[: 1 << 20] if spec.kind == "markov3" else spec.window(0, 1 << 20)
    return effective_sigma(sample[: 1 << 20])


def single() -> Workload:
    spec = gen.uniform_text(1 << 20, 4, seed=1)
    t = spec.host()
    p = gen.substring_patterns(t, 8, 1, seed=2)[0]
    return Workload("single_n1048576_sigma4_m8", [t], [spec], [Query(0, p, 4)])


def sweep(n: int = SWEEP_N, per_m: int = SWEEP_PER_M, ms=gen.SWEEP_M, seed: int = 11) -> Workload:
    specs = gen.sweep_texts(n, seed)
    texts = [s.host() for s in specs]
    w = Workload(f"sweep_10texts_n{n}_m2-1024_x{per_m}", texts, specs)
    for ti, (spec, t) in enumerate(zip(specs, texts)):
        hint = sigma_hint(spec, t)
        for m in ms:
            for p in gen.substring_patterns(t, m, per_m, seed=seed * 1000 + ti * 16 + m.bit_length()):
                w.queries.append(Query(ti, p, hint))
    return w


BANDWIDTH_N = 8 << 30
BANDWIDTH_M = (4, 32, 256, 1024)
DENSE_PREFIX = 64 << 20


def bandwidth(n: int = BANDWIDTH_N, per_m: int = 20, ms=BANDWIDTH_M, seed: int = 21) -> Workload:
    """Device-built text: texts[0] is the TextSpec (see gen.TextSpec.window
    for host windows).  The dense stress queries search a^m in the first
    64 MiB, which the caller overwrites with gen.plant_prefix."""
    spec = gen.uniform_text(n, 4, seed)
    w = Workload(f"bandwidth_n{n}_sigma4", [spec], [spec])
    alphabet = np.arange(4, dtype=np.uint8)
    for m in ms:
        for p in gen.substring_patterns_spec(spec, m, per_m, seed=seed * 100 + m):
            w.queries.append(Query(0, p, 4))
        for p in gen.random_patterns(alphabet, m, per_m, seed=seed * 100 + m + 1):
            w.queries.append(Query(0, p, 4))
    return w


def bandwidth_dense(ms=BANDWIDTH_M, prefix: int = DENSE_PREFIX) -> list[Query]:
    return [Query(0, bytes(m), 4, n=prefix) for m in ms]


BATCHED_SHARED_N = 1 << 30
BATCHED_SHARED_Q = 4096
BATCHED_PAIRS = 10_000


def batched_shared(n: int = BATCHED_SHARED_N, nq: int = BATCHED_SHARED_Q, seed: int = 31) -> Workload:
    """One shared protein-like text (device-built; texts[0] is its TextSpec)
    and nq patterns of length floor(2 * 512**u), u uniform: even queries are
    substrings at seeded offsets, odd ones i.i.d. uniform over the 20
    symbols."""
    spec = gen.protein_text(n, seed)
    w = Workload(f"batched_shared_n{n}_sigma20_q{nq}", [spec], [spec])
    klen = gen.stream_key(seed, gen.STREAM_LENGTHS)
    alphabet = np.arange(20, dtype=np.uint8)
    hint = sigma_hint(spec)
    for i in range(nq):
        m = gen.log_uniform_int(klen, i, 2, 1024)
        if i % 2 == 0:
            o = gen.pattern_offsets(n, m, 1, seed=seed * 1_000_003 + i)[0]
            p = bytes(spec.window(o, m))
        else:
            p = gen.random_patterns(alphabet, m, 1, seed=seed * 1_000_003 + i)[0]
        w.queries.append(Query(0, p, hint))
    return w


def batched_pairs(count: int = BATCHED_PAIRS, seed: int = 41, lo: int = 4096,
                  hi: int = 64 << 20) -> Workload:
    """count (pattern, text) pairs.  Pair i has its own text of
    floor(lo * (hi/lo)**u) bytes over sigma 4 (even i) or 64 (odd i): a
    disjoint slice of one long device-built text per sigma (texts[0] for
    sigma 4, texts[1] for 64), and a substring pattern of length
    floor(2 * 512**u') at a seeded offset inside it."""
    ksz = gen.stream_key(seed, gen.STREAM_SIZES)
    klen = gen.stream_key(seed, gen.STREAM_LENGTHS)
    sizes = [gen.log_uniform_int(ksz, i, lo, hi) for i in range(count)]
    total = [0, 0]
    offs = []
    for i, n in enumerate(sizes):
        offs.append(total[i % 2])
        total[i % 2] += n
    specs = [gen.uniform_text(total[0], 4, seed + 4), gen.uniform_text(total[1], 64, seed + 64)]
    w = Workload(f"batched_pairs_{count}_n{lo}-{hi}_sigma4-64", specs, specs)
    for i, n in enumerate(sizes):
        spec = specs[i % 2]
        m = min(gen.log_uniform_int(klen, i, 2, 1024), n)
        o = gen.pattern_offsets(n, m, 1, seed=seed * 1_000_003 + i)[0]
        w.queries.append(Query(i % 2, bytes(spec.window(offs[i] + o, m)), spec.sigma, n=n, offset=offs[i]))
    return w
