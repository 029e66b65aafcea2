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
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import gen

SWEEP_N = 4_194_304
SWEEP_PER_M = 100


@dataclass
class Query:
    text_id: int
    pattern: bytes
    sigma_hint: int
    n: int | None = None  # None = the whole text


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


def sigma_hint(spec: gen.TextSpec) -> int:
    return 4 if spec.kind == "markov3" else spec.sigma


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
        for m in ms:
            for p in gen.substring_patterns(t, m, per_m, seed=seed * 1000 + ti * 16 + m.bit_length()):
                w.queries.append(Query(ti, p, sigma_hint(spec)))
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
