"""Autotuner: (m bucket, sigma bucket) -> kernel configuration, measured on
the device.

Section 3 of the paper finds that no single algorithm is best for every
pattern length and alphabet size.  The library therefore keeps a table of
configurations indexed by the bucket of m (floor(log2 m), 0..11) and of
sigma (0 = unknown, else floor(log2 sigma) clamped to 1..8), used by
sm_prepare when no explicit configuration is given (include/smgpu.h,
sm_tuning_*).  This module fills that table by timing candidate
configurations on a batch of substring patterns of a uniform text of each
alphabet size, as one graph-captured batch per candidate, and keeping the
fastest: first every kernel family and its parameter (Shift-Or with a 32-
or 64-bit state, q-gram filter for q in {3, ..., 8}, the automaton where
its table fits), then the work-item size (the `tile` field) of the
fastest.  The table can be saved to and loaded from JSON.
"""
from __future__ import annotations

import json
import math
import os
import statistics
import time

import numpy as np

from . import Batch, _lib, gen, prepare_many, search_batch, sync, tuning_get, tuning_set

M_BUCKETS = _lib.TUNE_M_BUCKETS
S_BUCKETS = _lib.TUNE_S_BUCKETS
VARIANT_IDS = {"shiftor": 1, "qgram": 2, "linear": 3, "dfa": 4}
DFA_MAX_TABLE = 32768 - 256  # the library's bound on an automaton's table (bytes)
# Work-item sizes tried for the fastest family (log2 bytes; 0 = the
# library's default): Shift-Or: shortest work item; q-gram and automaton:
# start positions per thread range.  q-gram ranges stay at most 4 KiB: an
# item that falls back to the linear scan runs one thread per range, so
# long ranges would leave a dense short text to a few blocks.
TILES = {"shiftor": (0, 17, 19), "qgram": (0, 9, 11, 12), "dfa": (0, 12), "linear": (0,)}


def m_bucket(m: int) -> int:
    """floor(log2 m), capped at M_BUCKETS - 1 (same rule as the library)."""
    return min(M_BUCKETS - 1, max(0, int(m).bit_length() - 1))


def s_bucket(sigma: int) -> int:
    """0 for unknown, else floor(log2 sigma) clamped to 1..S_BUCKETS-1."""
    if sigma <= 0:
        return 0
    return max(1, min(S_BUCKETS - 1, int(sigma).bit_length() - 1))


def builtin(m: int, sigma: int = 0) -> dict:
    """The library's built-in choice for length m on an alphabet of sigma
    (tuning cell variant 0): Shift-Or up to m = 16, and up to m = 64 when
    sigma is 2 or 3; else the q-gram filter with the smallest q such that
    sigma**q >= 2**11 * m, clamped to 3..8 (sigma 4 when unknown)."""
    if m <= 16 or (m <= 64 and sigma in (2, 3)):
        return {"variant": "shiftor", "word_bits": 32 if m <= 32 else 64}
    sg = sigma if sigma >= 2 else 4
    q = min(8, max(3, math.ceil(math.log(2048.0 * m) / math.log(sg) - 1e-9)))
    return {"variant": "qgram", "q": min(q, m)}


def dfa_fits(p: bytes) -> bool:
    """The automaton of p has (m+1) x C two-byte entries, C = distinct bytes + 1."""
    return (len(p) + 1) * (len(set(p)) + 1) * 2 <= DFA_MAX_TABLE


def candidates(m: int, patterns=None) -> list[dict]:
    """Kernel families (with their parameter) able to serve length m; the
    automaton only when every given pattern's table fits."""
    out = []
    if m <= 32:
        out.append({"variant": "shiftor", "word_bits": 32})
    if m <= 64:
        out.append({"variant": "shiftor", "word_bits": 64})
    for q in (3, 4, 5, 6, 7, 8):
        if q <= m and m - q + 1 >= 2:
            out.append({"variant": "qgram", "q": q})
    if patterns is not None and patterns and all(dfa_fits(p) for p in patterns):
        out.append({"variant": "dfa"})
    return out


def cfg_key(cfg: dict) -> str:
    v = cfg["variant"]
    k = v + (f"{cfg.get('word_bits')}" if v == "shiftor" else f"q{cfg.get('q')}" if v == "qgram" else "")
    return k + (f"t{cfg['tile']}" if cfg.get("tile") else "")


def _time_batch(text, pats, sigma, cfg, reps, flush):
    import torch
    plans = prepare_many(pats, sigma_hint=sigma, **cfg)
    cnt = torch.zeros(len(plans), dtype=torch.int64, device=text.device)
    search_batch([(text, p, None, cnt[i:i + 1]) for i, p in enumerate(plans)])
    sync()
    c = cnt.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum(c)])
    out = torch.empty(max(int(c.sum()), 1), dtype=torch.int64, device=text.device)
    b = Batch([(text, p, out[int(offs[i]):int(offs[i + 1])], cnt[i:i + 1])
               for i, p in enumerate(plans)])
    ts = []
    for r in range(reps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.launch()
        e1.record()
        torch.cuda.synchronize()
        if r:
            ts.append(e0.elapsed_time(e1) / 1e3)
    sync()
    b.free()
    for p in plans:
        p.free()
    return statistics.median(ts)


def tune(sigmas=(2, 4, 8, 16, 32, 64, 128), ms=gen.SWEEP_M, n: int = 4 << 20, per: int = 100,
         reps: int = 3, seed: int = 101, apply: bool = True, verbose: bool = False,
         margin: float = 0.05) -> dict:
    """Measure every candidate for each (sigma, m) and return (and by
    default apply) the tuning table.  Cells not measured keep variant 0
    (the library's built-in rule).  `per` patterns per cell run as one
    batch: the ranking of the kernels depends on the batch size (a small
    batch gives short work items), so it should match the batches the
    table will serve.  A candidate replaces the built-in choice only when
    it is faster by more than `margin`, so that near-ties do not flip from
    run to run."""
    import torch

    from . import gen_text

    t0 = time.perf_counter()
    cells = [{"variant": 0, "q": 0, "word_bits": 0, "tile": 0} for _ in range(M_BUCKETS * S_BUCKETS)]
    report = []
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for sigma in sigmas:
        spec = gen.uniform_text(n, sigma, seed + sigma)
        text = torch.empty(n, dtype=torch.uint8, device="cuda")
        gen_text(text, 0, spec.key, sigma)
        sync()
        host = None
        for m in ms:
            offs = gen.pattern_offsets(n, m, per, seed * 7 + m)
            pats = [bytes(spec.window(o, m)) for o in offs]
            res = {}
            for cfg in candidates(m, pats):
                res[cfg_key(cfg)] = (_time_batch(text, pats, sigma, cfg, reps, flush), cfg)
            # Work-item sizes of the fastest family.
            top = res[min(res, key=lambda k: res[k][0])][1]
            for tile in TILES[top["variant"]][1:]:
                cfg = dict(top, tile=tile)
                res[cfg_key(cfg)] = (_time_batch(text, pats, sigma, cfg, reps, flush), cfg)
            best_key = min(res, key=lambda k: res[k][0])
            b = builtin(m, sigma)
            b_key = next((k for k, v in res.items() if v[1] == b), None)
            if b_key is not None and res[best_key][0] > (1.0 - margin) * res[b_key][0]:
                best_key = b_key
            best_t, best_cfg = res[best_key]
            idx = m_bucket(m) * S_BUCKETS + s_bucket(sigma)
            cells[idx] = {"variant": VARIANT_IDS[best_cfg["variant"]], "q": best_cfg.get("q", 0),
                          "word_bits": best_cfg.get("word_bits", 0), "tile": best_cfg.get("tile", 0)}
            row = {"sigma": sigma, "m": m, "best": best_key,
                   "gbs": {k: round(per * n / v[0] / 1e9, 1) for k, v in res.items()}}
            report.append(row)
            if verbose:
                print(json.dumps(row), flush=True)
        del host
    if apply:
        tuning_set(cells)
    return {"cells": cells, "report": report, "seconds": round(time.perf_counter() - t0, 2),
            "n": n, "patterns_per_cell": per}


def save(result: dict, path: str) -> None:
    with open(path, "w") as f:
        json.dump(result, f, indent=1)


def load(path: str, apply: bool = True) -> dict:
    with open(path) as f:
        result = json.load(f)
    if len(result["cells"]) != M_BUCKETS * S_BUCKETS:
        raise ValueError("tuning table has the wrong shape")
    if apply:
        tuning_set(result["cells"])
    return result


def current() -> list[dict]:
    return tuning_get()


# The table measured on GB300 with tune() (sigmas 2..128, the sweep's m, 100
# patterns a cell), loaded by bench.py unless it is asked to re-measure.
GB300_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.json")


if __name__ == "__main__":  # python -m paper_1012_2547_gb300.tuner out.json
    import sys
    r = tune(verbose=True)
    if len(sys.argv) > 1:
        save(r, sys.argv[1])
    print("tuned in", r["seconds"], "s")
