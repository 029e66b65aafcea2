"""Shared helpers of the GPU tests: upload, search through the C ABI, compare."""
import numpy as np

import oracle


def torch():
    import torch as _t
    return _t


def to_dev(arr: np.ndarray, offset: int = 0):
    """Copy a uint8 array to the GPU, starting `offset` bytes into a fresh
    allocation (offset != 0 gives a text pointer that is not 16-aligned)."""
    t = torch()
    buf = t.empty(len(arr) + offset + 64, dtype=t.uint8, device="cuda")
    a = np.ascontiguousarray(arr)
    if not a.flags.writeable:  # torch wants writable arrays
        a = a.copy()
    buf[offset: offset + len(arr)] = t.from_numpy(a).cuda()
    return buf[offset: offset + len(arr)]


def gpu_search(text_dev, pattern: bytes, variant="auto", q=0, word_bits=0, tile=0, cap=None):
    import paper_1012_2547_gb300 as smg
    t = torch()
    plan = smg.prepare(pattern, variant=variant, q=q, word_bits=word_bits, tile=tile)
    n = text_dev.numel()
    if cap is None:
        cnt = t.zeros(1, dtype=t.int64, device="cuda")
        smg.search_into(text_dev, plan, None, cnt, n=n, cap=0)
        smg.sync()
        cap = int(cnt.item())
    out = t.full((max(cap, 1),), -1, dtype=t.int64, device="cuda")
    cnt = t.zeros(1, dtype=t.int64, device="cuda")
    smg.search_into(text_dev, plan, out, cnt, n=n, cap=cap)
    smg.sync()
    total = int(cnt.item())
    return out[: min(cap, total)].cpu().numpy().astype(np.uint64), total, plan


DFA_MAX_TABLE = 32768 - 256  # the library's bound on an automaton's table (bytes)


def dfa_fits(p: bytes) -> bool:
    """The automaton of p has (m+1) x C two-byte entries, C = distinct bytes + 1."""
    return (len(p) + 1) * (len(set(p)) + 1) * 2 <= DFA_MAX_TABLE


def variants_for(m: int, p: bytes | None = None):
    """(variant, q, word_bits) configurations able to serve length m (and the
    automaton when pattern p is given and its table fits)."""
    out = [("auto", 0, 0), ("linear", 0, 0)]
    if p is not None and dfa_fits(p):
        out.append(("dfa", 0, 0))
    if m <= 32:
        out.append(("shiftor", 0, 32))
    if m <= 64:
        out.append(("shiftor", 0, 64))
    for q in sorted({1, min(m, 3), min(m, 8)}):
        out.append(("qgram", q, 0))
    return out


def expect(text: np.ndarray, pattern: bytes) -> np.ndarray:
    if len(pattern) > 64 or len(text) > (1 << 22):
        return oracle.kmp(text, pattern)
    return oracle.naive(text, pattern)
