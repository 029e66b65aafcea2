"""GPU parity at the benchmark configurations' full sizes, in the launch
configuration bench.py times (the committed GB300 tuning table loaded).

  * 8 GiB bandwidth configuration: for a substring and a random pattern of
    every m in {4, 32, 256, 1024}, the GPU's total over the whole text
    equals the oracle's count over the host's regenerated text (streamed in
    256 MiB chunks of start positions, each with its m-1 following bytes),
    every position in the last GiB (which holds the last byte) equals the
    oracle's, and every hit in 32 random 1 MiB windows elsewhere too; the
    dense a^m stress on the 64 MiB a^n-dominated prefix is exact in full.
  * batched configuration (i), 4096 patterns on one 1 GiB sigma = 20 skewed
    text, as one graph-captured batch with multi-pattern packing on: every
    query with m <= 3 (the densest outputs) and a stratified sample of at
    least 16 queries per length class floor(log2 m) are exact (count and
    every position).
  * the sweep's ten 4 MiB texts, every (text, m), 3 patterns each, as one
    graph-captured batch, all exact.
"""
import numpy as np
import pytest

import oracle
from paper_1012_2547_gb300 import gen, workloads

from _helpers import expect, torch

pytestmark = pytest.mark.gpu

CHUNK = 256 << 20
TAIL = 1 << 30


@pytest.fixture
def gb300_tuning():
    """The tuning table bench.py loads, reset afterwards."""
    import paper_1012_2547_gb300 as smg
    from paper_1012_2547_gb300 import tuner
    tuner.load(tuner.GB300_TABLE)
    yield
    smg.tuning_reset()


def _device_text(spec):
    import paper_1012_2547_gb300 as smg
    t = torch()
    out = t.empty(spec.n, dtype=t.uint8, device="cuda")
    if spec.kind == "uniform":
        smg.gen_text(out, 0, spec.key, spec.sigma)
    else:
        thr = t.tensor(np.asarray(spec.thresholds, dtype=np.uint32).view(np.int32), device="cuda")
        bm = t.tensor(np.asarray(spec.byte_map, dtype=np.uint8), device="cuda")
        smg.gen_text(out, 0, spec.key, 0, thr, bm)
    return out


def _range(got, lo, hi):
    """got[a:b] with lo <= got[a:b] < hi (got sorted, on the device)."""
    t = torch()
    a = int(t.searchsorted(got, t.tensor([lo], device=got.device)).item())
    b = int(t.searchsorted(got, t.tensor([hi], device=got.device)).item())
    return got[a:b]


def _check_windows(spec, got, pattern, lo_min, hi_max, rng, windows=32, width=1 << 20):
    m = len(pattern)
    for _ in range(windows):
        lo = int(rng.integers(lo_min, hi_max - width))
        win = spec.window(lo, width + m - 1)
        exp = oracle.naive(win, pattern).astype(np.int64) + lo
        assert np.array_equal(_range(got, lo, lo + width).cpu().numpy(), exp), (m, lo)


def test_bandwidth_config_8gib_full(gb300_tuning):
    import paper_1012_2547_gb300 as smg
    t = torch()
    n = workloads.BANDWIDTH_N
    w = workloads.bandwidth(n=n, per_m=1)  # one substring and one random pattern per m
    spec = w.specs[0]
    text = t.empty(n, dtype=t.uint8, device="cuda")
    smg.gen_text(text, 0, spec.key, 4)
    pre = workloads.DENSE_PREFIX
    host_pre = spec.window(0, pre).copy()
    gen.plant_prefix(host_pre, pre, 4096, seed=77)
    text[:pre].copy_(t.from_numpy(host_pre))
    smg.sync()
    plans = smg.prepare_many([q.pattern for q in w.queries], sigma_hint=4)
    got = []
    for q, plan in zip(w.queries, plans):
        g = smg.search(text, plan)
        assert g.dtype == t.int64
        if g.numel() > 1:
            assert bool((g[1:] > g[:-1]).all())
        got.append(g)

    # Totals over the whole text and exact positions over the last GiB, from
    # the host's regenerated text in chunks of start positions.
    mmax = max(len(q.pattern) for q in w.queries)
    totals = [0] * len(w.queries)
    for c in range(0, n, CHUNK):
        win = spec.window(c, CHUNK + mmax - 1)
        if c < pre:
            win[: pre - c] = host_pre[c:]
        for i, q in enumerate(w.queries):
            m = len(q.pattern)
            span = win[: min(CHUNK, n - c) + m - 1]
            if c >= n - TAIL:
                exp = oracle.naive_mt(span, q.pattern).astype(np.int64) + c
                gpu = _range(got[i], c, c + CHUNK).cpu().numpy()
                assert np.array_equal(gpu, exp), (m, c)
                totals[i] += len(exp)
            else:
                totals[i] += oracle.count_mt(span, q.pattern)
    for i, q in enumerate(w.queries):
        assert got[i].numel() == totals[i], (len(q.pattern), got[i].numel(), totals[i])

    rng = np.random.default_rng(9)
    for q, g in zip(w.queries, got):
        _check_windows(spec, g, q.pattern, pre, n - TAIL, rng)
    del got
    for q in workloads.bandwidth_dense():
        g = smg.search(text[:pre], q.pattern).cpu().numpy().astype(np.uint64)
        assert np.array_equal(g, expect(host_pre, q.pattern)), len(q.pattern)


def test_batched_shared_config_full(gb300_tuning):
    import paper_1012_2547_gb300 as smg
    t = torch()
    w = workloads.batched_shared()
    spec = w.specs[0]
    text = _device_text(spec)
    smg.sync()
    nq = len(w.queries)
    hint = w.queries[0].sigma_hint
    assert all(q.sigma_hint == hint for q in w.queries)
    plans = smg.prepare_many([q.pattern for q in w.queries], sigma_hint=hint)
    cnt = t.zeros(nq, dtype=t.int64, device="cuda")
    smg.search_batch([(text, plans[i], None, cnt[i:i + 1]) for i in range(nq)])
    smg.sync()
    c = cnt.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum(c)])
    out = t.empty(max(int(c.sum()), 1), dtype=t.int64, device="cuda")
    cnt2 = t.zeros(nq, dtype=t.int64, device="cuda")
    b = smg.Batch([(text, plans[i], out[int(offs[i]):int(offs[i + 1])], cnt2[i:i + 1]) for i in range(nq)],
                  graph=True)
    b.launch()
    smg.sync()
    assert t.equal(cnt, cnt2)

    ms = np.array([len(q.pattern) for q in w.queries])
    short = [i for i in range(nq) if ms[i] <= 3]
    rng = np.random.default_rng(17)
    strat = []
    for cls in range(1, 11):
        idx = [i for i in range(nq) if int(ms[i]).bit_length() - 1 == cls and ms[i] > 3]
        if idx:
            strat += rng.choice(idx, min(16, len(idx)), replace=False).tolist()
    assert len(strat) >= 128
    host = spec.host()
    last, exp = None, None
    # Equal patterns side by side: each distinct pattern runs the oracle once.
    for i in sorted(set(short) | set(strat), key=lambda i: (w.queries[i].pattern, i)):
        p = w.queries[i].pattern
        if p != last:
            last, exp = p, oracle.naive_mt(host, p)
        assert int(c[i]) == len(exp), (i, len(p))
        gpu = out[int(offs[i]):int(offs[i + 1])].cpu().numpy().astype(np.uint64)
        assert np.array_equal(gpu, exp), (i, len(p))
    b.free()


def test_sweep_config_subset_batched(gb300_tuning):
    """The sweep's ten 4 MiB texts, every m in {2, ..., 1024}, 3 patterns per
    (text, m), as one batch (the bench's launch form), all exact."""
    import paper_1012_2547_gb300 as smg
    t = torch()
    w = workloads.sweep(per_m=3)
    dev = [t.from_numpy(x).cuda() for x in w.texts]
    plans = [None] * len(w.queries)
    by_hint = {}
    for i, q in enumerate(w.queries):
        by_hint.setdefault(q.sigma_hint, []).append(i)
    for hint, idx in by_hint.items():
        for i, p in zip(idx, smg.prepare_many([w.queries[i].pattern for i in idx], sigma_hint=hint)):
            plans[i] = p
    cnt = t.zeros(len(w.queries), dtype=t.int64, device="cuda")
    smg.search_batch([(dev[q.text_id], plans[i], None, cnt[i:i + 1]) for i, q in enumerate(w.queries)])
    smg.sync()
    c = cnt.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum(c)])
    out = t.empty(max(int(c.sum()), 1), dtype=t.int64, device="cuda")
    b = smg.Batch([(dev[q.text_id], plans[i], out[int(offs[i]):int(offs[i + 1])], cnt[i:i + 1])
                   for i, q in enumerate(w.queries)], graph=True)
    b.launch()
    smg.sync()
    host = out.cpu().numpy().astype(np.uint64)
    for i, q in enumerate(w.queries):
        exp = oracle.kmp(w.texts[q.text_id], q.pattern) if len(q.pattern) > 64 else \
            oracle.naive_mt(w.texts[q.text_id], q.pattern)
        assert int(cnt[i].item()) == len(exp), (i, len(q.pattern))
        assert np.array_equal(host[int(offs[i]):int(offs[i + 1])], exp), (i, len(q.pattern))
    b.free()
