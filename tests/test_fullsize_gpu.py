"""GPU parity at the benchmark configurations' full sizes, in the launch
configuration bench.py times.  Outputs too large for the oracle are checked
on samples it can compute: windows of the text (every hit inside, and no
other), single reported positions (the text there equals the pattern), and
the properties that hold at any size (strictly increasing positions)."""
import numpy as np
import pytest

import oracle
from paper_1012_2547_gb300 import gen, workloads

from _helpers import expect, torch

pytestmark = pytest.mark.gpu


def _check_windows(spec, got, pattern, lo_min, n, rng, windows=4, width=1 << 20):
    t = torch()
    m = len(pattern)
    for _ in range(windows):
        lo = int(rng.integers(lo_min, n - width))
        hi = lo + width
        win = spec.window(lo, width + m - 1)
        exp = oracle.naive(win, pattern).astype(np.int64) + lo
        a = int(t.searchsorted(got, t.tensor([lo], device=got.device)).item())
        b = int(t.searchsorted(got, t.tensor([hi], device=got.device)).item())
        assert np.array_equal(got[a:b].cpu().numpy(), exp), (m, lo)


def test_bandwidth_config_8gib_sampled():
    """8 GiB uniform sigma = 4 text, m in {4, 32, 256, 1024}, a substring and
    a random pattern each, plus a^m on the 64 MiB a^n-dominated prefix."""
    import paper_1012_2547_gb300 as smg
    t = torch()
    n = workloads.BANDWIDTH_N
    w = workloads.bandwidth(n=n, per_m=1)
    spec = w.specs[0]
    text = t.empty(n, dtype=t.uint8, device="cuda")
    smg.gen_text(text, 0, spec.key, 4)
    pre = workloads.DENSE_PREFIX
    host_pre = spec.window(0, pre).copy()
    gen.plant_prefix(host_pre, pre, 4096, seed=77)
    text[:pre].copy_(t.from_numpy(host_pre))
    smg.sync()
    rng = np.random.default_rng(9)
    for q in w.queries:
        m = len(q.pattern)
        got = smg.search(text, q.pattern)
        assert got.dtype == t.int64
        if got.numel() > 1:
            assert bool((got[1:] > got[:-1]).all())
        # single reported positions: the text there is the pattern
        if got.numel():
            idx = t.randint(0, got.numel(), (min(256, got.numel()),), device="cuda")
            for pos in got[idx].cpu().numpy().tolist():
                if pos >= pre:
                    assert bytes(spec.window(pos, m)) == q.pattern
        _check_windows(spec, got, q.pattern, pre, n, rng)
        del got
    for q in workloads.bandwidth_dense():
        got = smg.search(text[:pre], q.pattern).cpu().numpy().astype(np.uint64)
        assert np.array_equal(got, expect(host_pre, q.pattern)), len(q.pattern)


def test_sweep_config_subset_batched():
    """The sweep's ten 4 MiB texts, every m in {2, ..., 1024}, 3 patterns per
    (text, m), as one batch (the bench's launch form), all exact."""
    import paper_1012_2547_gb300 as smg
    t = torch()
    w = workloads.sweep(per_m=3)
    dev = [t.from_numpy(x).cuda() for x in w.texts]
    plans = smg.prepare_many([q.pattern for q in w.queries])
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
