"""Serving loop: scheduling policy (CPU) and continuous batching (GPU)."""
import concurrent.futures as cf
import time

import numpy as np
import pytest

import oracle
from paper_1012_2547_gb300 import gen
from paper_1012_2547_gb300.serve import Policy, Request, length_class


def req(i, m, text_len=None, t=0.0, cap=16):
    text = None if text_len is None else np.zeros(text_len, np.uint8)
    return Request(i, b"a" * m, None if text is not None else "c", text, cap, t)


def test_length_class():
    assert [length_class(m) for m in (1, 2, 3, 4, 512, 5000)] == [0, 1, 1, 2, 9, 11]


def test_batches_take_one_class_in_arrival_order():
    p = Policy(budget_bytes=1 << 30, max_batch=3, workspace_per_batch=1 << 20)
    for i, m in enumerate([8, 2, 9, 12, 3, 15]):
        p.push(req(i, m))
    b, res, rej = p.take()
    assert [r.rid for r in b] == [0, 2, 3] and not rej      # class of m=8 (3): 8, 9, 12
    assert [r.rid for r in p.pending] == [1, 4, 5]           # others keep their order
    b2, res2, _ = p.take()
    assert [r.rid for r in b2] == [1, 4]                     # class 1: m = 2, 3
    assert p.used == res + res2
    p.release(res)
    b3, _, _ = p.take()
    assert [r.rid for r in b3] == [5]


def test_admission_respects_budget_and_rejects_impossible():
    ws = 1 << 20
    p = Policy(budget_bytes=ws + 3 * (1 << 20), max_batch=100, workspace_per_batch=ws)
    p.push(req(0, 8, text_len=10 << 20))                     # can never fit
    for i in range(1, 6):
        p.push(req(i, 8, text_len=(1 << 20) - 20000))
    b, reserved, rej = p.take()
    assert [r.rid for r in rej] == [0]
    assert 1 <= len(b) <= 3 and p.used <= p.budget
    b2, _, _ = p.take()
    assert b2 == []                                          # budget exhausted until release
    p.release(reserved)
    b3, _, _ = p.take()
    assert b3 and b3[0].rid == b[-1].rid + 1


def test_batch_output_cap():
    p = Policy(budget_bytes=1 << 40, max_batch=100, workspace_per_batch=0, max_batch_out_bytes=8 * 100)
    for i, cap in enumerate([60, 30, 20, 500, 10]):
        r = req(i, 8, cap=cap)
        p.push(r)
    b, _, _ = p.take()
    assert [r.rid for r in b] == [0, 1, 4]                   # 60 + 30 + 10 <= 100 positions
    b2, _, _ = p.take()
    assert [r.rid for r in b2] == [2]
    b3, _, _ = p.take()
    assert [r.rid for r in b3] == [3]                        # alone, though above the cap


def test_batch_scan_cap():
    """A batch scans at most max_batch_scan_bytes of text (corpus or own
    text); a request alone above the cap still runs, by itself."""
    p = Policy(budget_bytes=1 << 40, max_batch=100, workspace_per_batch=0,
               corpus_bytes={"c": 3 << 20}, max_batch_scan_bytes=8 << 20)
    p.push(req(0, 8))                          # corpus c: 3 MiB
    p.push(req(1, 8, text_len=4 << 20))        # own text: 4 MiB
    p.push(req(2, 8))                          # 3 MiB: over the cap (10 MiB)
    p.push(req(3, 8, text_len=1 << 20))        # 1 MiB: fits (8 MiB)
    p.push(req(4, 8, text_len=20 << 20))       # 20 MiB
    b, _, _ = p.take()
    assert [r.rid for r in b] == [0, 1, 3]
    b2, _, _ = p.take()
    assert [r.rid for r in b2] == [2]          # 3 + 20 MiB > 8 MiB
    b3, _, _ = p.take()
    assert [r.rid for r in b3] == [4]          # alone, though above the cap


def test_batch_scan_cap_grows_with_backlog():
    """With scan_backlog pending requests per step, the scan bound grows by
    one cap per step: a backlog drains in larger batches."""
    p = Policy(budget_bytes=1 << 40, max_batch=100, workspace_per_batch=0,
               corpus_bytes={"c": 4 << 20}, max_batch_scan_bytes=8 << 20, scan_backlog=4)
    for i in range(10):                        # 10 pending: bound 8 MiB x (1 + 10 // 4) = 24 MiB
        p.push(req(i, 8))
    b, _, _ = p.take()
    assert [r.rid for r in b] == list(range(6))
    b2, _, _ = p.take()                        # 4 pending: 16 MiB
    assert [r.rid for r in b2] == [6, 7, 8, 9]


def test_pinned_pool_size_classes():
    from paper_1012_2547_gb300.serve import PinnedPool
    for n in (1, 1 << 20, (1 << 20) + 1, 1_300_000, 3 << 20, (8 << 20) + 5, 1 << 31):
        c = PinnedPool.size_class(n)
        assert c >= n and c >= PinnedPool.MIN_BYTES
        assert c <= 1.25 * max(n, PinnedPool.MIN_BYTES) + 1     # under a fifth wasted


def test_batch_time_bound_and_rates():
    """A batch's estimated GPU time (scan bytes / scan rate + output bytes /
    copy rate) stays under max_batch_seconds, one step per scan_backlog
    pending requests; measured batches move the rates."""
    p = Policy(budget_bytes=1 << 40, max_batch=100, workspace_per_batch=0, corpus_bytes={"c": 1 << 30},
               max_batch_seconds=0.001, scan_rate=1e12, copy_rate=1e11, scan_backlog=100)
    for i in range(5):
        p.push(req(i, 8, cap=1000))            # 1.07 ms of scan each: one per batch
    b, _, _ = p.take()
    assert [r.rid for r in b] == [0]
    p.max_batch_seconds = 0.0025
    b, _, _ = p.take()
    assert [r.rid for r in b] == [1, 2]
    p.observe(4 << 30, 0.002, 0, 0.0)         # 2.1 TB/s measured: the estimate moves up
    assert 1e12 < p.scan_rate <= 1e12 * 1.25
    p.observe(4 << 30, 1e-9, 0, 0.0)           # an outlier counts at most 4x
    assert p.scan_rate <= 1e12 * 1.25 * 1.6


def test_ready_rules():
    p = Policy(budget_bytes=1 << 30, max_batch=2, max_wait=0.01)
    assert not p.ready(0.0, busy=0)
    p.push(req(0, 4, t=0.0))
    assert p.ready(0.0, busy=0)                               # idle GPU: go
    assert not p.ready(0.001, busy=1)                         # busy, young, not full
    assert p.ready(0.02, busy=1)                              # old enough
    p.push(req(1, 4, t=0.0))
    assert p.ready(0.0, busy=1)                               # full batch


@pytest.mark.gpu
def test_server_results_equal_alone_and_in_mix():
    import torch

    import paper_1012_2547_gb300 as smg
    from paper_1012_2547_gb300.serve import Server
    spec4 = gen.uniform_text(3 << 20, 4, 41)
    specE = gen.english_text(2 << 20, 42)
    corp4, corpE = spec4.host(), specE.host()
    dev = {"rand4": torch.from_numpy(corp4.copy()).cuda(), "english": torch.from_numpy(corpE.copy()).cuda()}
    rng = np.random.default_rng(5)
    key = gen.stream_key(7, 9)
    reqs = []
    for k in range(300):
        m = gen.log_uniform_int(key, k, 2, 512)
        if k % 10 < 7:
            name = "rand4" if k % 2 else "english"
            t = corp4 if name == "rand4" else corpE
            p = gen.substring_patterns(t, m, 1, seed=k)[0]
            reqs.append((p, name, None, t))
        else:
            n = int(4096 * (4096 ** rng.random()))
            t = rng.integers(0, 4, n, dtype=np.uint8)
            p = gen.substring_patterns(t, min(m, n), 1, seed=k)[0] if n >= m else bytes(m)
            reqs.append((p, None, t, t))
    reqs.append((b"\x00\x01", "rand4", None, corp4))          # dense: triggers a retry
    # cap_factor 0: first attempts get only first_cap positions, so dense
    # results take the truncation-and-retry path.
    srv = Server(dev, budget_bytes=2 << 30, streams=3, max_batch=64, sigma_hints={"rand4": 4, "english": 90},
                 cap_factor=0.0)
    futs = []
    for i, (p, name, own, _) in enumerate(reqs):
        futs.append(srv.submit(p, corpus=name, text=own))
        if i % 37 == 0:
            time.sleep(0.002)                                 # arrivals while batches run
    results = [f.result(timeout=120) for f in futs]
    srv.close()
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["batches"] > 1 and st["retries"] >= 1
    for (p, name, own, host), got in zip(reqs, results):
        alone = smg.search(dev[name] if name else torch.from_numpy(own).cuda(), p).cpu().numpy().astype(np.uint64)
        assert np.array_equal(got, alone)
        assert np.array_equal(got, oracle.kmp(host, p))


@pytest.mark.gpu
def test_pinned_pool_recycles_blocks():
    """A large result is a view of a pooled pinned block; the block goes
    back to the pool when the result is freed, and is then reused."""
    import gc

    import torch

    from paper_1012_2547_gb300.serve import PinnedPool
    pool = PinnedPool(torch)
    b, c = pool.take(3 << 20)
    b[: 8 * 5].view(torch.int64).copy_(torch.arange(5))
    a = pool.view(b, c, 5)
    assert a.dtype == np.uint64 and a.tolist() == [0, 1, 2, 3, 4]
    del b
    gc.collect()
    assert not pool._free[c]                                  # still backing `a`
    del a
    gc.collect()
    assert len(pool._free[c]) == 1
    b2, c2 = pool.take(3 << 20)
    assert c2 == c and pool.allocated_bytes == c             # reused, not reallocated
