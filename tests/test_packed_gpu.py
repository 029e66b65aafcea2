"""GPU parity of multi-pattern packs (several Shift-And patterns of one text
scanned in one 32-bit state): a packed batch equals the unpacked batch and
the oracle, for mixed pattern lengths in one pack, unaligned texts, several
tiles with ragged tails, truncation, and a dense text that sends every item
down the per-pattern fallback."""
import numpy as np
import pytest

import oracle
from paper_1012_2547_gb300 import gen

from _helpers import to_dev, torch

pytestmark = pytest.mark.gpu


def _run(dev, plans, pack, caps=None):
    import paper_1012_2547_gb300 as smg
    t = torch()
    nq = len(plans)
    cnt = t.zeros(nq, dtype=t.int64, device="cuda")
    if caps is None:
        smg.search_batch([(dev, p, None, cnt[i:i + 1]) for i, p in enumerate(plans)])
        smg.sync()
        caps = cnt.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum(caps)])
    out = t.full((max(int(offs[-1]), 1),), -1, dtype=t.int64, device="cuda")
    cnt.zero_()
    b = smg.Batch([(dev, p, out[int(offs[i]):int(offs[i + 1])], cnt[i:i + 1]) for i, p in enumerate(plans)],
                  graph=True, pack=pack)
    b.launch()
    smg.sync()
    b.free()
    host = out.cpu().numpy().astype(np.uint64)
    return [host[int(offs[i]):int(offs[i + 1])] for i in range(nq)], cnt.cpu().numpy()


@pytest.mark.parametrize("sigma,n", [(4, 3_000_017), (20, 1_500_001), (256, 700_003)])
def test_packed_equals_unpacked_and_oracle(sigma, n):
    import paper_1012_2547_gb300 as smg
    rng = np.random.default_rng(sigma)
    t = rng.integers(0, sigma, n, dtype=np.uint8)
    ms = [m for m in range(2, 17) if m * np.log2(sigma) >= 14] * 3
    pats = []
    for k, m in enumerate(ms):
        if k % 3 == 2:
            pats.append(bytes(rng.integers(0, sigma, m, dtype=np.uint8)))
        else:
            pats.append(gen.substring_patterns(t, m, 1, seed=1000 * sigma + k)[0])
    # plant some occurrences so every pattern has hits
    for k, p in enumerate(pats):
        for o in rng.integers(0, n - len(p), 5):
            t[o:o + len(p)] = np.frombuffer(p, np.uint8)
    for off in (0, 9):
        dev = to_dev(t, off)
        plans = smg.prepare_many(pats, sigma_hint=sigma)
        packed, cp = _run(dev, plans, True)
        plain, cu = _run(dev, plans, False)
        for i, p in enumerate(pats):
            exp = oracle.naive(t, p)
            assert cp[i] == len(exp) and cu[i] == len(exp), (sigma, off, len(p))
            assert np.array_equal(packed[i], exp), (sigma, off, len(p))
            assert np.array_equal(plain[i], exp), (sigma, off, len(p))


def test_packed_truncation_keeps_first_positions():
    import paper_1012_2547_gb300 as smg
    rng = np.random.default_rng(3)
    t = rng.integers(0, 64, 2_000_000, dtype=np.uint8)
    pats = [gen.substring_patterns(t, m, 1, seed=m)[0] for m in (4, 5, 6, 7, 3, 3)]
    for p in pats:
        for o in rng.integers(0, len(t) - 8, 40):
            t[o:o + len(p)] = np.frombuffer(p, np.uint8)
    dev = to_dev(t)
    plans = smg.prepare_many(pats, sigma_hint=64)
    exp = [oracle.naive(t, p) for p in pats]
    caps = np.array([max(len(e) // 2, 1) for e in exp])
    got, cnt = _run(dev, plans, True, caps)
    for i in range(len(pats)):
        assert cnt[i] == len(exp[i])                            # the true count
        assert np.array_equal(got[i], exp[i][:caps[i]])


def test_dense_text_falls_back_exactly():
    """Patterns packed on a sparse-alphabet hint, searched in a text made of
    the patterns' own bytes: every work item overflows its records and is
    rewritten by the per-pattern pass."""
    import paper_1012_2547_gb300 as smg
    n = 600_001
    t = np.zeros(n, dtype=np.uint8)
    t[::7] = 1
    pats = [bytes(m) for m in (2, 3, 4, 5, 6)] + [b"\x00\x01", b"\x01\x00\x00"]
    dev = to_dev(t, 3)
    plans = smg.prepare_many(pats, sigma_hint=256)               # claims sparse, is dense
    got, cnt = _run(dev, plans, True)
    for i, p in enumerate(pats):
        exp = oracle.naive(t, p)
        assert cnt[i] == len(exp)
        assert np.array_equal(got[i], exp), len(p)


def test_moderately_dense_pack_lane_reextraction():
    """Packs denser than their alphabet hint says (sigma = 4 text, hint 256):
    lanes with more records than they keep in registers extract them again
    from the staged segment; results stay exact."""
    import paper_1012_2547_gb300 as smg
    rng = np.random.default_rng(11)
    t = rng.integers(0, 4, 2_500_003, dtype=np.uint8)
    pats = [gen.substring_patterns(t, m, 1, seed=200 + k)[0] for k, m in enumerate((5, 5, 6, 6, 5, 5))]
    dev = to_dev(t, 5)
    plans = smg.prepare_many(pats, sigma_hint=256)
    packed, cp = _run(dev, plans, True)
    for i, p in enumerate(pats):
        exp = oracle.naive(t, p)
        assert cp[i] == len(exp)
        assert np.array_equal(packed[i], exp), len(p)


def test_shared_long_text_interleaved_items():
    """Queries of every kernel family on one 40 MiB text (long enough for the
    batch to interleave their work items by text position) plus queries on
    a second long text and on short texts, as one batch and as a replayed
    graph: every result equals the oracle's."""
    import torch

    import paper_1012_2547_gb300 as smg
    rng = np.random.default_rng(77)
    n = 40 << 20
    big = [rng.integers(0, 4, n, dtype=np.uint8), rng.integers(0, 64, n, dtype=np.uint8)]
    big[0][: 1 << 20] = 0                                    # a dense stretch for a^m patterns
    small = [rng.integers(0, 4, 300_000, dtype=np.uint8)]
    texts = big + small
    dev = [torch.from_numpy(t).cuda() for t in texts]
    items = []
    for ti, t in enumerate(texts):
        for m in (2, 4, 8, 12, 16, 17, 24, 32, 40, 64, 100, 300, 1000):
            for r in range(2):
                o = int(rng.integers(0, len(t) - m))
                items.append((ti, bytes(t[o:o + m])))
        items.append((ti, bytes(17)))                        # a^17: dense where t is 0
        items.append((ti, bytes(100)))
    plans = [smg.prepare(p, sigma_hint=4 if ti != 1 else 64) for ti, p in items]
    cnt = torch.zeros(len(items), dtype=torch.int64, device="cuda")
    smg.search_batch([(dev[ti], plans[i], None, cnt[i:i + 1]) for i, (ti, _) in enumerate(items)])
    smg.sync()
    c = cnt.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum(c)])
    for graph in (False, True):
        out = torch.full((max(int(c.sum()), 1),), -1, dtype=torch.int64, device="cuda")
        cnt2 = torch.zeros_like(cnt)
        qs = [(dev[ti], plans[i], out[int(offs[i]):int(offs[i + 1])], cnt2[i:i + 1]) for i, (ti, _) in enumerate(items)]
        if graph:
            b = smg.Batch(qs, graph=True)
            b.launch()
            b.launch()
            smg.sync()
            b.free()
        else:
            smg.search_batch(qs)
            smg.sync()
        host = out.cpu().numpy().astype(np.uint64)
        assert torch.equal(cnt, cnt2)
        for i, (ti, p) in enumerate(items):
            exp = oracle.kmp(texts[ti], p)
            assert int(c[i]) == len(exp), (ti, len(p))
            assert np.array_equal(host[int(offs[i]):int(offs[i + 1])], exp), (ti, len(p), graph)
