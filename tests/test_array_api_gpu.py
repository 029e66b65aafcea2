"""The array form of the batch API (prepare_array -> PlanArray,
query_array, search_batch_async_array in caller workspace): every query's
positions and count equal the oracle's; a PlanArray holds the same plans
as prepare_many and frees them together."""
import numpy as np
import pytest

import oracle

from _helpers import to_dev, torch

pytestmark = pytest.mark.gpu


def _workload():
    rng = np.random.default_rng(5)
    texts = [rng.integers(0, s, n, dtype=np.uint8) for s, n in ((2, 70_001), (4, 300_017), (20, 1 << 20))]
    pats, tid = [], []
    for ti, t in enumerate(texts):
        for m in (1, 2, 3, 4, 5, 7, 8, 12, 16, 24, 31, 48, 64, 100, 257, 1000):
            for k in range(2):
                o = int(rng.integers(0, len(t) - m))
                p = t[o:o + m].tobytes() if k == 0 else rng.integers(0, 4, m, dtype=np.uint8).tobytes()
                pats.append(p)
                tid.append(ti)
    return texts, pats, np.asarray(tid)


@pytest.mark.parametrize("joined", [False, True])
def test_prepare_array_async_batch_matches_oracle(joined):
    import paper_1012_2547_gb300 as smg
    t = torch()
    texts, pats, tid = _workload()
    texts_d = [to_dev(x) for x in texts]
    exp = [oracle.kmp(texts[tid[i]], p) for i, p in enumerate(pats)]
    counts = np.array([len(e) for e in exp], dtype=np.uint64)
    offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.uint64)
    out = t.full((int(offs[-1]) + 1,), -1, dtype=t.int64, device="cuda")
    cnt = t.zeros(len(pats), dtype=t.int64, device="cuda")
    arg = (b"".join(pats), np.array([len(p) for p in pats], dtype=np.uint32)) if joined else pats
    plans = smg.prepare_array(arg, sigma_hint=4)
    assert len(plans) == len(pats)
    ref = smg.prepare_many(pats, sigma_hint=4)
    for i in range(0, len(pats), 7):
        a, b = plans.info(i), ref[i].info()
        assert (a.m, a.variant, a.kernel, a.q) == (b.m, b.variant, b.kernel, b.q)
    qa = smg.query_array(np.array([texts_d[i].data_ptr() for i in tid], dtype=np.uint64),
                         np.array([len(texts[i]) for i in tid], dtype=np.uint64), plans,
                         np.uint64(out.data_ptr()) + 8 * offs[:-1], counts,
                         np.uint64(cnt.data_ptr()) + 8 * np.arange(len(pats), dtype=np.uint64))
    ws_bytes = smg.batch_workspace_size_array(qa)
    ws = t.empty(ws_bytes + 256, dtype=t.uint8, device="cuda")
    smg.search_batch_async_array(qa, (ws.data_ptr() + 255) & ~255, ws_bytes)
    smg.sync()
    got_cnt = cnt.cpu().numpy().astype(np.uint64)
    got = out.cpu().numpy().astype(np.uint64)
    assert np.array_equal(got_cnt, counts)
    for i, e in enumerate(exp):
        assert np.array_equal(got[int(offs[i]):int(offs[i + 1])], e), (i, len(pats[i]))
    plans.free()
    plans.free()  # a second free is a no-op
    assert plans.handles is None
    for p in ref:
        p.free()


def test_prepare_array_empty():
    import paper_1012_2547_gb300 as smg
    pa = smg.prepare_array([])
    assert len(pa) == 0
    pa.free()
