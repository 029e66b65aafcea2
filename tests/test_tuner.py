"""Autotuner: bucket rules (CPU) and tuned searches staying exact (GPU)."""
import numpy as np
import pytest

import oracle
from paper_1012_2547_gb300 import gen, tuner


def test_buckets_match_library_rule():
    assert [tuner.m_bucket(m) for m in (1, 2, 3, 4, 7, 8, 1024, 2047, 5000)] == [0, 1, 1, 2, 2, 3, 10, 10, 11]
    assert [tuner.s_bucket(s) for s in (0, 1, 2, 3, 4, 20, 90, 128, 256, 1000)] == [0, 1, 1, 1, 2, 4, 6, 7, 8, 8]


def test_candidates_respect_limits():
    for m in (1, 2, 5, 17, 33, 64, 65, 1024):
        for c in tuner.candidates(m):
            if c["variant"] == "shiftor":
                assert m <= c["word_bits"]
            else:
                assert c["q"] <= m


@pytest.mark.gpu
def test_tuned_table_applies_and_stays_exact():
    import torch

    import paper_1012_2547_gb300 as smg
    smg.tuning_reset()
    r = tuner.tune(sigmas=(4, 64), ms=(8, 64, 256), n=1 << 20, per=4, reps=1)
    cells = smg.tuning_get()
    assert cells == r["cells"]
    for row in r["report"]:
        i = tuner.m_bucket(row["m"]) * tuner.S_BUCKETS + tuner.s_bucket(row["sigma"])
        assert cells[i]["variant"] in (1, 2)
    rng = np.random.default_rng(3)
    for sigma in (4, 64):
        t = rng.integers(0, sigma, 300_000, dtype=np.uint8)
        dev = torch.from_numpy(t).cuda()
        for m in (8, 64, 256):
            p = gen.substring_patterns(t, m, 1, seed=m)[0]
            plan = smg.prepare(p, sigma_hint=sigma)
            got = smg.search(dev, plan).cpu().numpy().astype(np.uint64)
            assert np.array_equal(got, oracle.kmp(t, p)), (sigma, m, plan.info())
    smg.tuning_reset()


def test_committed_gb300_table_loads():
    import json
    import os

    from paper_1012_2547_gb300 import tuner
    assert os.path.exists(tuner.GB300_TABLE)
    r = tuner.load(tuner.GB300_TABLE, apply=False)
    assert len(r["cells"]) == tuner.M_BUCKETS * tuner.S_BUCKETS
    for c in r["cells"]:
        assert c["variant"] in (0, 1, 2, 3, 4)
        if c["variant"] == 2:
            assert 1 <= c["q"] <= 8
    with open(tuner.GB300_TABLE) as f:
        assert json.load(f)["patterns_per_cell"] == 100


def test_builtin_choice_rule():
    from paper_1012_2547_gb300 import tuner
    assert tuner.builtin(8)["variant"] == "shiftor" and tuner.builtin(8)["word_bits"] == 32
    assert tuner.builtin(16, 4)["variant"] == "shiftor"
    assert tuner.builtin(40, 2) == {"variant": "shiftor", "word_bits": 64}
    assert tuner.builtin(32, 4) == {"variant": "qgram", "q": 8}       # 4**8 = 2**11 * 32
    assert tuner.builtin(40) == {"variant": "qgram", "q": 8}          # unknown sigma counts as 4
    assert tuner.builtin(100, 20) == {"variant": "qgram", "q": 5}     # ceil(log 204800 / log 20)
    assert tuner.builtin(1024, 128) == {"variant": "qgram", "q": 3}
    assert tuner.builtin(1024, 2) == {"variant": "qgram", "q": 8}
    for m in (8, 40, 100, 1024):
        for sg in (2, 4, 20, 128):
            assert tuner.builtin(m, sg) in tuner.candidates(m)


def test_library_sigma_buckets():
    """The library reads the cell of floor(log2 sigma): a config put in the
    sigma = 4 cell of m = 32 serves sigma hints 4 to 7, the sigma = 2 cell
    serves 2 and 3, the sigma = 8 cell 8 (no GPU: plan images only)."""
    import paper_1012_2547_gb300 as smg
    cells = [{"variant": 0, "q": 0, "word_bits": 0, "tile": 0} for _ in range(tuner.M_BUCKETS * tuner.S_BUCKETS)]
    mb = tuner.m_bucket(32)
    cells[mb * tuner.S_BUCKETS + 1] = {"variant": 1, "q": 0, "word_bits": 64, "tile": 0}
    cells[mb * tuner.S_BUCKETS + 2] = {"variant": 2, "q": 5, "word_bits": 0, "tile": 0}
    cells[mb * tuner.S_BUCKETS + 3] = {"variant": 2, "q": 7, "word_bits": 0, "tile": 0}
    smg.tuning_set(cells)
    try:
        p = bytes(range(32))
        got = {sg: smg.plan_image(p, sigma_hint=sg)[1] for sg in (2, 3, 4, 7, 8)}
        for sg in (2, 3):
            assert got[sg]["variant"] == "shiftor" and got[sg]["word_bits"] == 64, sg
        for sg in (4, 7):
            assert got[sg]["variant"] == "qgram" and got[sg]["q"] == 5, sg
        assert got[8]["variant"] == "qgram" and got[8]["q"] == 7
    finally:
        smg.tuning_reset()
