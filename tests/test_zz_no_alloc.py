"""GPU test of sm_search_noalloc, the entry point for callers that cannot
allocate device memory (stream capture, pre-reserved serving memory,
framework-owned memory).  It must return exactly what sm_search returns,
on two calls in a row that reuse its static scratch.  Collected last so that
a run stopping at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_1012_2547_gb300 import _lib, gen

pytestmark = pytest.mark.gpu


def _call(fn, text, pattern, out, cnt, stream):
    return fn(text.data_ptr(), text.numel(), pattern, len(pattern), out.data_ptr(), out.numel(),
              cnt.data_ptr(), stream)


def test_noalloc_matches_sm_search_twice():
    import torch
    lib = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(123)
    cases = []
    for sigma, n, off in ((4, 1 << 20, 0), (2, 300_001, 3), (128, 2_000_003, 7)):
        t = rng.integers(0, sigma, n, dtype=np.uint8)
        buf = torch.zeros(n + 64, dtype=torch.uint8, device="cuda")
        buf[off:off + n] = torch.from_numpy(t).cuda()
        text = buf[off:off + n]
        for m in (1, 2, 8, 17, 31, 40, 64):
            o = int(rng.integers(0, n - m))
            cases.append((text, bytes(t[o:o + m])))
    cases.append((cases[0][0], bytes(1000 * [0])[:64]))  # no occurrence expected
    for text, p in cases:
        ref_out = torch.full((4096,), -1, dtype=torch.int64, device="cuda")
        ref_cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        assert _call(lib.sm_search, text, p, ref_out, ref_cnt, stream) == 0
        assert lib.sm_sync(stream) == 0
        total = int(ref_cnt.item())
        for _ in range(2):  # second call reuses (and must clear) the scratch
            out = torch.full((4096,), -1, dtype=torch.int64, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            assert _call(lib.sm_search_noalloc, text, p, out, cnt, stream) == 0
            torch.cuda.synchronize()
            assert int(cnt.item()) == total
            k = min(total, 4096)
            assert torch.equal(out[:k], ref_out[:k])
            assert bool((out[k:] == -1).all())
