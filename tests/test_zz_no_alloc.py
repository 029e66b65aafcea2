"""GPU test of sm_search_noalloc, the entry point for callers that may not
allocate device memory while they serve requests (serving loops that reserve
all their memory at start-up, plugins whose host framework owns every device
byte).  It must return exactly what sm_search returns, on two calls in a row
that reuse its static scratch, and what the CPU oracle returns.  Collected
last so that a run stopping at the first failure has already run every other
test."""
import numpy as np
import pytest

import oracle
from paper_1012_2547_gb300 import _lib

pytestmark = pytest.mark.gpu

CAP = 4096


def _call(fn, text, pattern, out, cnt, stream):
    return fn(text.data_ptr(), text.numel(), pattern, len(pattern), out.data_ptr(), out.numel(),
              cnt.data_ptr(), stream)


def _cases(torch):
    rng = np.random.default_rng(123)
    cases = []
    for sigma, n, off in ((4, 1 << 20, 0), (2, 300_001, 3), (128, 2_000_003, 7)):
        t = rng.integers(0, sigma, n, dtype=np.uint8)
        buf = torch.zeros(n + 64, dtype=torch.uint8, device="cuda")
        buf[off:off + n] = torch.from_numpy(t).cuda()
        text = buf[off:off + n]
        for m in (1, 2, 8, 17, 31, 40, 64):
            o = int(rng.integers(0, n - m))
            cases.append((text, t, bytes(t[o:o + m])))
    cases.append((cases[0][0], cases[0][1], bytes(64)))  # byte 0 runs of 64: none expected
    return cases


def test_noalloc_matches_sm_search_twice():
    import torch
    lib = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream
    for text, _, p in _cases(torch):
        ref_out = torch.full((CAP,), -1, dtype=torch.int64, device="cuda")
        ref_cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        assert _call(lib.sm_search, text, p, ref_out, ref_cnt, stream) == 0
        assert lib.sm_sync(stream) == 0
        total = int(ref_cnt.item())
        for _ in range(2):  # the second call reuses (and must clear) the scratch
            out = torch.full((CAP,), -1, dtype=torch.int64, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            l0 = lib.sm_kernel_launches()
            assert _call(lib.sm_search_noalloc, text, p, out, cnt, stream) == 0
            assert lib.sm_kernel_launches() - l0 == 3
            torch.cuda.synchronize()
            assert int(cnt.item()) == total
            k = min(total, CAP)
            assert torch.equal(out[:k], ref_out[:k])
            assert bool((out[k:] == -1).all())


def test_noalloc_matches_oracle():
    """Every case straight against the oracle (positions below the cap and
    the total), so the result does not rest on sm_search alone."""
    import torch
    lib = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream
    for text, host, p in _cases(torch):
        exp = oracle.naive(host, p)
        for _ in range(2):
            out = torch.full((CAP,), -1, dtype=torch.int64, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            assert _call(lib.sm_search_noalloc, text, p, out, cnt, stream) == 0
            torch.cuda.synchronize()
            assert int(cnt.item()) == len(exp), (len(p), len(host))
            k = min(len(exp), CAP)
            assert np.array_equal(out[:k].cpu().numpy().astype(np.uint64), exp[:k])
