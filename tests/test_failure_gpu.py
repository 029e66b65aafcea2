"""Failure reporting on the GPU without a fault: a bounded device-side wait
on a flag that nothing sets runs out, the kernel returns, the host reads
SM_ETIMEOUT once, and the stream and context go on working."""
import time

import numpy as np
import pytest

from _helpers import gpu_search, to_dev

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_is_reported_and_the_context_survives():
    import paper_1012_2547_gb300 as smg
    from paper_1012_2547_gb300 import _lib
    lib = _lib.load()
    smg.sync()
    t0 = time.perf_counter()
    assert lib.sm_selftest_wait(None) == _lib.SM_OK
    st = lib.sm_sync(None)
    dt = time.perf_counter() - t0
    assert st == _lib.SM_ETIMEOUT
    assert 1.0 < dt < 60.0                       # the wait's bound is 2 s of device time
    assert lib.sm_sync(None) == _lib.SM_OK       # reported once, then cleared
    with pytest.raises(smg.SmError):             # the Python wrapper raises on it
        lib.sm_selftest_wait(None)
        smg.sync()
    n = 100_003
    got, total, _ = gpu_search(to_dev(np.zeros(n, dtype=np.uint8)), bytes(5))
    assert total == n - 4 and np.array_equal(got, np.arange(n - 4, dtype=np.uint64))
    assert lib.sm_sync(None) == _lib.SM_OK
