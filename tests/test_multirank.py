"""The multi-process side of bench.py on CPU: world_size-2 gloo ranks.

bench.py runs one process per GPU ("replicas only": no data-path
collective); the ranks meet in a barrier around the timed region and the
step time is the maximum over ranks.  These tests run that aggregation over
gloo on the host, and check that the reference arm runs on rank 0 alone."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    w, r, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        bench.barrier(w)
        step = 0.010 * (r + 1)                       # rank 1 is the slower one
        worst = bench.max_over_ranks(step, w, "cpu")
        scanned = 1_000_000                          # bytes one rank scans per step
        value = w * scanned / worst                  # whole-job aggregate, as bench.py reports it
        bench.barrier(w)
        out.put((r, worst, value))
    finally:
        dist.destroy_process_group()


def test_barrier_and_max_over_ranks_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    for _, worst, value in res:
        assert worst == pytest.approx(0.020)          # the max, seen by every rank
        assert value == pytest.approx(2 * 1_000_000 / 0.020)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.25, 1) == 1.25
    bench.barrier(1)                                  # no process group needed


def test_reference_arm_only_on_rank_0():
    """Under torchrun the reference arm prints on rank 0 only; other ranks
    exit 0 without work (and without a process group)."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(_free_port()))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "1"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
