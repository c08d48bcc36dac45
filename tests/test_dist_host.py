"""Multi-rank host logic of bench.py on CPU: two gloo ranks (127.0.0.1).

Covers the rank/world-size read from the environment, the max-over-ranks
reduction of step times, the whole-job weak-scaling arithmetic, and that the
reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method="env://")
    try:
        got_ws, got_rank, got_local = bench._dist()
        mx = bench.max_over_ranks(10.0 + 5.0 * rank, got_ws, "cpu")
        ref = bench.run_reference(type("A", (), {"steps": 1, "warmup": 3})(), None) \
            if rank == 1 else "skipped"
        q.put((rank, got_ws, got_rank, got_local, mx, ref))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got_ws, got_rank, got_local, mx, ref in res:
        assert (got_ws, got_rank, got_local) == (2, rank, rank)
        assert mx == 15.0                       # the slower rank's time, on every rank
    assert res[1][5] is None                    # reference arm: rank 1 returns without work


def test_whole_job_is_weak_scaling_sum():
    sys.path.insert(0, ROOT)
    import bench
    v1, f1 = bench.whole_job(1280, 720, 64, 1.25, 1)
    v2, f2 = bench.whole_job(1280, 720, 64, 1.25, 2)
    assert v1 == pytest.approx(1280 * 720 * 64 / 1.25e-3 * 1e-6)
    assert (v2, f2) == pytest.approx((2 * v1, 2 * f1))
    assert f1 == pytest.approx(800.0)
