"""The multi-rank path of bench.py on CPU: two processes joined over gloo
(127.0.0.1), the max-over-ranks timing and the whole-job throughput of
independent replicas (the single-grid solve does not shard)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    try:
        r, w = bench.dist_init()
        local_ms = 10.0 * (rank + 1)  # rank 1 is the slow one
        max_ms = bench.dist_max(local_ms, w)
        bench.dist_barrier(w)
        rate = bench.job_rate(1000, 5, w, max_ms)
        q.put((r, w, max_ms, rate))
    finally:
        if dist.is_initialized():
            dist.destroy_process_group()


def test_two_gloo_ranks_time_by_the_slowest_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[:2] for o in out] == [(0, 2), (1, 2)]
    # both ranks see the slowest rank's 20 ms; 2 replicas x 5 steps x 1000
    # unknowns in 20 ms
    for _, _, max_ms, rate in out:
        assert max_ms == 20.0
        assert rate == pytest.approx(2 * 5 * 1000 / 0.020)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.dist_max(3.5, 1) == 3.5
    assert bench.job_rate(10, 2, 1, 4.0) == pytest.approx(10 * 2 / 0.004)
