"""The N > 1 path of bench.py (replicas only: every rank runs the whole workload) on the CPU
with two gloo ranks: the timed region is closed by the slowest rank and the whole-job rate
counts every replica's work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [3.0, 5.0][rank]
    mx = bench.max_over_ranks(ms, world)
    rate = bench.whole_job_rate(2e9, mx, world)
    dist.barrier()
    q.put((rank, mx, rate))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [5.0, 5.0]
    # 2 replicas x 2e9 flop in 5 ms = 800 GFLOP/s
    assert all(abs(o[2] - 800.0) < 1e-9 for o in out)


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(7.5, 1) == 7.5
    assert bench.whole_job_rate(1e9, 1.0, 1) == 1000.0
