"""The multi-replica path of bench.py (one process per GPU, no data-path collective):
the slowest rank's time is taken over a gloo process group of two CPU ranks, and the
whole-job rate counts every replica's work."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank  # rank 1 is the slower replica
    total = bench.max_over_ranks(local_ms)
    q.put((rank, total, bench.aggregate_rate(1e9, 4, world, total)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_time():
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
    assert [o[1] for o in out] == [150.0, 150.0]
    # 2 replicas x 1e9 units x 4 steps in 150 ms
    assert abs(out[0][2] - 2 * 1e9 * 4 / 0.150) < 1.0


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.aggregate_rate(10.0, 2, 1, 1000.0) == 20.0
