"""The N > 1 path of bench.py on CPU: two gloo ranks, each an independent
replica with its own seed; the job's time is the slowest rank's and the
value counts every rank's trials."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = str(rank)
    os.environ["WORLD_SIZE"] = str(world)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    from paper_1508_02748_gb300 import workloads
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank
    total = bench.reduce_max_ms(local_ms, world, "cpu")
    w = workloads.REWL_L8
    seed = w.seed(bench.replica_seed_index(rank))
    r, ws, _ = bench.dist_env()
    q.put((rank, total, seed, r, ws))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_and_distinct_seeds():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[1] for o in out] == [150.0, 150.0]          # max over ranks on every rank
    assert out[0][2] != out[1][2]                          # independent replicas
    assert [(o[3], o[4]) for o in out] == [(0, 2), (1, 2)]


def test_aggregate_rate_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench
    v1 = bench.aggregate_rate(360000, 10, 1, 20.0)
    v2 = bench.aggregate_rate(360000, 10, 2, 20.0)
    assert v1 == pytest.approx(360000 * 10 / 0.02)
    assert v2 == pytest.approx(2 * v1)
