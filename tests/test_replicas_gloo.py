"""Multi-rank host logic with world size 2 on the gloo backend (CPU): the
round-robin partition of independent solves, the max-over-ranks timing the
benchmark reports and the gathering of per-solve results."""
import os

import pytest
import torch.multiprocessing as mp

from paper_1503_08718_gb300 import replicas


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = replicas.partition(7, rank, world)
        slowest = replicas.max_over_ranks(10.0 + rank)
        results = replicas.gather_results({i: 100.0 + i for i in mine}, 7)
        dist.barrier()
        out.put((rank, mine, slowest, results))
    finally:
        dist.destroy_process_group()


def test_partition_covers_every_item_once():
    for n in (0, 1, 5, 192):
        for world in (1, 2, 3, 8):
            parts = [replicas.partition(n, r, world) for r in range(world)]
            flat = sorted(i for p in parts for i in p)
            assert flat == list(range(n))
    with pytest.raises(ValueError):
        replicas.partition(4, 2, 2)


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, s0, res0), (r1, m1, s1, res1) = got
    assert m0 == [0, 2, 4, 6] and m1 == [1, 3, 5]
    assert s0 == s1 == 11.0
    assert res0 == res1 == [100.0 + i for i in range(7)]


def test_single_process_is_identity():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.gather_results({0: 1.0, 2: 3.0}, 3)[::2] == [1.0, 3.0]
