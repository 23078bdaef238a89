"""Host-side logic of the multi-rank batch path on CPU: the size-balanced split
and the gather of per-problem results across two gloo ranks."""
import os

import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1408_6299_gb300.shard import gather_reports, partition


def test_partition_covers_and_balances():
    costs = [64 ** 2] * 146 + [128 ** 2 * 2] * 73 + [256 ** 2 * 4] * 37
    for world in (1, 2, 4, 8):
        parts = partition(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs)


def _worker(rank, world, port, costs, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = partition(costs, world)[rank]
    local = {i: {"rank": rank, "result": costs[i] * 2} for i in mine}
    merged = gather_reports(local, world, rank)
    if rank == 0:
        q.put(merged)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gather_with_gloo():
    costs = [5, 3, 8, 1, 9, 2, 7]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert sorted(merged) == list(range(len(costs)))
    assert all(merged[i]["result"] == 2 * costs[i] for i in merged)
    assert {merged[i]["rank"] for i in merged} == {0, 1}
