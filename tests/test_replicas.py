"""Multi-process host logic of replica runs (CPU, gloo, world size 2): the
timing reduction, per-rank seeds and the cost-balanced batch partition."""
import os

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import rte_synth
from paper_1802_03061_gb300 import replicas


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r "took" 10 (r + 1) ms for 3 (r + 1) units
        t, u, v = replicas.aggregate(10.0 * (rank + 1), 3 * (rank + 1))
        seeds = [replicas.rank_seed(2, rank, i) for i in range(4)]
        inst = rte_synth.batch_instances(count=24, seed=4)
        mine = replicas.shard(inst, world, rank)
        dist.barrier()
        q.put((rank, t, u, v, seeds, mine))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregate_seeds_and_shard():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, t, u, v, seeds, mine in res:
        assert t == 20.0            # slowest rank
        assert u == 9.0             # 3 + 6 units in total
        assert v == pytest.approx(9.0 / 0.020)
    s0, s1 = res[0][4], res[1][4]
    assert not set(s0) & set(s1)   # distinct sources per rank
    m0, m1 = res[0][5], res[1][5]
    assert sorted(m0 + m1) == list(range(24)) and not set(m0) & set(m1)


def test_shard_balances_cost_and_is_deterministic():
    inst = rte_synth.batch_instances(count=64, seed=4)
    parts = [replicas.shard(inst, 4, r) for r in range(4)]
    assert sorted(sum(parts, [])) == list(range(64))
    loads = [sum(replicas.instance_cost(inst[i]) for i in p) for p in parts]
    # greedy LPT: no rank exceeds the mean by more than the largest single item
    assert max(loads) - sum(loads) / 4 <= max(replicas.instance_cost(d) for d in inst)
    assert parts == [replicas.shard(inst, 4, r) for r in range(4)]


def test_single_process_aggregate():
    assert replicas.aggregate(50.0, 10) == (50.0, 10.0, 200.0)
    with pytest.raises(ValueError):
        replicas.shard([], 2, 2)
