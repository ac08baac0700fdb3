"""Host logic of multi-GPU runs (one process per GPU).

A single solve does not shard (its FFTs would need a distributed transpose and
one grid fits a GPU many times over), so several GPUs run replicas: each rank
solves its own problems and the ranks only agree on timing at the end.  A
batch of independent instances is partitioned across ranks by estimated cost.
No collective touches the data path; the only collectives are the barrier
around the timed region and the max/sum reductions of the timing result.
"""
import math

import torch.distributed as dist


def rank_seed(base, rank, step):
    """Seed of the source solved by `rank` at `step`: distinct across ranks."""
    return int(base) + 1000 * int(rank) + int(step)


def instance_cost(inst):
    """Relative cost of one batch instance: unknowns (2L+1) n^2 times the
    FFT length factor log2(Q) times the expected iteration count, which grows
    like log(1/tol) / -log(mu_s/mu_t) (the contraction rate of K)."""
    n = int(inst["n"])
    L = len(inst["sigma_hat"]) - 1
    rho = min(max(float(inst["mu_s"]) / float(inst["mu_t"]), 1e-3), 0.999)
    return (2 * L + 1) * n * n * math.log2(2 * n) / -math.log(rho)


def shard(instances, world, rank):
    """Indices of the instances rank `rank` of `world` solves: greedy longest-
    processing-time partition by `instance_cost` (deterministic: ties go to the
    lower rank and to the lower index), every instance on exactly one rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    order = sorted(range(len(instances)), key=lambda i: (-instance_cost(instances[i]), i))
    load = [0.0] * world
    mine = []
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += instance_cost(instances[i])
        if r == rank:
            mine.append(i)
    return sorted(mine)


def aggregate(local_ms, local_units, group=None):
    """Whole-job result over ranks: the slowest rank's time and the units all
    ranks processed; value = units / time (units per second).  Without an
    initialised process group this is the single-process result."""
    if dist.is_available() and dist.is_initialized():
        import torch

        dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
        t = torch.tensor([float(local_ms)], dtype=torch.float64, device=dev)
        u = torch.tensor([float(local_units)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
        dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
        t_max, units = float(t.item()), float(u.item())
    else:
        t_max, units = float(local_ms), float(local_units)
    return t_max, units, units / (t_max / 1e3) if t_max > 0 else 0.0
