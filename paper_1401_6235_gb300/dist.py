"""Sums and dots split across ranks (one GPU per rank) in the fixed blocked
pairwise order.

The order (leaves of L elements, then a pairwise tree with the odd node
carried) makes every aligned block of 2^k leaves a subtree.  The plan gives
rank r the elements of leaves [r B, (r+1) B) with B the smallest power of two
covering ceil(leaves / ranks), so each shard is a subtree: every rank
reduces its shard with the single-GPU entry point, the (z0, z1) partials are
all-gathered, and the pairwise tree over them in rank order finishes on the
GPU (twofold_combine).  The result is the single-GPU result, bit for bit, on
every rank.  With a rank count that is not a power of two the trailing ranks
may get empty shards (the price of aligned subtrees).
"""
from __future__ import annotations

from . import _torch, tf_params, twofold_combine, twofold_dot, twofold_sum


def shard_plan(n: int, leaf: int, world: int):
    """[start, end) element range of every rank; the non-empty ranges come
    first and tile [0, n)."""
    if leaf < 1 or world < 1 or n < 0:
        raise ValueError("need leaf >= 1, world >= 1, n >= 0")
    m = (n + leaf - 1) // leaf
    if m == 0:
        return [(0, 0)] * world
    per = -(-m // world)
    B = 1 << (per - 1).bit_length()
    return [(min(n, r * B * leaf), min(n, (r + 1) * B * leaf)) for r in range(world)]


def shards_in_use(n: int, leaf: int, world: int) -> int:
    return sum(1 for a, b in shard_plan(n, leaf, world) if b > a)


def reduce_sharded(local, combine, n: int, leaf: int, rank: int, world: int, device=None, group=None):
    """One sharded reduction: `local()` gives this rank's partial (z0, z1)
    (called only for a non-empty shard); the partials of all ranks are
    all-gathered and `combine(z0s, z1s)` (1-d float64 tensors, rank order)
    runs the tree over the non-empty ones.  Returns what combine returns."""
    import torch.distributed as dist
    torch = _torch()
    a, b = shard_plan(n, leaf, world)[rank]
    if b > a:
        z0, z1 = local()
        t = torch.stack([torch.as_tensor(z0, dtype=torch.float64).reshape(()).to(device),
                         torch.as_tensor(z1, dtype=torch.float64).reshape(()).to(device)])
    else:
        t = torch.zeros(2, dtype=torch.float64, device=device)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    p = torch.stack(parts[:shards_in_use(n, leaf, world)]) if n else t.new_zeros((0, 2))
    return combine(p[:, 0].contiguous(), p[:, 1].contiguous())


def _check_shard(n_total, leaf, rank, world, *arrays):
    a, b = shard_plan(n_total, leaf, world)[rank]
    for t in arrays:
        if t is not None and t.numel() != b - a:
            raise ValueError(f"rank {rank} must hold elements [{a}, {b}) of the plan, got {t.numel()}")


def twofold_dot_sharded(x, y, n_total: int, rank: int, world: int, xl=None, yl=None,
                        p: tf_params | None = None, group=None):
    """This rank's shard of a dot of n_total elements (x, y and the optional
    tails: CUDA float64 tensors holding the plan's range for this rank);
    returns (z0, z1, flags) of the whole dot, the same on every rank."""
    leaf = p.leaf if p is not None else 256
    _check_shard(n_total, leaf, rank, world, x, y, xl, yl)
    return reduce_sharded(lambda: twofold_dot(x, y, xl, yl, p=p)[:2], lambda u, v: twofold_combine(u, v, p=p),
                          n_total, leaf, rank, world, x.device, group)


def twofold_sum_sharded(x, n_total: int, rank: int, world: int, xl=None, p: tf_params | None = None, group=None):
    """As twofold_dot_sharded, for a sum."""
    leaf = p.leaf if p is not None else 256
    _check_shard(n_total, leaf, rank, world, x, xl)
    return reduce_sharded(lambda: twofold_sum(x, xl, p=p)[:2], lambda u, v: twofold_combine(u, v, p=p),
                          n_total, leaf, rank, world, x.device, group)


def max_over_ranks(value: float, device="cpu", group=None) -> float:
    """The largest of every rank's value (a step time timed on each rank)."""
    import torch.distributed as dist
    torch = _torch()
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
