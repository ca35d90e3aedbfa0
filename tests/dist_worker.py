"""Rank body of the multi-process tests (a module of its own so that spawned
children import it by name).  Every rank builds the same seeded inputs, keeps
its shard of the plan, reduces it with the oracle and finishes with the
oracle's tree through the real all-gather, then checks the result against the
one-process reduction."""
import datetime
import os

import numpy as np


def _cases():
    # (kind, n, L, seed): ragged tails, fewer leaves than ranks, n = 0,
    # plans with empty trailing shards.
    return [("dot", 4096 * 5 + 17, 256, 1), ("dot", 1000, 64, 2), ("sum", 3 * 128, 128, 3),
            ("sum", 7, 256, 4), ("dot", 0, 256, 5), ("dot2", 33 * 32 + 5, 32, 6), ("sum2", 4 * 100, 100, 7)]


def _inputs(kind, n, seed):
    import synth
    if kind.startswith("dot"):
        x, y, _, _ = synth.cond_dot(seed, max(n, 2), 1e20)
        x, y = x[:n].copy(), y[:n].copy()
    else:
        x = synth.loguniform(seed, 0, n, -20.0, 20.0, True)
        y = None
    xl = synth.ulp_tails(seed, 5, x) if kind.endswith("2") else None
    yl = synth.ulp_tails(seed, 6, y) if kind == "dot2" else None
    return x, xl, y, yl


def run(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    import oracle as O
    from paper_1401_6235_gb300.dist import max_over_ranks, reduce_sharded, shard_plan

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=120))
    try:
        got = []
        for kind, n, L, seed in _cases():
            x, xl, y, yl = _inputs(kind, n, seed)
            a, b = shard_plan(n, L, world)[rank]
            sl = lambda v: None if v is None else v[a:b]
            local = lambda: O.reduce(sl(x), sl(xl), sl(y), sl(yl), L=L)
            combine = lambda u, v: O.tree(np.stack([u.numpy(), v.numpy()], 1))
            z = reduce_sharded(local, combine, n, L, rank, world)
            want = O.reduce(x, xl, y, yl, L=L) if n else (0.0, 0.0)
            assert np.array_equal(np.array(z).view(np.uint64), np.array(want).view(np.uint64)), \
                (kind, n, L, world, rank, z, want)
            got.append(z)
        m = max_over_ranks(1.5 * rank + 0.25)
        assert m == 1.5 * (world - 1) + 0.25, m
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.array(got))
    finally:
        dist.destroy_process_group()
