"""The sharded reduction (one rank per GPU): the plan's shards are aligned
2^k-leaf subtrees of the blocked pairwise order, so the tree over the shard
results in rank order is the one-process result, bit for bit.  Checked on the
oracle without processes for many sizes and rank counts, and through a real
all-gather with world_size 2 and 3 gloo ranks on the CPU (the combine step and
the benchmark's max-over-ranks timing)."""
import socket

import numpy as np
import pytest

import oracle as O
import synth
from paper_1401_6235_gb300.dist import shard_plan, shards_in_use


def bits(z):
    return np.array(z, np.float64).view(np.uint64)


@pytest.mark.parametrize("world", [1, 2, 3, 4, 5, 7, 8])
def test_plan_tiles_aligned_power_of_two_blocks(world):
    for L in (1, 7, 256):
        for n in list(range(0, 40)) + [255, 256, 257, 4096, 10 ** 5 + 3]:
            plan = shard_plan(n, L, world)
            assert len(plan) == world
            k = shards_in_use(n, L, world)
            assert all(b > a for a, b in plan[:k]) and all(a == b for a, b in plan[k:])
            ends = [0] + [b for _, b in plan[:k]]
            assert all(plan[i][0] == ends[i] for i in range(k)) and ends[-1] == n
            if k:
                B = (plan[0][1] - plan[0][0]) // L if k > 1 else None
                m = (n + L - 1) // L
                for i, (a, b) in enumerate(plan[:k]):
                    assert a % L == 0
                    if i < k - 1:
                        assert (b - a) == B * L and B & (B - 1) == 0
                assert k <= world and (k == 1 or B * (k - 1) < m <= B * k)


@pytest.mark.parametrize("world", [2, 3, 4, 6, 8])
def test_tree_over_shards_equals_whole(world):
    rng = np.random.default_rng(world)
    for trial in range(12):
        L = int(rng.choice([1, 3, 32, 256]))
        n = int(rng.integers(0, 60 * L + 50))
        x = synth.loguniform(100 * world + trial, 0, n, -30.0, 30.0, True)
        y = synth.loguniform(100 * world + trial, 1, n, -30.0, 30.0, True) if trial % 2 else None
        xl = synth.ulp_tails(100 * world + trial, 2, x) if trial % 3 == 0 else None
        parts = [O.reduce(x[a:b], None if xl is None else xl[a:b], None if y is None else y[a:b], L=L)
                 for a, b in shard_plan(n, L, world) if b > a]
        whole = O.reduce(x, xl, y, L=L)
        assert np.array_equal(bits(O.tree(parts)), bits(whole)), (world, L, n)


def test_unaligned_split_changes_the_bits():
    """Six leaves split 3 + 3 (even, but not on a 2^k-leaf boundary) give a
    different tree and, on data of wide range and mixed signs, other bits;
    the plan's split (4 + 2) gives the one-process bits."""
    L = 16
    differs = 0
    for seed in range(20):
        x = synth.loguniform(seed, 0, 6 * L, -40.0, 40.0, True)
        parts = [O.reduce(x[a:b], L=L) for a, b in [(0, 3 * L), (3 * L, 6 * L)]]
        differs += not np.array_equal(bits(O.tree(parts)), bits(O.reduce(x, L=L)))
        assert shard_plan(6 * L, L, 2) == [(0, 4 * L), (4 * L, 6 * L)]
        aligned = [O.reduce(x[a:b], L=L) for a, b in shard_plan(6 * L, L, 2)]
        assert np.array_equal(bits(O.tree(aligned)), bits(O.reduce(x, L=L)))
    assert differs > 0


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_reduce_sharded(world, tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    from tests import dist_worker
    O.lib()
    synth.lib()
    mp.spawn(dist_worker.run, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [np.load(tmp_path / f"rank{r}.npy") for r in range(world)]
    for r in res[1:]:
        assert np.array_equal(r.view(np.uint64), res[0].view(np.uint64))


def test_input_slices_regenerate_on_their_own():
    """A rank builds only its shard: the generator's slice [a, b) equals the
    same elements of the whole stream."""
    full = synth.uniform(7, 1, 10007, -1.0, 1.0)
    for a, b in [(0, 10007), (256, 4096), (9999, 10007), (5, 5)]:
        assert np.array_equal(synth.uniform_slice(7, 1, a, b, -1.0, 1.0), full[a:b])
