"""The multi-GPU split emulated in one process: the plan's shards reduced by
separate twofold_dot / twofold_sum calls, their partials finished by
twofold_combine, give the one-call result and the oracle's bits (z0, z1 and
flag) for every rank count, including ragged last shards, empty trailing
shards, single-shard plans and both reduction schedules; twofold_combine over
arbitrary partials is the oracle's tree and flag."""
import numpy as np
import pytest

import oracle as O
import paper_1401_6235_gb300 as T
import synth
from paper_1401_6235_gb300.dist import shard_plan
from tests.gpu_util import assert_bits, assert_flags, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as e
    e.build()


def one(t):
    return host(t)[:1]


def emulate(x, xl, y, yl, n, L, world, p):
    import torch
    parts = []
    for a, b in shard_plan(n, L, world):
        if b == a:
            continue
        sl = lambda v: None if v is None else v[a:b]
        if y is None:
            z0, z1, _ = T.twofold_sum(sl(x), sl(xl), p=p)
        else:
            z0, z1, _ = T.twofold_dot(sl(x), sl(y), sl(xl), sl(yl), p=p)
        parts.append((z0, z1))
    if not parts:
        z = torch.zeros(0, dtype=torch.float64, device="cuda")
        return T.twofold_combine(z, z, p=p)
    return T.twofold_combine(torch.cat([u for u, _ in parts]), torch.cat([v for _, v in parts]), p=p)


CASES = [
    # (kind, n, L): latency schedule (<= 2048 leaves), block schedule, ragged tails
    ("dot", 65536, 256), ("dot", 1 << 22, 256), ("dot", 1000003, 64), ("sum", 300, 256),
    ("sum", 1 << 21, 128), ("dot2", 123457, 32), ("sum2", 2 ** 20 + 77, 1000), ("dot", 0, 256),
]


@pytest.mark.parametrize("kind,n,L", CASES)
def test_sharded_equals_one_call_and_oracle(kind, n, L):
    seed = n % 9973
    if kind.startswith("dot"):
        x, y = synth.dot_uniform(n, seed=seed) if n else (np.zeros(0), np.zeros(0))
    else:
        x, y = synth.loguniform(seed, 0, n, -30.0, 30.0, True), None
    xl = synth.ulp_tails(seed, 5, x) if kind.endswith("2") else None
    yl = synth.ulp_tails(seed, 6, y) if kind == "dot2" else None
    p = T.params(leaf=L, panic_tau=2.0 ** -70)
    g = [None if v is None else dev(v) for v in (x, xl, y, yl)]
    if y is None:
        w0, w1, wf = T.twofold_sum(g[0], g[1], p=p)
    else:
        w0, w1, wf = T.twofold_dot(g[0], g[2], g[1], g[3], p=p)
    r = O.reduce(x, xl, y, yl, L=L) if n else (0.0, 0.0)
    rf = O.flags(np.array([r[0]]), np.array([r[1]]), tau=2.0 ** -70)
    for world in (1, 2, 3, 4, 8, 13):
        z0, z1, fl = emulate(*g, n, L, world, p)
        what = f"{kind} n={n} L={L} world={world}"
        assert_bits(one(z0), one(w0), what + " z0 vs one call")
        assert_bits(one(z1), one(w1), what + " z1 vs one call")
        assert_bits(one(z0), np.array([r[0]]), what + " z0 vs oracle")
        assert_bits(one(z1), np.array([r[1]]), what + " z1 vs oracle")
        assert_flags(one(fl), rf, what + " flag")
        assert_flags(one(wf), rf, what + " one-call flag")


@pytest.mark.parametrize("m", [0, 1, 2, 3, 255, 256, 257, 5000, 70001])
def test_combine_is_the_oracle_tree(m):
    rng = np.random.default_rng(m)
    z0 = synth.loguniform(m + 1, 0, m, -10.0, 10.0, True)
    z1 = z0 * 2.0 ** -60 * rng.uniform(-1, 1, m)
    if m > 3:
        z0[3] = np.inf if m % 2 else np.nan
    p = T.params(panic_mode=O.ULP, panic_ulps=2.0)
    g0, g1 = dev(z0), dev(z1)
    c0, c1, cf = T.twofold_combine(g0, g1, p=p)
    r = O.tree(np.stack([z0, z1], 1)) if m else (0.0, 0.0)
    assert_bits(one(c0), np.array([r[0]]), f"m={m} z0")
    assert_bits(one(c1), np.array([r[1]]), f"m={m} z1")
    assert_flags(one(cf), O.flags(np.array([r[0]]), np.array([r[1]]), mode=O.ULP, m=2.0), f"m={m} flag")
    assert np.array_equal(host(g0).view(np.uint64), z0.view(np.uint64)), "inputs left unchanged"


def test_sharded_entry_points_single_rank_nccl():
    """twofold_dot_sharded / twofold_sum_sharded through a real NCCL process
    group of one rank (the all-gather and the combine on the GPU): the
    one-call bits."""
    import datetime
    import os
    import socket
    import torch
    import torch.distributed as dist
    from paper_1401_6235_gb300.dist import twofold_dot_sharded, twofold_sum_sharded
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("nccl", rank=0, world_size=1, timeout=datetime.timedelta(seconds=60),
                            device_id=torch.device("cuda", torch.cuda.current_device()))
    try:
        n = 1000003
        x, y = synth.dot_uniform(n, seed=5)
        gx, gy = dev(x), dev(y)
        z0, z1, fl = twofold_dot_sharded(gx, gy, n, 0, 1)
        w0, w1, wf = T.twofold_dot(gx, gy)
        for a, b in ((z0, w0), (z1, w1), (fl, wf)):
            assert np.array_equal(host(a).view(np.uint8), host(b).view(np.uint8))
        s0, s1, _ = twofold_sum_sharded(gx, n, 0, 1)
        r = O.reduce(x, L=256)
        assert_bits(one(s0), np.array([r[0]]), "sum z0")
        assert_bits(one(s1), np.array([r[1]]), "sum z1")
    finally:
        dist.destroy_process_group()
