"""GPU parity of the sum and dot entry points (C ABI) with the oracle: bit-
exact z0, z1 and flags for every operand kind, leaf sizes, sizes that span
several blocks with ragged tails, empty input, uneven and empty batched
jobs, the n = 65536 dot and the 4096 x 2^16 ill-conditioned batch in full."""
import numpy as np
import pytest

import oracle as O
import paper_1401_6235_gb300 as T
import synth
from tests.fp import rand_tails
from tests.gpu_util import assert_bits, assert_flags, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as e
    e.build()


def tails(x, seed):
    return rand_tails(np.random.default_rng(seed), x, 30, 60)


SIZES = [0, 1, 2, 255, 256, 257, 65536, 65537, 1000003]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("kinds", ["dd", "tt", "td", "dt"])
def test_dot_kinds_sizes(n, kinds):
    x, y = synth.dot_uniform(n, seed=n + 1)
    xl = tails(x, 1) if kinds[0] == "t" else None
    yl = tails(y, 2) if kinds[1] == "t" else None
    e0, e1 = O.reduce(x, xl, y, yl, L=256)
    z0, z1, fl = T.twofold_dot(dev(x), dev(y), None if xl is None else dev(xl),
                               None if yl is None else dev(yl))
    assert_bits(z0, [e0], "z0")
    assert_bits(z1, [e1], "z1")
    assert_flags(fl, [O.flag(e0, e1)], "flag")
    if kinds == "dd":
        assert_bits(T.plain_dot(dev(x), dev(y)), [O.reduce_plain(x, y)], "plain")


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("dotted", [True, False])
def test_sum_sizes(n, dotted):
    x, _ = synth.dot_uniform(n, seed=n + 7)
    xl = None if dotted else tails(x, 3)
    e0, e1 = O.reduce(x, xl, L=256)
    z0, z1, fl = T.twofold_sum(dev(x), None if xl is None else dev(xl))
    assert_bits(z0, [e0], "z0")
    assert_bits(z1, [e1], "z1")
    assert_flags(fl, [O.flag(e0, e1)], "flag")
    if dotted:
        assert_bits(T.plain_sum(dev(x)), [O.reduce_plain(x)], "plain")


@pytest.mark.parametrize("kinds", ["dd", "tt", "td", "dt", "s", "st"])
@pytest.mark.parametrize("shift", [(1, 1), (0, 1), (1, 0)])
def test_throughput_schedule_unaligned_leaves(kinds, shift):
    """The throughput schedule reads a leaf's elements as 16-byte pairs only
    when every array of the leaf starts on a 16-byte boundary.  Views one
    element into their allocations (8 bytes off) take the one-element walk,
    alone or mixed with aligned arrays; every kind of operand, ragged tail."""
    n = 600011
    sx, sy = shift
    x, y = synth.dot_uniform(n + 1, seed=17)
    xt, yt = tails(x, 5), tails(y, 6)
    gx, gy, gxt, gyt = dev(x), dev(y), dev(xt), dev(yt)
    vx, vy = x[sx:sx + n], y[sy:sy + n]
    use_xl = kinds in ("tt", "td", "st")
    use_yl = kinds in ("tt", "dt")
    xl = xt[sx:sx + n] if use_xl else None
    yl = yt[sy:sy + n] if use_yl else None
    dgx, dgy = gx[sx:sx + n], gy[sy:sy + n]
    dxl = gxt[sx:sx + n] if use_xl else None
    dyl = gyt[sy:sy + n] if use_yl else None
    if kinds.startswith("s"):
        e0, e1 = O.reduce(vx, xl, L=256)
        z0, z1, fl = T.twofold_sum(dgx, dxl)
    else:
        e0, e1 = O.reduce(vx, xl, vy, yl, L=256)
        z0, z1, fl = T.twofold_dot(dgx, dgy, dxl, dyl)
    assert_bits(z0, [e0], f"{kinds} {shift} z0")
    assert_bits(z1, [e1], f"{kinds} {shift} z1")
    assert_flags(fl, [O.flag(e0, e1)], f"{kinds} {shift} flag")


def test_throughput_schedule_jobs_of_both_parities():
    """Batched jobs that start on even and odd elements: within one launch
    some CTAs take the 16-byte walk and some the one-element walk."""
    x, y = synth.dot_uniform(1_500_007, seed=23)
    offs = np.array([0, 300001, 600002, 900004, 1200005, 1500007], np.int64)
    r0, r1, rf = O.dot_batched(x, None, y, None, offs)
    z0, z1, fl = T.twofold_dot_batched(dev(x), dev(y), offs)
    assert_bits(z0, r0, "z0")
    assert_bits(z1, r1, "z1")
    assert_flags(fl, rf, "flags")


@pytest.mark.parametrize("L", [1, 3, 7, 64, 1000, 1 << 20])
def test_leaf_sizes(L):
    n = 300007
    x, y = synth.dot_uniform(n, seed=L)
    p = T.params(leaf=L)
    e0, e1 = O.reduce(x, None, y, None, L=L)
    z0, z1, fl = T.twofold_dot(dev(x), dev(y), p=p)
    assert_bits(z0, [e0], f"L={L} z0")
    assert_bits(z1, [e1], f"L={L} z1")
    assert_bits(T.plain_dot(dev(x), dev(y), p=p), [O.reduce_plain(x, y, L=L)], "plain")


@pytest.mark.parametrize("L,n", [(1, 2000), (3, 5003), (33, 40000), (256, 8191), (512, 300001), (1024, 1000000),
                                 (2048, 300001)])
def test_latency_schedule_leaf_sizes(L, n):
    """Jobs of at most 2048 leaves of at most 2048 elements take the latency
    schedule (up to 32 leaves and 2048 elements per CTA, one lane per leaf, ragged last
    leaf and last block); dot with tails on one side, dotted sum, plain twins."""
    x, y = synth.dot_uniform(n, seed=L + n)
    xl = tails(x, L)
    p = T.params(leaf=L)
    e0, e1 = O.reduce(x, xl, y, None, L=L)
    z0, z1, fl = T.twofold_dot(dev(x), dev(y), dev(xl), p=p)
    assert_bits(z0, [e0], f"L={L} dot z0")
    assert_bits(z1, [e1], f"L={L} dot z1")
    assert_flags(fl, [O.flag(e0, e1)], f"L={L} dot flag")
    s0, s1 = O.reduce(x, None, L=L)
    q0, q1, _ = T.twofold_sum(dev(x), p=p)
    assert_bits(q0, [s0], f"L={L} sum z0")
    assert_bits(q1, [s1], f"L={L} sum z1")
    assert_bits(T.plain_dot(dev(x), dev(y), p=p), [O.reduce_plain(x, y, L=L)], f"L={L} plain dot")
    assert_bits(T.plain_sum(dev(x), p=p), [O.reduce_plain(x, L=L)], f"L={L} plain sum")


@pytest.mark.parametrize("n", [65536, 5000])
@pytest.mark.parametrize("kinds", ["x", "y", "xy"])
def test_latency_schedule_operand_kinds(n, kinds):
    """The latency schedule (a CTA pair per block of leaves: products and z0
    chains on one SM, product tails and z1 chains on the other) with tails
    on x, on y or on both, and a sum with tails: the oracle's bits."""
    x, y = synth.dot_uniform(n, seed=n + len(kinds))
    xl = tails(x, 256) if "x" in kinds else None
    yl = tails(y, 257) if "y" in kinds else None
    e0, e1 = O.reduce(x, xl, y, yl)
    z0, z1, fl = T.twofold_dot(dev(x), dev(y), None if xl is None else dev(xl), None if yl is None else dev(yl))
    assert_bits(z0, [e0], f"{kinds} dot z0")
    assert_bits(z1, [e1], f"{kinds} dot z1")
    assert_flags(fl, [O.flag(e0, e1)], f"{kinds} dot flag")
    if xl is not None:
        s0, s1 = O.reduce(x, xl)
        q0, q1, _ = T.twofold_sum(dev(x), dev(xl))
        assert_bits(q0, [s0], "sum z0")
        assert_bits(q1, [s1], "sum z1")


def test_latency_schedule_waits_never_ran_out():
    """In ordinary calls no CTA pair's bounded wait for its partner's chunks
    runs out."""
    before = T.wait_timeouts()
    x, y = synth.dot_uniform(65536, seed=3)
    e0, e1 = O.reduce(x, None, y, None)
    z0, z1, _ = T.twofold_dot(dev(x), dev(y))
    assert_bits(z0, [e0], "z0")
    assert_bits(z1, [e1], "z1")
    assert T.wait_timeouts() == before


@pytest.mark.parametrize("chunk", [0, 2])
def test_latency_schedule_wait_that_runs_out(chunk):
    """Failure injection on the host: the producers skip one chunk of tails,
    so each consumer's bounded wait runs out.  Every block's result is NaN
    (flag NONFINITE), the timeout count grows by the number of blocks (64
    pairs at n = 65536), and the next ordinary call is correct again (the
    context stays usable)."""
    import numpy as np
    x, y = synth.dot_uniform(65536, seed=4)
    before = T.wait_timeouts()
    prev = T.inject_pair_drop(chunk)
    try:
        z0, z1, fl = T.twofold_dot(dev(x), dev(y))
        got = (host(z0)[0], host(z1)[0], int(host(fl)[0]))
    finally:
        T.inject_pair_drop(prev)
    assert np.isnan(got[0]) and np.isnan(got[1]) and got[2] & T.NONFINITE
    assert T.wait_timeouts() - before == 64
    e0, e1 = O.reduce(x, None, y, None)
    z0, z1, fl = T.twofold_dot(dev(x), dev(y))
    assert_bits(z0, [e0], "z0 after")
    assert_bits(z1, [e1], "z1 after")


def test_config_dot_65536_zero_tails_equal_dotted():
    """n = 65536 uniform[-1,1] seed 0: tails materialised as +0 and tails
    absent give the same bits, equal to the oracle."""
    import torch
    x, y = synth.dot_uniform(65536, seed=0)
    e0, e1 = O.reduce(x, None, y, None)
    a = T.twofold_dot(dev(x), dev(y))
    z = torch.zeros(65536, dtype=torch.float64, device="cuda")
    b = T.twofold_dot(dev(x), dev(y), z, z)
    for t in (a, b):
        assert_bits(t[0], [e0], "z0")
        assert_bits(t[1], [e1], "z1")
        assert_flags(t[2], [O.flag(e0, e1)], "flag")


def test_batched_uneven_with_empty_jobs():
    rng = np.random.default_rng(5)
    lens = rng.integers(0, 200000, 70)
    lens[[0, 5, 6, 69]] = 0
    lens[10] = 1
    lens[11] = 256
    lens[12] = 1 << 20
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    n = int(offs[-1])
    x, y = synth.dot_uniform(n, seed=77)
    xl = tails(x, 9)
    r0, r1, rf = O.dot_batched(x, xl, y, None, offs)
    z0, z1, fl = T.twofold_dot_batched(dev(x), dev(y), offs, xl=dev(xl))
    assert_bits(z0, r0, "z0")
    assert_bits(z1, r1, "z1")
    assert_flags(fl, rf, "flags")
    s0, s1, sf = O.sum_batched(x, xl, offs)
    q0, q1, qf = T.twofold_sum_batched(dev(x), offs, xl=dev(xl))
    assert_bits(q0, s0, "sum z0")
    assert_bits(q1, s1, "sum z1")
    assert_flags(qf, sf, "sum flags")
    pl = np.array([O.reduce_plain(x[a:b], y[a:b]) for a, b in zip(offs[:-1], offs[1:])])
    assert_bits(T.plain_dot_batched(dev(x), dev(y), offs), pl, "plain batched")


def test_batched_offset_start_and_few_jobs():
    """Jobs need not start at 0 and small tables travel in the launch."""
    x, y = synth.dot_uniform(100000, seed=4)
    offs = np.array([1000, 1000, 1257, 99999], np.int64)
    r0, r1, rf = O.dot_batched(x, None, y, None, offs)
    z0, z1, fl = T.twofold_dot_batched(dev(x), dev(y), offs)
    assert_bits(z0, r0, "z0")
    assert_bits(z1, r1, "z1")


def test_ill_conditioned_batch_full():
    """4096 dots of 2^16 with condition 10^U(2,30): bit-exact in full; the
    panic rate grows with the realised condition number (near 0 below
    10^3.5, near 1 above 10^16, non-decreasing over two-decade bins)."""
    x, y, offs, exact, cond, _ = synth.cond_dots(4096, 1 << 16, seed=0)
    r0, r1, rf = O.dot_batched(x, None, y, None, offs)
    z0, z1, fl = T.twofold_dot_batched(dev(x), dev(y), offs)
    assert_bits(z0, r0, "z0")
    assert_bits(z1, r1, "z1")
    assert_flags(fl, rf, "flags")
    f = host(fl) & 1
    lc = np.log10(cond)
    lo, hi = f[lc < 3.5], f[lc > 16]
    assert lo.mean() < 0.05 and hi.mean() > 0.95
    # monotone over two-decade bins of the realised condition (sampling noise allowed)
    rates = [f[(lc >= b) & (lc < b + 2)].mean() for b in range(2, 30, 2) if ((lc >= b) & (lc < b + 2)).sum() >= 20]
    assert all(r2 >= r1 - 0.1 for r1, r2 in zip(rates, rates[1:])), rates
    pl = T.plain_dot_batched(dev(x), dev(y), offs)
    assert_bits(pl, r0, "plain twin == z0")


@pytest.mark.parametrize("fill", [0x00, 0xFF, "counts"])
def test_latency_schedule_any_workspace_contents(fill):
    """Whatever the workspace holds before a call (zeros, all ones, small
    integers at every word), repeated latency-schedule sums and dots on the
    same workspace give the oracle's bits, plain twin included."""
    import torch
    n = 65536 + 77
    x, y = synth.dot_uniform(n, seed=90)
    gx, gy = dev(x), dev(y)
    nb = T.lib().twofold_workspace_bytes(T.KIND_DOT, n, 1, None)
    ws = T.workspace(nb)
    e0, e1 = O.reduce(x, None, y, None)
    s0, s1 = O.reduce(x)
    for rep in range(3):
        if fill == "counts":
            ws.view(torch.int64)[:nb // 8] = torch.arange(nb // 8, device="cuda", dtype=torch.int64) % 300
        else:
            ws.fill_(fill)
        z0, z1, fl = T.twofold_dot(gx, gy, ws=ws)
        assert_bits(z0, [e0], f"rep {rep} z0")
        assert_bits(z1, [e1], f"rep {rep} z1")
        assert_flags(fl, [O.flag(e0, e1)], f"rep {rep} flag")
        u0, u1, _ = T.twofold_sum(gx, ws=ws)              # the same workspace, after the dot
        assert_bits(u0, [s0], f"rep {rep} sum z0")
        assert_bits(u1, [s1], f"rep {rep} sum z1")
        assert_bits(T.plain_dot(gx, gy, ws=ws), [O.reduce_plain(x, y)], f"rep {rep} plain")


def test_latency_schedule_graph_replays():
    """A dot captured in a CUDA graph (two launches with programmatic
    dependent launch): every replay, with new data copied into the same
    buffers, gives the oracle's bits for that data."""
    import torch
    n = 65536
    gx = torch.empty(n, dtype=torch.float64, device="cuda")
    gy = torch.empty(n, dtype=torch.float64, device="cuda")
    ws = T.workspace(T.lib().twofold_workspace_bytes(T.KIND_DOT, n, 1, None))
    out = (torch.empty(1, dtype=torch.float64, device="cuda"), torch.empty(1, dtype=torch.float64, device="cuda"),
           torch.empty(1, dtype=torch.uint8, device="cuda"))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        T.twofold_dot(gx, gy, out=out, ws=ws)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        T.twofold_dot(gx, gy, out=out, ws=ws)
    for rep in range(5):
        x, y = synth.dot_uniform(n, seed=200 + rep)
        gx.copy_(torch.from_numpy(x))
        gy.copy_(torch.from_numpy(y))
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = O.reduce(x, None, y, None)
        assert_bits(out[0], [e0], f"replay {rep} z0")
        assert_bits(out[1], [e1], f"replay {rep} z1")
        assert_flags(out[2], [O.flag(e0, e1)], f"replay {rep} flag")


@pytest.mark.parametrize("n", [1, 65536, 1000003])
def test_dot_and_sum_on_mapped_host_buffers(n):
    """Pinned host inputs and outputs that the device maps: the same bits as
    device buffers (both schedules)."""
    import torch
    x, y = synth.dot_uniform(n, seed=n + 41)
    hx, hy = torch.from_numpy(x).pin_memory(), torch.from_numpy(y).pin_memory()
    z0, z1, fl = T.twofold_dot(hx, hy)
    torch.cuda.synchronize()
    assert not z0.is_cuda
    d0, d1, df = T.twofold_dot(dev(x), dev(y))
    for a, b in ((z0, d0), (z1, d1), (fl, df)):
        assert np.array_equal(a.numpy().view(np.uint8), host(b).view(np.uint8))
    s0, s1, sf = T.twofold_sum(hx)
    torch.cuda.synchronize()
    e0, e1 = O.reduce(x, L=256)
    assert_bits(s0.numpy(), [e0], "sum z0")
    assert_bits(s1.numpy(), [e1], "sum z1")


def test_sum_beyond_2_31_elements():
    """A dotted sum of 2^31 + 3 elements (16 GiB): element and leaf indices
    past 32 bits; the whole result against the oracle."""
    import torch
    n = (1 << 31) + 3
    x = synth.uniform(17, 0, n, -1.0, 1.0)
    gx = torch.from_numpy(x).cuda()
    z0, z1, fl = T.twofold_sum(gx)
    e0, e1 = O.reduce(x, L=256)
    assert_bits(z0, [e0], "z0")
    assert_bits(z1, [e1], "z1")
    assert_flags(fl, [O.flag(e0, e1)], "flag")
    del gx
    torch.cuda.empty_cache()
