"""GPU parity of the binary32 sum and dot (C ABI twofold_sum_f32 /
twofold_dot_f32 and their plain twins) with the binary32 oracle: bit-exact
z0, z1 and flags for every operand kind, leaf sizes, sizes spanning several
blocks with ragged tails and the empty input; and the float rows of the
paper's test100h log reproduced on the GPU (the sequential counter is one
leaf of the full length)."""
import numpy as np
import pytest

import oracle as O
import paper_1401_6235_gb300 as T
import synth
from tests.fp import split32
from tests.gpu_util import assert_flags, dev, host
from tests.test_gpu_ew_f32 import assert_bits32
from tests.test_oracle_applications import g6, golden

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as e
    e.build()


def data32(n, seed):
    x, y = synth.dot_uniform(n, seed=seed)
    x = (x * 2.0 ** synth.uniform(seed, 7, n, -10, 10).round()).astype(np.float32)
    y = y.astype(np.float32)
    return x, y


def tails32(x, seed):
    rng = np.random.default_rng(seed)
    return (x.astype(np.float64) * 2.0 ** -30 * rng.uniform(-1, 1, x.size)).astype(np.float32)


SIZES = [0, 1, 2, 255, 256, 257, 65536, 65537, 1000003]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("kinds", ["dd", "tt", "td", "dt"])
def test_dot32_kinds_sizes(n, kinds):
    x, y = data32(n, n + 3)
    xl = tails32(x, 1) if kinds[0] == "t" else None
    yl = tails32(y, 2) if kinds[1] == "t" else None
    p = T.params(panic_tau=2.0 ** -18)
    r0, r1 = O.reduce32(x, xl, y, yl)
    z0, z1, fl = T.twofold_dot_f32(dev(x), dev(y), None if xl is None else dev(xl),
                                   None if yl is None else dev(yl), p=p)
    assert_bits32(z0, np.float32([r0]), "z0")
    assert_bits32(z1, np.float32([r1]), "z1")
    assert_flags(fl, [O.flag32(r0, r1, tau=2.0 ** -18)], "flag")
    if kinds == "dd":
        assert_bits32(T.plain_dot_f32(dev(x), dev(y)), np.float32([O.reduce32_plain(x, y)]), "plain")


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("dotted", [True, False])
def test_sum32_sizes(n, dotted):
    x, _ = data32(n, n + 11)
    xl = None if dotted else tails32(x, 3)
    r0, r1 = O.reduce32(x, xl)
    z0, z1, fl = T.twofold_sum_f32(dev(x), None if xl is None else dev(xl))
    assert_bits32(z0, np.float32([r0]), "z0")
    assert_bits32(z1, np.float32([r1]), "z1")
    assert_flags(fl, [O.flag32(r0, r1)], "flag (binary32 default tau 2^-18)")
    if dotted:
        assert_bits32(T.plain_sum_f32(dev(x)), np.float32([O.reduce32_plain(x)]), "plain")


@pytest.mark.parametrize("L", [1, 3, 64, 1000, 1 << 20])
def test_reduce32_leaf_sizes(L):
    n = 300007
    x, y = data32(n, L)
    p = T.params(leaf=L, panic_mode=T.PANIC_ULP, panic_ulps=2.0)
    for dot in (False, True):
        r0, r1 = O.reduce32(x, None, y if dot else None, None, L=L)
        if dot:
            z0, z1, fl = T.twofold_dot_f32(dev(x), dev(y), p=p)
        else:
            z0, z1, fl = T.twofold_sum_f32(dev(x), p=p)
        assert_bits32(z0, np.float32([r0]), f"L={L} dot={dot} z0")
        assert_bits32(z1, np.float32([r1]), f"L={L} dot={dot} z1")
        assert_flags(fl, [O.flag32(r0, r1, mode=O.ULP, m=2.0)], f"L={L} dot={dot} flag")


@pytest.mark.parametrize("h", [100, 1000])
def test_test100h_float_logs_on_gpu(h):
    """The paper's float test100h: 10 ticks of 0.1[-1.49012e-09] per second
    for h hours summed sequentially (one leaf), then DTF 1.1 by 3600; the
    printed 96.3958[3.54008] and 582.542[461.249]."""
    n = h * 3600 * 10
    t0, t1 = split32(0.1)
    x0 = np.full(n, t0, np.float32)
    x1 = np.full(n, t1, np.float32)
    s0, s1, _ = T.twofold_sum_f32(dev(x0), dev(x1), p=T.params(leaf=n, panic_tau=2.0 ** -18))
    r = O.reduce32(x0, x1, L=n)
    assert_bits32(s0, np.float32([r[0]]), "sum z0")
    assert_bits32(s1, np.float32([r[1]]), "sum z1")
    import torch
    three600 = torch.full((1,), 3600.0, dtype=torch.float32, device="cuda")
    z0, z1, _ = T.twofold_ew_f32([(T.DIV, 2, 0, 1)], [(s0, s1), (three600, None)])
    assert (g6(float(host(z0)[0])), g6(float(host(z1)[0]))) == golden()[("test100h_f32", str(h))]


def test_dot32_large_both_tails_exact_workspace():
    """2^26 + 3 elements with tails on both operands (the largest staged
    tile, so fewer leaves per block) in a workspace of exactly the queried
    size: the oracle's bits."""
    import torch
    n = (1 << 26) + 3
    x, y = data32(n, 77)
    xl, yl = tails32(x, 78), tails32(y, 79)
    nb = T.lib().twofold_workspace_bytes(T.KIND_DOT, n, 1, None)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    z0, z1, fl = T.twofold_dot_f32(dev(x), dev(y), dev(xl), dev(yl), ws=ws)
    r0, r1 = O.reduce32(x, xl, y, yl)
    assert_bits32(z0, np.float32([r0]), "z0")
    assert_bits32(z1, np.float32([r1]), "z1")
    assert_flags(fl, [O.flag32(r0, r1)], "flag")


def test_dot32_small_workspace_takes_larger_blocks():
    """2^26 dotted elements (2^18 leaves) in a workspace that holds the
    partials of 256-leaf blocks but not of the preferred 128-leaf blocks:
    the call takes the larger blocks, with the oracle's bits; a workspace
    too small for those too is refused."""
    import torch
    n = 1 << 26
    x, y = data32(n, 91)
    ws = torch.empty(2 * 4096, dtype=torch.uint8, device="cuda")    # two arrays of 1024 floats
    z0, z1, fl = T.twofold_dot_f32(dev(x), dev(y), ws=ws)
    r0, r1 = O.reduce32(x, None, y, None)
    assert_bits32(z0, np.float32([r0]), "z0")
    assert_bits32(z1, np.float32([r1]), "z1")
    assert_flags(fl, [O.flag32(r0, r1)], "flag")
    with pytest.raises(T.TwofoldError):
        T.twofold_dot_f32(dev(x), dev(y), ws=ws[:4096])


def test_dot32_full_size_bench_configuration():
    """The binary32 dot workload at full size: 2^28 dotted elements, uniform
    [-1, 1] floats of seed 0, the benchmark's call; the whole result against
    the oracle."""
    import torch
    n = 1 << 28
    x = synth.uniform(0, 0, n, -1.0, 1.0).astype(np.float32)
    y = synth.uniform(0, 1, n, -1.0, 1.0).astype(np.float32)
    z0, z1, fl = T.twofold_dot_f32(dev(x), dev(y))
    r0, r1 = O.reduce32(x, None, y, None)
    assert_bits32(z0, np.float32([r0]), "z0")
    assert_bits32(z1, np.float32([r1]), "z1")
    assert_flags(fl, [O.flag32(r0, r1)], "flag")
    assert_bits32(T.plain_dot_f32(dev(x), dev(y)), np.float32([O.reduce32_plain(x, y)]), "plain")
    torch.cuda.empty_cache()


@pytest.mark.parametrize("shift", [0, 1, 2, 4])
def test_dot32_alignment_paths(shift):
    """Arrays starting 4, 8 or 16 bytes into an allocation (the 4-byte copy
    path when a leaf start is not 16-byte aligned, the 16-byte path
    otherwise) with a ragged end: the same bits either way."""
    n = 200003
    x, y = data32(n + shift, 91)
    xl, yl = tails32(x, 92), tails32(y, 93)
    g = [dev(v)[shift:] for v in (x, y, xl, yl)]
    r0, r1 = O.reduce32(x[shift:], xl[shift:], y[shift:], yl[shift:])
    z0, z1, _ = T.twofold_dot_f32(g[0], g[1], g[2], g[3])
    assert_bits32(z0, np.float32([r0]), f"shift {shift} z0")
    assert_bits32(z1, np.float32([r1]), f"shift {shift} z1")
    d0, d1 = O.reduce32(x[shift:], None, y[shift:], None, L=100)
    w0, w1, _ = T.twofold_dot_f32(g[0], g[1], p=T.params(leaf=100, panic_tau=2.0 ** -18))
    assert_bits32(w0, np.float32([d0]), f"shift {shift} L=100 z0")
    assert_bits32(w1, np.float32([d1]), f"shift {shift} L=100 z1")
