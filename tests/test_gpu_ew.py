"""GPU parity of twofold_ew / plain_ew (through the C ABI) with the oracle:
bit-exact z0, z1 and flags on every op and operand kind, on edge values, on
random programs, on the elementwise chain z = sqrt((a*b + c)/d) at several
tile-spanning sizes with ragged tails, and at the full 2^28 size on sampled
outputs."""
import itertools

import numpy as np
import pytest

import oracle as O
import paper_1401_6235_gb300 as T
import synth
from tests.fp import rand_doubles, rand_tails
from tests.gpu_util import SPECIAL, assert_bits, assert_flags, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as e
    e.build()


def edge_operands():
    """All pairs of special heads, each with a few tails."""
    tails = np.array([0.0, -0.0, 1e-17, -3e-300, 2.0 ** -1074, np.inf, np.nan, 0.25])
    rng = np.random.default_rng(0)
    x0, y0 = [a.ravel() for a in np.meshgrid(SPECIAL, SPECIAL)]
    reps = 4
    x0 = np.tile(x0, reps)
    y0 = np.tile(y0, reps)
    x1 = tails[rng.integers(0, tails.size, x0.size)]
    y1 = tails[rng.integers(0, tails.size, y0.size)]
    x1[: SPECIAL.size ** 2] = 0.0
    y1[: SPECIAL.size ** 2] = 0.0
    return x0, x1, y0, y1


def random_operands(n=200003, seed=1):
    rng = np.random.default_rng(seed)
    x0 = rand_doubles(rng, n, -80, 80)
    y0 = rand_doubles(rng, n, -80, 80)
    return x0, rand_tails(rng, x0, 0, 70), y0, rand_tails(rng, y0, 0, 70)


@pytest.mark.parametrize("op", [O.ADD, O.SUB, O.MUL, O.DIV, O.SQRT])
@pytest.mark.parametrize("xd,yd", list(itertools.product([False, True], repeat=2)))
@pytest.mark.parametrize("data", ["edge", "random"])
def test_single_op_kinds(op, xd, yd, data):
    x0, x1, y0, y1 = edge_operands() if data == "edge" else random_operands()
    prog = [(op, 2, 0, 1)]
    ins = [(x0, None if xd else x1), (y0, None if yd else y1)]
    r0, r1, rf = O.ew(prog, ins)
    g = [(dev(h), None if lo is None else dev(lo)) for h, lo in ins]
    z0, z1, fl = T.twofold_ew(prog, g)
    assert_bits(z0, r0, "z0")
    assert_bits(z1, r1, "z1")
    assert_flags(fl, rf, "flags")
    pz = T.plain_ew(prog, [g[0][0], g[1][0]])
    assert_bits(pz, O.ew_plain(prog, [x0, y0]), "plain")
    assert_bits(pz, r0, "plain == z0")


@pytest.mark.parametrize("n", [1, 31, 128, 129, 4097, 100003, (1 << 20) + 13])
def test_chain_config_sizes(n):
    d = synth.ew_chain(n, seed=n)
    ins = [(d["a0"], d["a1"]), (d["b0"], d["b1"]), (d["c0"], d["c1"]), (d["d0"], d["d1"])]
    r0, r1, rf = O.ew(T.CHAIN_SQRT_MAD_DIV, ins)
    g = [(dev(h), dev(lo)) for h, lo in ins]
    z0, z1, fl = T.twofold_ew(T.CHAIN_SQRT_MAD_DIV, g)
    assert_bits(z0, r0, "z0")
    assert_bits(z1, r1, "z1")
    assert_flags(fl, rf, "flags")
    pz = T.plain_ew(T.CHAIN_SQRT_MAD_DIV, [h for h, _ in g])
    assert_bits(pz, r0, "plain twin == z0")


def test_chain_kernel_equals_interpreter():
    """The chain-form program runs in the register-resident chain kernel; the
    same computation with a dead first instruction is not chain-shaped and
    runs in the shared-memory interpreter: identical bits."""
    n = 100003
    d = synth.ew_chain(n, seed=21)
    g = [(dev(d[k + "0"]), dev(d[k + "1"])) for k in "abcd"]
    a = T.twofold_ew(T.CHAIN_SQRT_MAD_DIV, g)
    prog = [(O.ADD, 8, 0, 0)] + list(T.CHAIN_SQRT_MAD_DIV)
    b = T.twofold_ew(prog, g)
    for u, v in zip(a, b):
        assert np.array_equal(host(u).view(np.uint8), host(v).view(np.uint8))


def test_host_buffer_form_equals_device_buffers():
    """Pinned host tensors that the device maps stand in for device buffers
    (the kernels read and write them across the host link): the same bits
    as device buffers and as the oracle; an unpinned host tensor is refused."""
    import torch
    n = 100003
    d = synth.ew_chain(n, seed=5)
    ins = [(d[k + "0"], d[k + "1"]) for k in "abcd"]
    pin = lambda a: torch.from_numpy(a).pin_memory()
    hins = [(pin(h), pin(lo)) for h, lo in ins]
    assert T.lib().twofold_host_mapped(T.ctypes.c_void_p(hins[0][0].data_ptr())) == 1
    dz = T.twofold_ew(T.CHAIN_SQRT_MAD_DIV, [(dev(h), dev(lo)) for h, lo in ins])
    hz = T.twofold_ew(T.CHAIN_SQRT_MAD_DIV, hins)
    torch.cuda.synchronize()
    assert all(not t.is_cuda and t.is_pinned() for t in hz)
    for u, v in zip(dz, hz):
        assert np.array_equal(host(u).view(np.uint8), v.numpy().view(np.uint8))
    r0, r1, rf = O.ew(T.CHAIN_SQRT_MAD_DIV, ins)
    assert_bits(hz[0].numpy(), r0, "host z0")
    assert_bits(hz[1].numpy(), r1, "host z1")
    pz = T.plain_ew(T.CHAIN_SQRT_MAD_DIV, [h for h, _ in hins])
    torch.cuda.synchronize()
    assert_bits(pz.numpy(), r0, "host plain == z0")
    with pytest.raises(ValueError):
        T.twofold_ew(T.CHAIN_SQRT_MAD_DIV, [(torch.from_numpy(h), None) for h, _ in ins])


def coupled_operands(n=100003, seed=5):
    """Non-overlapping ("coupled") operands: |tail| <= ulp(head)/2."""
    rng = np.random.default_rng(seed)
    x0 = rand_doubles(rng, n, -80, 80)
    y0 = rand_doubles(rng, n, -80, 80)
    ux = np.ldexp(1.0, np.frexp(np.abs(x0))[1] - 53)
    uy = np.ldexp(1.0, np.frexp(np.abs(y0))[1] - 53)
    return x0, ux / 2 * rng.uniform(-1, 1, n), y0, uy / 2 * rng.uniform(-1, 1, n)


@pytest.mark.parametrize("op", [O.PADD, O.PSUB, O.PMUL, O.PDIV, O.PSQRT])
@pytest.mark.parametrize("xd,yd", list(itertools.product([False, True], repeat=2)))
@pytest.mark.parametrize("data", ["edge", "random", "coupled"])
def test_coupled_op_kinds(op, xd, yd, data):
    """Coupled (Dekker emulation) operations, every operand kind, special
    values, general twofolds and non-overlapping ones: bit-exact."""
    x0, x1, y0, y1 = {"edge": edge_operands, "random": random_operands, "coupled": coupled_operands}[data]()
    prog = [(op, 2, 0, 1 if op != O.PSQRT else 0)]
    ins = [(x0, None if xd else x1), (y0, None if yd else y1)]
    r0, r1, rf = O.ew(prog, ins)
    g = [(dev(h), None if lo is None else dev(lo)) for h, lo in ins]
    z0, z1, fl = T.twofold_ew(prog, g)
    assert_bits(z0, r0, "z0")
    assert_bits(z1, r1, "z1")
    assert_flags(fl, rf, "flags")


def test_coupled_chain_and_mixed_programs():
    """A chain of coupled ops (chain kernel) and random programs mixing
    twofold and coupled ops (interpreter): bit-exact; the plain twin of a
    coupled op is its basic op."""
    n = 50021
    d = synth.ew_chain(n, seed=13)
    ins = [(d[k + "0"], d[k + "1"]) for k in "abcd"]
    pchain = [(O.PMUL, 4, 0, 1), (O.PADD, 5, 4, 2), (O.PDIV, 6, 5, 3), (O.PSQRT, 7, 6, 6)]
    r0, r1, rf = O.ew(pchain, ins)
    g = [(dev(h), dev(lo)) for h, lo in ins]
    z0, z1, fl = T.twofold_ew(pchain, g)
    assert_bits(z0, r0, "p-chain z0")
    assert_bits(z1, r1, "p-chain z1")
    assert_flags(fl, rf, "p-chain flags")
    assert_bits(T.plain_ew(pchain, [h for h, _ in g]), O.ew_plain(T.CHAIN_SQRT_MAD_DIV, [h for h, _ in ins]),
                "plain twin")
    rng = np.random.default_rng(17)
    m = 20011
    for trial in range(8):
        nin = int(rng.integers(1, 5))
        ins_np = []
        for k in range(nin):
            h = np.abs(rand_doubles(rng, m, -6, 6))
            lo = None if rng.random() < 0.3 else rand_tails(rng, h, 40, 60)
            ins_np.append((h, lo))
        prog, defined = [], list(range(nin))
        for s_ in range(int(rng.integers(1, 9))):
            op = int(rng.integers(1, 11))
            a, b = int(rng.choice(defined)), int(rng.choice(defined))
            prog.append((op, nin + s_, a, a if op in (O.SQRT, O.PSQRT) else b))
            defined.append(nin + s_)
        r0, r1, rf = O.ew(prog, ins_np)
        gg = [(dev(h), None if lo is None else dev(lo)) for h, lo in ins_np]
        z0, z1, fl = T.twofold_ew(prog, gg)
        assert_bits(z0, r0, f"trial {trial} z0")
        assert_bits(z1, r1, f"trial {trial} z1")
        assert_flags(fl, rf, f"trial {trial} flags")


@pytest.mark.parametrize("mode", [T.PANIC_REL, T.PANIC_ULP])
def test_chain_flag_modes(mode):
    n = 50001
    d = synth.ew_chain(n, seed=3)
    ins = [(d["a0"], d["a1"]), (d["b0"], d["b1"]), (d["c0"], d["c1"]), (d["d0"], d["d1"])]
    tau, m = 2.0 ** -52, 3.0
    p = T.params(panic_mode=mode, panic_tau=tau, panic_ulps=m)
    r0, r1, rf = O.ew(T.CHAIN_SQRT_MAD_DIV, ins, mode=mode, tau=tau, m=m)
    z0, z1, fl = T.twofold_ew(T.CHAIN_SQRT_MAD_DIV, [(dev(h), dev(lo)) for h, lo in ins], p=p)
    assert_flags(fl, rf, "flags")
    assert 0 < np.mean(rf & 1) < 1


def test_random_programs():
    rng = np.random.default_rng(11)
    n = 30011
    for trial in range(12):
        nin = int(rng.integers(1, 6))
        ins_np = []
        for k in range(nin):
            h = rand_doubles(rng, n, -6, 6)
            if k % 2 == 0:
                h = np.abs(h)
            lo = None if rng.random() < 0.4 else rand_tails(rng, h, 20, 60)
            ins_np.append((h, lo))
        prog, defined = [], list(range(nin))
        nsteps = int(rng.integers(1, 10))
        for s in range(nsteps):
            op = int(rng.integers(1, 6))
            dst = nin + s
            a, b = int(rng.choice(defined)), int(rng.choice(defined))
            prog.append((op, dst, a, b if op != O.SQRT else a))
            defined.append(dst)
        r0, r1, rf = O.ew(prog, ins_np)
        g = [(dev(h), None if lo is None else dev(lo)) for h, lo in ins_np]
        z0, z1, fl = T.twofold_ew(prog, g)
        assert_bits(z0, r0, f"trial {trial} z0")
        assert_bits(z1, r1, f"trial {trial} z1")
        assert_flags(fl, rf, f"trial {trial} flags")
        assert_bits(T.plain_ew(prog, [h for h, _ in g]), r0, f"trial {trial} plain")


def test_deterministic_and_empty():
    d = synth.ew_chain(70001, seed=9)
    g = [(dev(d[k + "0"]), dev(d[k + "1"])) for k in "abcd"]
    a = [host(t) for t in T.twofold_ew(T.CHAIN_SQRT_MAD_DIV, g)]
    b = [host(t) for t in T.twofold_ew(T.CHAIN_SQRT_MAD_DIV, g)]
    for u, v in zip(a, b):
        assert np.array_equal(u.view(np.uint8), v.view(np.uint8))
    import torch
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    z0, z1, fl = T.twofold_ew(T.CHAIN_SQRT_MAD_DIV, [(e, e)] * 4)
    assert z0.numel() == 0


def test_chain_full_size_sampled():
    """The full workload (n = 2^28) in the launch configuration the benchmark
    times, checked on 2^20 sampled elements against the oracle."""
    import torch
    n = 1 << 28
    d = synth.ew_chain(n, seed=0)
    g = {k: dev(v) for k, v in d.items()}
    ins = [(g["a0"], g["a1"]), (g["b0"], g["b1"]), (g["c0"], g["c1"]), (g["d0"], g["d1"])]
    z0, z1, fl = T.twofold_ew(T.CHAIN_SQRT_MAD_DIV, ins)
    pz = T.plain_ew(T.CHAIN_SQRT_MAD_DIV, [h for h, _ in ins])
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(0).choice(n, 1 << 20, replace=False))
    idx[:4] = [0, 1, n - 2, n - 1]
    idx = np.unique(idx)
    sub = [(d[k + "0"][idx], d[k + "1"][idx]) for k in "abcd"]
    r0, r1, rf = O.ew(T.CHAIN_SQRT_MAD_DIV, sub)
    ti = torch.from_numpy(idx).to("cuda")
    assert_bits(z0[ti], r0, "z0")
    assert_bits(z1[ti], r1, "z1")
    assert_flags(fl[ti], rf, "flags")
    assert_bits(pz[ti], r0, "plain twin")
    del g, ins, z0, z1, fl, pz
    torch.cuda.empty_cache()


def test_program_beyond_2_31_elements_sampled():
    """A two-input program over 2^31 + 3 twofolds (the largest index past 32
    bits), checked on sampled elements including both ends."""
    import torch
    n = (1 << 31) + 3
    a = synth.uniform(21, 0, n, 1.0, 2.0)
    b = synth.uniform(21, 1, n, 1.0, 2.0)
    ga, gb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    prog = [(O.MUL, 2, 0, 1), (O.DIV, 3, 2, 0)]
    z0, z1, fl = T.twofold_ew(prog, [(ga, None), (gb, None)])
    torch.cuda.synchronize()
    idx = np.unique(np.concatenate([[0, 1, (1 << 31) - 1, 1 << 31, n - 2, n - 1],
                                    np.random.default_rng(3).integers(0, n, 1 << 16)]))
    r0, r1, rf = O.ew(prog, [(a[idx], None), (b[idx], None)])
    ti = torch.from_numpy(idx).cuda()
    assert_bits(z0[ti], r0, "z0")
    assert_bits(z1[ti], r1, "z1")
    assert_flags(fl[ti], rf, "flags")
    del ga, gb, z0, z1, fl
    torch.cuda.empty_cache()
