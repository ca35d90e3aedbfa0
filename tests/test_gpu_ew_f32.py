"""GPU parity of the binary32 elementwise programs (C ABI twofold_ew_f32,
plain_ew_f32) with the binary32 oracle: every operation (twofold and
coupled) and operand kind on special values and random operands, the chain
workload in float, random programs, the sticky flag in both bases, and the
host-buffer form.  Bit-exact (NaN payloads aside)."""
import itertools

import numpy as np
import pytest

import oracle as O
import paper_1401_6235_gb300 as T
import synth
from tests.gpu_util import assert_flags, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as e
    e.build()


def canon32(a):
    a = np.ascontiguousarray(a, np.float32).copy()
    v = a.view(np.uint32).copy()
    v[np.isnan(a)] = np.uint32(0x7FC00000)
    return v


def assert_bits32(got, ref, what):
    g = canon32(got if isinstance(got, np.ndarray) else host(got))
    r = canon32(ref)
    if not np.array_equal(g, r):
        bad = np.nonzero(g != r)[0]
        raise AssertionError(f"{what}: {bad.size} mismatches, first at {bad[0]}: {g[bad[0]]:#x} vs {r[bad[0]]:#x}")


SPECIAL32 = np.array([0.0, -0.0, 1.0, -1.0, 3.0, 0.1, -0.75, 1e-45, -3e-44, 1.17549435e-38, 3.4028235e38,
                      -3.4028235e38, 1e30, 1e-30, np.inf, -np.inf, np.nan, 16777216.0, 2.0 ** -24], np.float32)


def edge32():
    tails = np.array([0.0, -0.0, 1e-9, -3e-40, 1e-45, np.inf, np.nan, 0.25], np.float32)
    rng = np.random.default_rng(0)
    x0, y0 = [a.ravel() for a in np.meshgrid(SPECIAL32, SPECIAL32)]
    x0, y0 = np.tile(x0, 4), np.tile(y0, 4)
    x1 = tails[rng.integers(0, tails.size, x0.size)]
    y1 = tails[rng.integers(0, tails.size, y0.size)]
    x1[: SPECIAL32.size ** 2] = 0.0
    y1[: SPECIAL32.size ** 2] = 0.0
    return x0, x1, y0, y1


def random32(n=200003, seed=1):
    rng = np.random.default_rng(seed)
    def heads():
        return (rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-12, 12, n)).astype(np.float32)
    x0, y0 = heads(), heads()
    def tails(h):
        return (h.astype(np.float64) * 2.0 ** -rng.integers(0, 40, n) * rng.uniform(-1, 1, n)).astype(np.float32)
    return x0, tails(x0), y0, tails(y0)


def d32(a):
    return dev(np.ascontiguousarray(a, np.float32))


@pytest.mark.parametrize("op", list(range(1, 11)))
@pytest.mark.parametrize("xd,yd", list(itertools.product([False, True], repeat=2)))
@pytest.mark.parametrize("data", ["edge", "random"])
def test_single_op_kinds_f32(op, xd, yd, data):
    x0, x1, y0, y1 = edge32() if data == "edge" else random32()
    prog = [(op, 2, 0, 0 if op in (O.SQRT, O.PSQRT) else 1)]
    ins = [(x0, None if xd else x1), (y0, None if yd else y1)]
    r0, r1, rf = O.ew32(prog, ins)
    z0, z1, fl = T.twofold_ew_f32(prog, [(d32(h), None if lo is None else d32(lo)) for h, lo in ins])
    assert_bits32(z0, r0, "z0")
    assert_bits32(z1, r1, "z1")
    assert_flags(fl, rf, "flags")


def chain32(n, seed):
    d = synth.ew_chain(n, seed=seed)
    ins = []
    for k in "abcd":
        h = d[k + "0"].astype(np.float32)
        ins.append((h, (d[k + "0"] - h.astype(np.float64)).astype(np.float32)))
    return ins


@pytest.mark.parametrize("n", [1, 129, 4097, 1000003])
def test_chain_f32(n):
    ins = chain32(n, n)
    r0, r1, rf = O.ew32(T.CHAIN_SQRT_MAD_DIV, ins)
    g = [(d32(h), d32(lo)) for h, lo in ins]
    z0, z1, fl = T.twofold_ew_f32(T.CHAIN_SQRT_MAD_DIV, g)
    assert_bits32(z0, r0, "z0")
    assert_bits32(z1, r1, "z1")
    assert_flags(fl, rf, "flags")
    assert_bits32(T.plain_ew_f32(T.CHAIN_SQRT_MAD_DIV, [h for h, _ in g]), r0, "plain twin == z0")


def test_random_programs_f32():
    rng = np.random.default_rng(12)
    n = 20011
    for trial in range(10):
        nin = int(rng.integers(1, 5))
        ins = []
        for k in range(nin):
            h = np.abs(rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 3, n)).astype(np.float32)
            lo = None if rng.random() < 0.3 else (h.astype(np.float64) * 2.0 ** -30 * rng.uniform(-1, 1, n)).astype(np.float32)
            ins.append((h, lo))
        prog, defined = [], list(range(nin))
        for s in range(int(rng.integers(1, 9))):
            op = int(rng.integers(1, 11))
            a, b = int(rng.choice(defined)), int(rng.choice(defined))
            prog.append((op, nin + s, a, a if op in (O.SQRT, O.PSQRT) else b))
            defined.append(nin + s)
        mode = int(rng.choice([O.REL, O.ULP, O.REL | O.STICKY, O.ULP | O.STICKY]))
        p = T.params(panic_mode=mode, panic_tau=2.0 ** -18, panic_ulps=2.0)
        r0, r1, rf = O.ew32(prog, ins, mode=mode, tau=2.0 ** -18, m=2.0)
        z0, z1, fl = T.twofold_ew_f32(prog, [(d32(h), None if lo is None else d32(lo)) for h, lo in ins], p=p)
        assert_bits32(z0, r0, f"trial {trial} z0")
        assert_bits32(z1, r1, f"trial {trial} z1")
        assert_flags(fl, rf, f"trial {trial} flags (mode {mode})")


@pytest.mark.parametrize("mode", [T.PANIC_REL | T.PANIC_STICKY, T.PANIC_ULP | T.PANIC_STICKY])
def test_sticky_flags_binary64(mode):
    """Sticky flags of binary64 programs (chain kernel and interpreter)."""
    n = 50021
    d = synth.ew_chain(n, seed=31)
    ins = [(d[k + "0"], d[k + "1"]) for k in "abcd"]
    tau, m = 2.0 ** -50, 2.0
    p = T.params(panic_mode=mode, panic_tau=tau, panic_ulps=m)
    g = [(dev(h), dev(lo)) for h, lo in ins]
    for prog in (T.CHAIN_SQRT_MAD_DIV, [(O.ADD, 8, 0, 0)] + list(T.CHAIN_SQRT_MAD_DIV)):
        r0, r1, rf = O.ew(prog, ins, mode=mode, tau=tau, m=m)
        z0, z1, fl = T.twofold_ew(prog, g, p=p)
        assert_flags(fl, rf, "sticky flags")
        plain = O.ew(prog, ins, mode=mode & 3, tau=tau, m=m)[2]
        assert np.all((rf & 1) >= (plain & 1))        # sticky never clears a panic


def test_host_buffer_form_f32():
    import torch
    ins = chain32(100003, 7)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hz = T.twofold_ew_f32(T.CHAIN_SQRT_MAD_DIV, [(pin(h), pin(lo)) for h, lo in ins])
    torch.cuda.synchronize()
    r0, r1, rf = O.ew32(T.CHAIN_SQRT_MAD_DIV, ins)
    assert_bits32(hz[0].numpy(), r0, "host z0")
    assert_bits32(hz[1].numpy(), r1, "host z1")
    assert np.array_equal(hz[2].numpy(), rf)


def test_chain_f32_full_size_sampled():
    """The binary32 chain workload at full size (n = 2^28, the benchmark's
    launch configuration: the specialised kernel), checked on 2^20 sampled
    elements against the binary32 oracle."""
    import torch
    n = 1 << 28
    g = {k: (torch.empty(n, dtype=torch.float32, device="cuda"), torch.empty(n, dtype=torch.float32, device="cuda"))
         for k in "abcd"}
    rng = np.random.default_rng(1)
    idx = np.unique(np.concatenate([[0, 1, n - 2, n - 1], rng.choice(n, 1 << 20, replace=False)]))
    sub = {k: (np.empty(idx.size, np.float32), np.empty(idx.size, np.float32)) for k in "abcd"}
    chunk = 1 << 24
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        d = synth.ew_chain(e - s, seed=3000 + s // chunk)
        sel = (idx >= s) & (idx < e)
        for k in "abcd":
            h = d[k + "0"].astype(np.float32)
            lo = (d[k + "0"] - h.astype(np.float64)).astype(np.float32)
            g[k][0][s:e].copy_(torch.from_numpy(h))
            g[k][1][s:e].copy_(torch.from_numpy(lo))
            sub[k][0][sel] = h[idx[sel] - s]
            sub[k][1][sel] = lo[idx[sel] - s]
    z0, z1, fl = T.twofold_ew_f32(T.CHAIN_SQRT_MAD_DIV, [g[k] for k in "abcd"])
    torch.cuda.synchronize()
    r0, r1, rf = O.ew32(T.CHAIN_SQRT_MAD_DIV, [sub[k] for k in "abcd"])
    ti = torch.from_numpy(idx).to("cuda")
    assert_bits32(z0[ti], r0, "z0")
    assert_bits32(z1[ti], r1, "z1")
    assert_flags(fl[ti], rf, "flags")
    del g, z0, z1, fl
    torch.cuda.empty_cache()
