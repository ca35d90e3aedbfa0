"""The runtime-specialised elementwise kernels (twofold_ew_jit modes): with
specialisation forced at every size, random programs of every operation
(twofold and coupled), operand kind, flag mode (REL/ULP, sticky) and both
bases give the oracle's bits and the generic kernels' bits, at sizes with
ragged tails for the two-elements-per-thread layout; in automatic mode large
calls build a kernel once per program and reuse it."""
import numpy as np
import pytest

import oracle as O
import paper_1401_6235_gb300 as T
import synth
from tests.fp import rand_doubles, rand_tails
from tests.gpu_util import assert_bits, assert_flags, dev, host
from tests.test_gpu_ew_f32 import assert_bits32, d32

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def jit_mode_restored():
    import __graft_entry__ as e
    e.build()
    prev = T.jit_mode(-1)[0]
    yield
    T.jit_mode(prev)


def random_program(rng, nin):
    prog, defined = [], list(range(nin))
    for s in range(int(rng.integers(1, 8))):
        op = int(rng.integers(1, 11))
        a, b = int(rng.choice(defined)), int(rng.choice(defined))
        prog.append((op, nin + s, a, a if op in (O.SQRT, O.PSQRT) else b))
        defined.append(nin + s)
    return prog


@pytest.mark.parametrize("n", [1, 127, 128, 129, 255, 256, 257, 20011])
def test_forced_specialisation_binary64(n):
    rng = np.random.default_rng(n)
    for trial in range(3):
        nin = int(rng.integers(1, 5))
        ins = []
        for k in range(nin):
            h = np.abs(rand_doubles(rng, n, -6, 6))
            ins.append((h, None if rng.random() < 0.3 else rand_tails(rng, h, 30, 60)))
        prog = random_program(rng, nin)
        mode = int(rng.choice([O.REL, O.ULP, O.REL | O.STICKY, O.ULP | O.STICKY]))
        p = T.params(panic_mode=mode, panic_tau=2.0 ** -48, panic_ulps=3.0)
        g = [(dev(h), None if lo is None else dev(lo)) for h, lo in ins]
        T.jit_mode(0)
        generic = [host(t) for t in T.twofold_ew(prog, g, p=p)]
        T.jit_mode(2)
        z0, z1, fl = T.twofold_ew(prog, g, p=p)
        r0, r1, rf = O.ew(prog, ins, mode=mode, tau=2.0 ** -48, m=3.0)
        assert_bits(z0, r0, f"n={n} trial {trial} z0")
        assert_bits(z1, r1, f"n={n} trial {trial} z1")
        assert_flags(fl, rf, f"n={n} trial {trial} flags")
        for u, v in zip((z0, z1, fl), generic):
            assert np.array_equal(host(u).view(np.uint8), v.view(np.uint8))
        assert_bits(T.plain_ew(prog, [h for h, _ in g]), O.ew_plain(prog, [h for h, _ in ins]), "plain twin")


@pytest.mark.parametrize("n", [1, 129, 257, 20011])
def test_forced_specialisation_binary32(n):
    rng = np.random.default_rng(1000 + n)
    for trial in range(3):
        nin = int(rng.integers(1, 5))
        ins = []
        for k in range(nin):
            h = np.abs(rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 3, n)).astype(np.float32)
            lo = None if rng.random() < 0.3 else (h * 2.0 ** -30 * rng.uniform(-1, 1, n)).astype(np.float32)
            ins.append((h, lo))
        prog = random_program(rng, nin)
        mode = int(rng.choice([O.REL, O.ULP | O.STICKY]))
        p = T.params(panic_mode=mode, panic_tau=2.0 ** -18, panic_ulps=2.0)
        T.jit_mode(2)
        z0, z1, fl = T.twofold_ew_f32(prog, [(d32(h), None if lo is None else d32(lo)) for h, lo in ins], p=p)
        r0, r1, rf = O.ew32(prog, ins, mode=mode, tau=2.0 ** -18, m=2.0)
        assert_bits32(z0, r0, f"n={n} trial {trial} z0")
        assert_bits32(z1, r1, f"n={n} trial {trial} z1")
        assert_flags(fl, rf, f"n={n} trial {trial} flags")
        assert_bits32(T.plain_ew_f32(prog, [d32(h) for h, _ in ins]), O.ew32_plain(prog, [h for h, _ in ins]),
                      "plain twin")


@pytest.mark.parametrize("shift,n", [(0, 4099), (1, 4099), (2, 4100), (0, 4096)])
def test_binary32_four_element_path_and_unaligned_views(shift, n):
    """The binary32 kernels (twofold and plain twin) take four consecutive
    elements per thread in 16-byte accesses when every array is 16-byte
    aligned, with the last partial group through scalar accesses; views that
    start 1 or 2 elements into an allocation take the two-element kernels.
    All give the oracle's bits."""
    import torch
    rng = np.random.default_rng(77 + shift + n)
    ins = []
    for k in range(4):
        h = np.abs(rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 3, n)).astype(np.float32)
        lo = None if k == 3 else (h * 2.0 ** -30 * rng.uniform(-1, 1, n)).astype(np.float32)
        ins.append((h, lo))

    def view(a):
        if a is None:
            return None
        buf = torch.empty(n + 8, dtype=torch.float32, device="cuda")
        buf[shift:shift + n].copy_(torch.from_numpy(a))
        return buf[shift:shift + n]

    prog = [(O.MUL, 4, 0, 1), (O.ADD, 5, 4, 2), (O.DIV, 6, 5, 3), (O.SQRT, 7, 6, 6)]
    T.jit_mode(2)
    p = T.params(panic_mode=O.REL, panic_tau=2.0 ** -18)
    z0, z1, fl = T.twofold_ew_f32(prog, [(view(h), view(lo)) for h, lo in ins], p=p)
    r0, r1, rf = O.ew32(prog, ins, mode=O.REL, tau=2.0 ** -18, m=2.0)
    assert_bits32(z0, r0, f"shift {shift} n {n} z0")
    assert_bits32(z1, r1, f"shift {shift} n {n} z1")
    assert_flags(fl, rf, f"shift {shift} n {n} flags")
    assert_bits32(T.plain_ew_f32(prog, [view(h) for h, _ in ins]), O.ew32_plain(prog, [h for h, _ in ins]),
                  f"shift {shift} n {n} plain twin")


def test_automatic_mode_builds_once_per_program():
    """n >= 2^20 specialises; the second call of the same program reuses the
    kernel; the results equal the oracle (sampled) and a small call of the
    same program stays generic."""
    T.jit_mode(1)
    n = (1 << 20) + 3
    d = synth.ew_chain(n, seed=77)
    g = [(dev(d[k + "0"]), dev(d[k + "1"])) for k in "abcd"]
    prog = [(O.MUL, 4, 0, 1), (O.SUB, 5, 4, 2), (O.DIV, 6, 5, 3), (O.SQRT, 7, 6, 6), (O.ADD, 8, 7, 7)]
    _, b0, _ = T.jit_mode(-1)
    z0, z1, fl = T.twofold_ew(prog, g)
    _, b1, _ = T.jit_mode(-1)
    T.twofold_ew(prog, g)
    _, b2, f2 = T.jit_mode(-1)
    assert b1 == b0 + 1 and b2 == b1 and f2 == 0
    idx = np.r_[0:5000, n - 5000:n]
    ins = [(d[k + "0"][idx], d[k + "1"][idx]) for k in "abcd"]
    r0, r1, rf = O.ew(prog, ins)
    assert_bits(host(z0)[idx], r0, "z0")
    assert_bits(host(z1)[idx], r1, "z1")
    assert_flags(host(fl)[idx], rf, "flags")
