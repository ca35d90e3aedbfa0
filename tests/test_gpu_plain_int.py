"""plain_ew with its division and square root on the integer pipes
(plain_divsqrt(PLAIN_INTEGER)): the plain binary64 twin the twofold kernels
are also measured against.  Its results must be the IEEE results bit for
bit (the oracle's plain twin, and plain_ew in native mode) on edge values,
on wide random operands and on the chain workload, in the generic kernel
and in the runtime-specialised one."""
import numpy as np
import pytest

import oracle as O
import paper_1401_6235_gb300 as T
import synth
from tests.fp import rand_doubles
from tests.gpu_util import SPECIAL, assert_bits, dev

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def modes_restored():
    import __graft_entry__ as e
    e.build()
    jit, pm = T.jit_mode(-1)[0], T.plain_divsqrt(-1)
    yield
    T.jit_mode(jit)
    T.plain_divsqrt(pm)


def operands():
    x0, y0 = [a.ravel() for a in np.meshgrid(SPECIAL, SPECIAL)]
    rng = np.random.default_rng(11)
    rx, ry = rand_doubles(rng, 300007, -300, 300), rand_doubles(rng, 300007, -300, 300)
    # near-subnormal quotients and roots, and exact quotients / squares
    sx = rand_doubles(rng, 20000, -1074, -1000)
    ex = np.floor(rng.uniform(-2 ** 26, 2 ** 26, 20000))
    ey = np.floor(rng.uniform(1, 2 ** 26, 20000))
    x = np.concatenate([x0, rx, sx, ex * ey, ex * ex])
    y = np.concatenate([y0, ry, ry[:20000], ey, np.abs(ex) + 1.0])
    return x, y


@pytest.mark.parametrize("jit", [0, 2])
@pytest.mark.parametrize("op", [O.DIV, O.SQRT, O.ADD, O.SUB, O.MUL])
def test_integer_plain_op_equals_ieee(jit, op):
    x, y = operands()
    prog = [(op, 2, 0, 0 if op == O.SQRT else 1)]
    gx, gy = dev(x), dev(y)
    T.jit_mode(jit)
    T.plain_divsqrt(T.PLAIN_NATIVE)
    native = T.plain_ew(prog, [gx, gy])
    assert T.plain_divsqrt(T.PLAIN_INTEGER) == T.PLAIN_NATIVE
    integer = T.plain_ew(prog, [gx, gy])
    ref = O.ew_plain(prog, [x, y])
    assert_bits(integer, ref, f"op {op} integer vs oracle")
    assert_bits(native, ref, f"op {op} native vs oracle")


@pytest.mark.parametrize("n", [1, 1000, 1 << 20, (1 << 20) + 77])
def test_integer_plain_chain(n):
    d = synth.ew_chain(n, seed=5)
    his = [d[k + "0"] for k in "abcd"]
    g = [dev(h) for h in his]
    T.plain_divsqrt(T.PLAIN_INTEGER)
    out = T.plain_ew(T.CHAIN_SQRT_MAD_DIV, g)
    assert_bits(out, O.ew_plain(T.CHAIN_SQRT_MAD_DIV, his), f"chain n={n}")

