"""The plain binary64 twins with plain_arith(PLAIN_INTEGER): plain_ew's
division and square root, and plain_horner(_batched)'s multiplication, on
the integer pipes.  These are the faster plain twins the twofold kernels
are also measured against.  Their results must be the IEEE results bit for
bit (the oracle's plain twins, and the same calls in native mode): edge
values, wide random operands and the benchmark's workloads, in every kernel
the calls choose (generic and runtime-specialised elementwise kernels).
The plain sum and dot keep their native operations in either mode."""
import math

import numpy as np
import pytest

import oracle as O
import paper_1401_6235_gb300 as T
import synth
from tests.fp import rand_doubles
from tests.gpu_util import SPECIAL, assert_bits, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def modes_restored():
    import __graft_entry__ as e
    e.build()
    jit, pm = T.jit_mode(-1)[0], T.plain_arith(-1)
    yield
    T.jit_mode(jit)
    T.plain_arith(pm)


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
    T.plain_arith(T.PLAIN_NATIVE)
    native = T.plain_ew(prog, [gx, gy])
    assert T.plain_arith(T.PLAIN_INTEGER) == T.PLAIN_NATIVE
    integer = T.plain_ew(prog, [gx, gy])
    ref = O.ew_plain(prog, [x, y])
    assert_bits(integer, ref, f"op {op} integer vs oracle")
    assert_bits(native, ref, f"op {op} native vs oracle")


@pytest.mark.parametrize("n", [1, 1000, 1 << 20, (1 << 20) + 77])
def test_integer_plain_chain(n):
    d = synth.ew_chain(n, seed=5)
    his = [d[k + "0"] for k in "abcd"]
    g = [dev(h) for h in his]
    T.plain_arith(T.PLAIN_INTEGER)
    out = T.plain_ew(T.CHAIN_SQRT_MAD_DIV, g)
    assert_bits(out, O.ew_plain(T.CHAIN_SQRT_MAD_DIV, his), f"chain n={n}")



def product_operands(rng, n):
    """Products of every class: ordinary, near the underflow and overflow
    thresholds, exact, and the special values."""
    x = rand_doubles(rng, n, -300, 300)
    y = rand_doubles(rng, n, -300, 300)
    k = n // 8
    x[:k] = rand_doubles(rng, k, -540, -500)          # products near 2^-1022 and below
    y[:k] = rand_doubles(rng, k, -540, -500)
    x[k:2 * k] = rand_doubles(rng, k, 500, 520)       # products near 2^1024 and beyond
    y[k:2 * k] = rand_doubles(rng, k, 500, 520)
    sx, sy = [a.ravel() for a in np.meshgrid(SPECIAL, SPECIAL)]
    x[2 * k:2 * k + sx.size] = sx
    y[2 * k:2 * k + sy.size] = sy
    return x, y


def test_plain_reductions_unchanged_by_the_mode():
    """plain_sum / plain_dot / plain_dot_batched give the oracle's bits in
    integer mode too (they keep the native operations)."""
    rng = np.random.default_rng(3)
    lens = [0, 1, 255, 257, 65536, 100003]
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    x, y = product_operands(rng, int(offs[-1]))
    T.plain_arith(T.PLAIN_INTEGER)
    got = T.plain_dot_batched(dev(x), dev(y), offs)
    ref = np.array([O.reduce_plain(x[a:b], y[a:b]) for a, b in zip(offs[:-1], offs[1:])])
    assert_bits(got, ref, "batched dot")
    assert_bits(T.plain_dot(dev(x), dev(y)), np.array([O.reduce_plain(x, y)]), "dot")
    assert_bits(T.plain_sum(dev(x)), np.array([O.reduce_plain(x)]), "sum")


@pytest.mark.parametrize("k", [0, 1, 5, 30])
def test_integer_plain_horner(k):
    rng = np.random.default_rng(100 + k)
    coef = rand_doubles(rng, k + 1, -4, 4)
    x = np.concatenate([rng.uniform(0.9, 1.1, 200003), rand_doubles(rng, 50000, -40, 40), SPECIAL])
    gc, gx = dev(coef), dev(x)
    T.plain_arith(T.PLAIN_NATIVE)
    native = T.plain_horner(gc, gx)
    T.plain_arith(T.PLAIN_INTEGER)
    integer = T.plain_horner(gc, gx)
    ref = O.horner_plain(coef, x)
    assert_bits(integer, ref, f"k={k} integer")
    assert_bits(native, ref, f"k={k} native")


def test_integer_plain_horner_batched_workload():
    """The benchmark's jobs: (x-1)^k expanded, k in {5, 10, 20, 30}, points
    uniform in [0.9, 1.1] (fewer points than the benchmark)."""
    rng = np.random.default_rng(7)
    ks = [5, 10, 20, 30]
    coefs, coff = [], []
    for k in ks:
        coff.append(sum(len(c) for c in coefs))
        coefs.append(np.array([float(math.comb(k, i) * (-1) ** (k - i)) for i in range(k + 1)]))
    npts = [100003, 65536, 1, 77777]
    xoff = np.concatenate([[0], np.cumsum(npts)]).astype(np.int64)
    x = rng.uniform(0.9, 1.1, int(xoff[-1]))
    T.plain_arith(T.PLAIN_INTEGER)
    got = host(T.plain_horner_batched(dev(np.concatenate(coefs)), coff, ks, dev(x), xoff))
    for j, k in enumerate(ks):
        a, b = xoff[j], xoff[j + 1]
        assert_bits(got[a:b], O.horner_plain(coefs[j], x[a:b]), f"job {j} k={k}")
