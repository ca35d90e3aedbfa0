"""Pins of the oracle's sum and dot (ATF1 accumulator, blocked pairwise order).

* z0 of every twofold reduction equals an independent plain-float
  implementation of the same order written here in Python (pins the leaf
  size, the left-to-right leaf order and the pairwise tree with odd carry);
* the tree is split-invariant on aligned 2^k-leaf blocks (what lets a GPU
  reduce blocks independently and combine the partials);
* z0 + z1 meets the compensated-summation bound gamma_n^2 * sum|terms|
  (Ogita, Rump, Oishi 2005) against exact values from an integer accumulator;
* dotted inputs and +0 tails give identical bits; n = 0 gives (+0, +0);
* panic flags rise with the condition number of ill-conditioned dots.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth
from tests.fp import bits

u = 2.0 ** -53


def gamma(n):
    return n * u / (1 - n * u)


def plain_tree_py(terms, L):
    """Plain binary64 sum in the blocked pairwise order, Python floats."""
    n = len(terms)
    if n == 0:
        return 0.0
    leaves = []
    for b in range(0, n, L):
        s = 0.0
        for t in terms[b:b + L]:
            s = s + t
        leaves.append(s)
    while len(leaves) > 1:
        nxt = [leaves[i] + leaves[i + 1] for i in range(0, len(leaves) - 1, 2)]
        if len(leaves) % 2:
            nxt.append(leaves[-1])
        leaves = nxt
    return leaves[0]


SIZES = [0, 1, 2, 255, 256, 257, 1000, 4097]
LEAVES = [1, 3, 256]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("L", LEAVES)
def test_sum_z0_is_plain_order(n, L):
    x, _ = synth.dot_uniform(n, seed=11)
    z0, z1 = O.reduce(x, L=L)
    ref = plain_tree_py([float(v) for v in x], L)
    assert bits(z0) == bits(ref)
    assert bits(O.reduce_plain(x, L=L)) == bits(ref)


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("L", LEAVES)
def test_dot_z0_is_plain_order(n, L):
    x, y = synth.dot_uniform(n, seed=12)
    z0, z1 = O.reduce(x, None, y, None, L=L)
    ref = plain_tree_py([float(a) * float(b) for a, b in zip(x, y)], L)
    assert bits(z0) == bits(ref)
    assert bits(O.reduce_plain(x, y, L=L)) == bits(ref)


def test_empty_is_positive_zero():
    z0, z1 = O.reduce(np.zeros(0))
    assert bits(z0) == 0 and bits(z1) == 0
    z0, z1 = O.reduce(np.zeros(0), None, np.zeros(0), None)
    assert bits(z0) == 0 and bits(z1) == 0


@pytest.mark.parametrize("m", [1, 2, 5, 8, 13, 64, 100])
def test_tree_split_on_aligned_blocks(m):
    """node i of level j covers leaves [i 2^j, min((i+1) 2^j, m)): reducing
    aligned 2^k blocks separately and then their results gives the same root."""
    rng = np.random.default_rng(m)
    nodes = np.stack([rng.standard_normal(m), rng.standard_normal(m) * 1e-17], 1)
    root = O.tree(nodes)
    for k in range(0, 7):
        b = 1 << k
        parts = [O.tree(nodes[s:s + b]) for s in range(0, m, b)]
        assert O.tree(parts) == root, (m, k)


@pytest.mark.parametrize("n,L", [(5000, 5000), (5000, 256), (20000, 7)])
def test_sum_accuracy_bound(n, L):
    rng = np.random.default_rng(n + L)
    x = rng.standard_normal(n) * np.exp2(rng.integers(-20, 20, n))
    z0, z1 = O.reduce(x, L=L)
    exact = synth.exact_sum(x)
    from fractions import Fraction as Fr
    err = abs(Fr(z0) + Fr(z1) - Fr(exact))
    bound = Fr(gamma(n) ** 2) * Fr(float(np.sum(np.abs(x)))) * 2 + Fr(u) * abs(Fr(exact))
    assert err <= bound


def test_dot_accuracy_and_flags_vs_condition():
    """Ill-conditioned dots (exact value by construction): z0 + z1 within the
    Dot2-style bound; the panic flag rate does not fall as condition grows."""
    from fractions import Fraction as Fr
    n = 4096
    conds = 10.0 ** np.linspace(2, 30, 29)
    flagged = []
    for j, c in enumerate(conds):
        x, y, exact, cr = synth.cond_dot(1000 + j, n, float(c))
        z0, z1 = O.reduce(x, None, y, None)
        s_abs = float(np.sum(np.abs(x * y)))
        err = abs(Fr(z0) + Fr(z1) - Fr(exact))
        bound = Fr(u) * abs(Fr(exact)) + Fr(gamma(2 * n) ** 2) * Fr(s_abs) * 2
        assert err <= bound, (c, cr)
        flagged.append((cr, O.flag(z0, z1) & O.PANIC))
    flagged.sort()
    lo = [f for cr, f in flagged if cr < 1e3]
    hi = [f for cr, f in flagged if cr > 1e16]
    assert sum(lo) == 0 and all(hi)


def test_dotted_equals_zero_tails():
    """Dotted x, y and twofolds with +0 tails give the same bits (MTF1 with
    zero tails is Two-Product; ATF1 with y1 = +0 is ATF1.1)."""
    x, y = synth.dot_uniform(3000, seed=5)
    z = np.zeros_like(x)
    a = O.reduce(x, None, y, None)
    b = O.reduce(x, z, y, z)
    assert bits(a[0]) == bits(b[0]) and bits(a[1]) == bits(b[1])
    a = O.reduce(x)
    b = O.reduce(x, z)
    assert bits(a[0]) == bits(b[0]) and bits(a[1]) == bits(b[1])


def test_batched_equals_single():
    x, y = synth.dot_uniform(10000, seed=8)
    offs = np.array([0, 1, 1, 300, 4096, 10000])
    z0, z1, fl = O.dot_batched(x, None, y, None, offs)
    for j in range(len(offs) - 1):
        a, b = offs[j], offs[j + 1]
        r = O.reduce(x[a:b], None, y[a:b], None)
        assert bits(z0[j]) == bits(r[0]) and bits(z1[j]) == bits(r[1])
        assert fl[j] == O.flag(*r)
