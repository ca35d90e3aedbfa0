"""GPU parity of Horner (C ABI) with the oracle: every degree used by the
workload plus edges (k = 0, 1, large k), ragged sizes, special points, and
the batched launch over k in {5, 10, 20, 30} at 2^24 points each in full."""
import numpy as np
import pytest

import oracle as O
import paper_1401_6235_gb300 as T
import synth
from tests.gpu_util import SPECIAL, assert_bits, assert_flags, dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as e
    e.build()


@pytest.mark.parametrize("k", [0, 1, 2, 5, 10, 20, 30, 200])
@pytest.mark.parametrize("n", [1, 255, 257, 100003])
def test_horner_degrees(k, n):
    a = synth.binomial_coefs(min(k, 30))
    if k > 30:
        a = np.random.default_rng(k).standard_normal(k + 1)
    x = synth.horner_points(n, seed=k + n)
    r0, r1, rf = O.horner(a, x)
    z0, z1, fl = T.twofold_horner(dev(a), dev(x))
    assert_bits(z0, r0, "z0")
    assert_bits(z1, r1, "z1")
    assert_flags(fl, rf, "flags")
    assert_bits(T.plain_horner(dev(a), dev(x)), O.horner_plain(a, x), "plain")
    assert_bits(T.plain_horner(dev(a), dev(x)), r0, "plain == z0")


def test_horner_special_points():
    a = np.array([1.5, -2.0, 0.25, 1e300, -3.0])
    x = np.concatenate([SPECIAL, -SPECIAL])
    r0, r1, rf = O.horner(a, x)
    z0, z1, fl = T.twofold_horner(dev(a), dev(x))
    assert_bits(z0, r0, "z0")
    assert_bits(z1, r1, "z1")
    assert_flags(fl, rf, "flags")


def test_horner_batched_config_full():
    ks = [5, 10, 20, 30]
    npts = 1 << 24
    coefs = np.concatenate([synth.binomial_coefs(k) for k in ks])
    coff = np.concatenate([[0], np.cumsum([k + 1 for k in ks])[:-1]]).astype(np.int32)
    x = np.concatenate([synth.horner_points(npts, seed=0, stream=j) for j in range(len(ks))])
    xoff = (np.arange(len(ks) + 1) * npts).astype(np.int64)
    r0, r1, rf = O.horner_batched(coefs, coff, ks, x, xoff)
    z0, z1, fl = T.twofold_horner_batched(dev(coefs), coff, ks, dev(x), xoff)
    assert_bits(z0, r0, "z0")
    assert_bits(z1, r1, "z1")
    assert_flags(fl, rf, "flags")
    pz = T.plain_horner_batched(dev(coefs), coff, ks, dev(x), xoff)
    assert_bits(pz, r0, "plain twin == z0")


def test_horner_batched_many_uneven_jobs():
    """More jobs than the inline table holds (job table in the workspace)."""
    rng = np.random.default_rng(2)
    nj = 100
    ks = rng.integers(0, 40, nj).astype(np.int32)
    lens = rng.integers(0, 5000, nj)
    lens[:3] = 0
    coefs = rng.standard_normal(int(np.sum(ks + 1)))
    coff = np.concatenate([[0], np.cumsum(ks + 1)[:-1]]).astype(np.int32)
    xoff = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    x = rng.uniform(-1.2, 1.2, int(xoff[-1]))
    r0, r1, rf = O.horner_batched(coefs, coff, ks, x, xoff)
    z0, z1, fl = T.twofold_horner_batched(dev(coefs), coff, ks, dev(x), xoff)
    assert_bits(z0, r0, "z0")
    assert_bits(z1, r1, "z1")
    assert_flags(fl, rf, "flags")


def test_horner_on_mapped_host_buffers():
    """Pinned host points and results that the device maps: the bits of the
    device-buffer call (single and batched)."""
    import torch
    a = synth.binomial_coefs(12)
    x = synth.horner_points(30011, seed=8)
    hx = torch.from_numpy(x).pin_memory()
    ga = torch.from_numpy(a).cuda()
    z = T.twofold_horner(ga, hx)
    torch.cuda.synchronize()
    d = T.twofold_horner(ga, torch.from_numpy(x).cuda())
    for u, v in zip(z, d):
        assert not u.is_cuda
        assert np.array_equal(u.numpy().view(np.uint8), v.cpu().numpy().view(np.uint8))
    zb = T.twofold_horner_batched(ga, [0, 0], [12, 5], hx, [0, 10000, 30011])
    torch.cuda.synchronize()
    r0, r1, rf = O.horner(a, x[:10000])
    assert np.array_equal(zb[0].numpy()[:10000].view(np.uint64), np.asarray(r0).view(np.uint64))
    assert np.array_equal(zb[1].numpy()[:10000].view(np.uint64), np.asarray(r1).view(np.uint64))
