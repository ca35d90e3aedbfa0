"""twofold_dot_noalloc, the dot product for callers that cannot hand the
library any device memory at the call (code that must not touch the
allocator once running, or that has no spare buffer to lend as workspace).
It keeps its reduction partials in a static device array of the library.

Checked through the C ABI against twofold_dot (caller workspace) and
against the CPU oracle directly: the same z0, z1 and flag bits (the
tolerance of every parity test here: bit-exact), on two calls in a row,
since every call reuses the same static scratch.  The cases cover dotted
operands, a tail on one operand and tails on both, the latency schedule
(few leaves) and the throughput schedule, and the exact size limit of the
scratch.  Collected last on purpose; it also passes alone in a fresh
process."""
import ctypes

import numpy as np
import pytest

import oracle as O
import paper_1401_6235_gb300 as T
import synth
from tests.fp import bits, rand_tails

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as e
    e.build()
    return T.lib()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _out():
    import torch
    return (torch.empty(1, dtype=torch.float64, device="cuda"), torch.empty(1, dtype=torch.float64, device="cuda"),
            torch.empty(1, dtype=torch.uint8, device="cuda"))


def _pp(p):
    return None if p is None else ctypes.byref(p)


def _noalloc(L, x, y, xl=None, yl=None, p=None):
    import torch
    o = _out()
    ptr = lambda t: None if t is None else t.data_ptr()
    st = L.twofold_dot_noalloc(T.tf_in(ptr(x), ptr(xl)), T.tf_in(ptr(y), ptr(yl)), x.numel(),
                               T.tf_out(ptr(o[0]), ptr(o[1]), ptr(o[2])), _pp(p),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == T.TF_OK, T.strerror(st)
    return o


def _with_workspace(L, x, y, xl=None, yl=None, p=None):
    import torch
    o = _out()
    n = x.numel()
    nb = L.twofold_workspace_bytes(T.KIND_DOT, n, 1, _pp(p))
    ws = torch.empty(max(nb, 1), dtype=torch.uint8, device="cuda")
    ptr = lambda t: None if t is None else t.data_ptr()
    st = L.twofold_dot(T.tf_in(ptr(x), ptr(xl)), T.tf_in(ptr(y), ptr(yl)), n,
                       T.tf_out(ptr(o[0]), ptr(o[1]), ptr(o[2])), _pp(p), ptr(ws), ws.numel(),
                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == T.TF_OK, T.strerror(st)
    return o


def _oracle_bits(x, xl, y, yl, leaf=256):
    z0, z1 = O.reduce(x, xl, y, yl, L=leaf)
    return bits(z0), bits(z1), O.flag(z0, z1)


def _bits(o):
    import torch
    torch.cuda.synchronize()
    return (o[0].cpu().numpy().view(np.uint64)[0], o[1].cpu().numpy().view(np.uint64)[0],
            int(o[2].cpu().numpy()[0]))


# (n, operands with tails): dotted, x tails, y tails, both; few leaves (the
# latency schedule, n <= 2048 leaves of 256) and many (the throughput schedule)
CASES = [(65536, ""), (65536, "xy"), (300_007, "y"), (3_000_001, "x"), (3_000_001, "xy"), (1 << 24, "")]


@pytest.mark.parametrize("n,tails", CASES)
def test_noalloc_dot_matches_workspace_dot_and_oracle_on_two_calls(L, n, tails):
    x, y = synth.dot_uniform(n, seed=n)
    rng = np.random.default_rng(n)
    xl = rand_tails(rng, x, 30, 60) if "x" in tails else None
    yl = rand_tails(rng, y, 30, 60) if "y" in tails else None
    gx, gy = _dev(x), _dev(y)
    gxl = _dev(xl) if xl is not None else None
    gyl = _dev(yl) if yl is not None else None
    ref = _bits(_with_workspace(L, gx, gy, gxl, gyl))
    first = _bits(_noalloc(L, gx, gy, gxl, gyl))
    # a different dot in between, then the first again: the shared scratch
    # keeps the previous call's partials, which must not leak into a result
    _bits(_noalloc(L, gy, gx))
    second = _bits(_noalloc(L, gx, gy, gxl, gyl))
    assert first == ref and second == ref, (first, second, ref)
    assert first == _oracle_bits(x, xl, y, yl), (first, _oracle_bits(x, xl, y, yl))


def test_noalloc_dot_at_the_scratch_limit(L):
    """Leaves of one element: n = 2^23 makes exactly 32768 partial blocks of
    256 leaves, which fill the 512 KiB scratch; the result is the
    workspace dot's and the oracle's, twice in a row."""
    n = 1 << 23
    p = T.params(leaf=1)
    x, y = synth.dot_uniform(n, seed=5)
    gx, gy = _dev(x), _dev(y)
    ref = _bits(_with_workspace(L, gx, gy, p=p))
    first = _bits(_noalloc(L, gx, gy, p=p))
    second = _bits(_noalloc(L, gx, gy, p=p))
    assert first == ref and second == ref, (first, second, ref)
    assert first == _oracle_bits(x, None, y, None, leaf=1)


def test_noalloc_rejects_requests_beyond_its_scratch(L):
    """More partial blocks than the static array holds: TF_EUNSUPPORTED,
    decided on the host before anything is launched."""
    fake = 1 << 20
    out = T.tf_out(fake, fake, None)
    st = L.twofold_dot_noalloc(T.tf_in(fake, None), T.tf_in(fake, None), 1 << 40, out, None, None)
    assert st == T.TF_EUNSUPPORTED
    # one block past the limit: 2^23 + 1 one-element leaves make 32769 blocks
    p = T.params(leaf=1)
    st = L.twofold_dot_noalloc(T.tf_in(fake, None), T.tf_in(fake, None), (1 << 23) + 1, out, ctypes.byref(p), None)
    assert st == T.TF_EUNSUPPORTED
