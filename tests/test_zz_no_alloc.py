"""twofold_dot_noalloc, the dot product for callers that cannot hand the
library any device memory at the call (code that must not touch the
allocator once running, or that has no spare buffer to lend as workspace).
It keeps its reduction partials in a static device array of the library.

Checked through the C ABI against twofold_dot (caller workspace): the same
z0, z1 and flag bits (the tolerance of every parity test here: bit-exact),
on two calls in a row, since every call reuses the same static scratch.
Collected last on purpose; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

import paper_1401_6235_gb300 as T
import synth
from tests.fp import rand_tails

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


def _noalloc(L, x, y, xl=None, yl=None):
    import torch
    o = _out()
    ptr = lambda t: None if t is None else t.data_ptr()
    st = L.twofold_dot_noalloc(T.tf_in(ptr(x), ptr(xl)), T.tf_in(ptr(y), ptr(yl)), x.numel(),
                               T.tf_out(ptr(o[0]), ptr(o[1]), ptr(o[2])), None,
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == T.TF_OK, T.strerror(st)
    return o


def _with_workspace(L, x, y, xl=None, yl=None):
    import torch
    o = _out()
    n = x.numel()
    nb = L.twofold_workspace_bytes(T.KIND_DOT, n, 1, None)
    ws = torch.empty(max(nb, 1), dtype=torch.uint8, device="cuda")
    ptr = lambda t: None if t is None else t.data_ptr()
    st = L.twofold_dot(T.tf_in(ptr(x), ptr(xl)), T.tf_in(ptr(y), ptr(yl)), n,
                       T.tf_out(ptr(o[0]), ptr(o[1]), ptr(o[2])), None, ptr(ws), ws.numel(),
                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == T.TF_OK, T.strerror(st)
    return o


def _bits(o):
    import torch
    torch.cuda.synchronize()
    return (o[0].cpu().numpy().view(np.uint64)[0], o[1].cpu().numpy().view(np.uint64)[0],
            int(o[2].cpu().numpy()[0]))


@pytest.mark.parametrize("n,tails", [(65536, False), (3_000_001, True), (1 << 24, False)])
def test_noalloc_dot_matches_workspace_dot_on_two_calls(L, n, tails):
    x, y = synth.dot_uniform(n, seed=n)
    xl = rand_tails(np.random.default_rng(1), x, 30, 60) if tails else None
    gx, gy = _dev(x), _dev(y)
    gxl = _dev(xl) if tails else None
    ref = _bits(_with_workspace(L, gx, gy, gxl))
    first = _bits(_noalloc(L, gx, gy, gxl))
    # a different dot in between, then the first again: the shared scratch
    # keeps the previous call's partials, which must not leak into a result
    _bits(_noalloc(L, gy, gx))
    second = _bits(_noalloc(L, gx, gy, gxl))
    assert first == ref and second == ref, (first, second, ref)


def test_noalloc_rejects_requests_beyond_its_scratch(L):
    """More partial blocks than the static array holds: TF_EUNSUPPORTED,
    decided on the host before anything is launched."""
    fake = 1 << 20
    out = T.tf_out(fake, fake, None)
    st = L.twofold_dot_noalloc(T.tf_in(fake, None), T.tf_in(fake, None), 1 << 40, out, None, None)
    assert st == T.TF_EUNSUPPORTED
