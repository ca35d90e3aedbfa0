"""The C-ABI library without a GPU: it builds, loads, exports every symbol
that include/twofold.h declares, and rejects bad arguments on the host
before any launch (no compute call is made here)."""
import ctypes
import os
import re

import numpy as np
import pytest

import __graft_entry__ as entry
import paper_1401_6235_gb300 as T

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "twofold.h")


@pytest.fixture(scope="module")
def L():
    entry.build()
    return T.lib()


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", src)) - {"sizeof"})


def test_every_declared_symbol_is_exported(L):
    names = declared()
    assert len(names) >= 17
    for name in names:
        assert hasattr(L, name), name
        assert name in T.SIGNATURES, f"binding lacks {name}"


def test_binding_names_match_header():
    assert sorted(T.SIGNATURES) == declared()


def test_strerror_and_version(L):
    assert T.strerror(0) == "ok"
    assert T.strerror(-2) == "workspace too small"
    assert L.twofold_version() >= 100


def _prog(rows):
    return np.ascontiguousarray(np.asarray(rows, np.int32).reshape(-1, 4))


FAKE = 1 << 20       # an aligned non-null address: never dereferenced by the host checks


def _call_ew(L, rows, nin=2, n=10, out_hi=FAKE, in_lo=None):
    p = _prog(rows)
    ins = (T.tf_in * nin)(*[T.tf_in(FAKE, in_lo) for _ in range(nin)])
    out = T.tf_out(out_hi, FAKE, None)
    return L.twofold_ew(p.ctypes.data, p.shape[0], ins, nin, n, out, None, None)


@pytest.mark.parametrize("rows", [
    [(11, 2, 0, 1)],                # unknown op
    [(0, 2, 0, 1)],                 # unknown op
    [(1, 1, 0, 1)],                 # writes an input register
    [(1, 2, 0, 3)],                 # reads an undefined register
    [(1, 40, 0, 1)],                # register out of range
    [(1, 2, 5, 1)],                 # reads an undefined register
    [(1, 3, 2, 0), (1, 2, 0, 1)],   # reads a temporary before it is written
])
def test_ew_rejects_bad_programs(L, rows):
    assert _call_ew(L, rows) == T.TF_EINVAL


def test_ew_rejects_bad_pointers_and_sizes(L):
    ok = [(1, 2, 0, 1)]
    assert _call_ew(L, ok, n=-1) == T.TF_EINVAL
    assert _call_ew(L, ok, out_hi=None) == T.TF_EINVAL
    assert _call_ew(L, ok, out_hi=FAKE + 4) == T.TF_EINVAL          # misaligned
    assert _call_ew(L, ok, in_lo=FAKE + 2) == T.TF_EINVAL
    assert _call_ew(L, ok, n=0) == T.TF_OK                           # nothing to do, no launch
    too_long = [(1, 2, 0, 1)] * 33
    assert _call_ew(L, too_long) == T.TF_EINVAL


def test_reduce_rejects_bad_offsets_and_small_workspace(L):
    x = T.tf_in(FAKE, None)
    out = T.tf_out(FAKE, FAKE, None)
    offs = np.array([0, 10, 5], np.int64)
    assert L.twofold_dot_batched(x, x, offs.ctypes.data, 2, out, None, FAKE, 1 << 20, None) == T.TF_EINVAL
    offs = np.array([-1, 5], np.int64)
    assert L.twofold_sum_batched(x, offs.ctypes.data, 1, out, None, FAKE, 1 << 20, None) == T.TF_EINVAL
    # 40 jobs (job table in the workspace) with a 16-byte workspace
    offs = np.arange(41, dtype=np.int64) * 100
    assert L.twofold_dot_batched(x, x, offs.ctypes.data, 40, out, None, FAKE, 16, None) == T.TF_ENOSPC
    bad = T.params(leaf=0)
    assert L.twofold_dot(x, x, 100, out, ctypes.byref(bad), FAKE, 1 << 20, None) == T.TF_EINVAL
    bad = T.params(panic_tau=-1.0)
    assert L.twofold_dot(x, x, 100, out, ctypes.byref(bad), FAKE, 1 << 20, None) == T.TF_EINVAL
    bad = T.params(panic_ulps=float("nan"))
    assert L.twofold_dot(x, x, 100, out, ctypes.byref(bad), FAKE, 1 << 20, None) == T.TF_EINVAL
    bad = T.params(panic_mode=7)
    assert L.twofold_sum(x, 100, out, ctypes.byref(bad), FAKE, 1 << 20, None) == T.TF_EINVAL
    assert L.twofold_sum(x, -5, out, None, FAKE, 1 << 20, None) == T.TF_EINVAL


def test_combine_rejects_bad_arguments(L):
    """Every case fails validation before any copy or launch."""
    out = T.tf_out(FAKE, FAKE, None)
    assert L.twofold_combine(FAKE, FAKE, -1, out, None, FAKE, 1 << 20, None) == T.TF_EINVAL
    assert L.twofold_combine(FAKE, FAKE, 4, T.tf_out(None, FAKE, None), None, FAKE, 1 << 20, None) == T.TF_EINVAL
    assert L.twofold_combine(FAKE, FAKE, 4, T.tf_out(FAKE, FAKE + 4, None), None, FAKE, 1 << 20, None) == T.TF_EINVAL
    assert L.twofold_combine(None, FAKE, 4, out, None, FAKE, 1 << 20, None) == T.TF_EINVAL
    assert L.twofold_combine(FAKE, FAKE + 2, 4, out, None, FAKE, 1 << 20, None) == T.TF_EINVAL
    bad = T.params(panic_mode=7)
    assert L.twofold_combine(FAKE, FAKE, 4, out, ctypes.byref(bad), FAKE, 1 << 20, None) == T.TF_EINVAL
    assert L.twofold_combine(FAKE, FAKE, 40, out, None, FAKE, 2 * 256 - 8, None) == T.TF_ENOSPC
    assert L.twofold_combine(FAKE, FAKE, 40, out, None, None, 1 << 20, None) == T.TF_ENOSPC
    assert L.twofold_combine(FAKE, FAKE, 40, out, None, FAKE + 4, 1 << 20, None) == T.TF_ENOSPC


def test_reduce32_rejects_bad_arguments(L):
    """Every case fails validation before any launch."""
    x = T.tf_in_f32(FAKE, None)
    out = T.tf_out_f32(FAKE, FAKE, None)
    assert L.twofold_sum_f32(x, -1, out, None, FAKE, 1 << 20, None) == T.TF_EINVAL
    assert L.twofold_sum_f32(x, 10, T.tf_out_f32(FAKE + 2, FAKE, None), None, FAKE, 1 << 20, None) == T.TF_EINVAL
    assert L.twofold_sum_f32(T.tf_in_f32(FAKE + 1, None), 10, out, None, FAKE, 1 << 20, None) == T.TF_EINVAL
    assert L.twofold_dot_f32(x, T.tf_in_f32(None, None), 10, out, None, FAKE, 1 << 20, None) == T.TF_EINVAL
    bad = T.params(panic_mode=7)
    assert L.twofold_dot_f32(x, x, 10, out, ctypes.byref(bad), FAKE, 1 << 20, None) == T.TF_EINVAL
    assert L.twofold_dot_f32(x, x, 10 ** 6, out, None, None, 0, None) == T.TF_ENOSPC   # several blocks
    assert L.plain_sum_f32(FAKE, 10 ** 6, FAKE, None, FAKE, 64, None) == T.TF_ENOSPC
    assert L.plain_dot_f32(FAKE, None, 10, FAKE, None, FAKE, 1 << 20, None) == T.TF_EINVAL


def test_workspace_bound_covers_every_split(L):
    """The workspace query is an upper bound of what the call needs for any
    job mix with that total length (host arithmetic only)."""
    for n, nj in [(0, 1), (1, 1), (65536, 1), (1 << 28, 4096), (1000, 1000), (1 << 20, 3)]:
        b = L.twofold_workspace_bytes(T.KIND_DOT, n, nj, None)
        assert b >= 16 * (nj + 1) + 2 * 8 * 2048


def test_horner_rejects_bad_degree(L):
    out = T.tf_out(FAKE, FAKE, None)
    assert L.twofold_horner(FAKE, -1, FAKE, 10, out, None, None) == T.TF_EINVAL
    assert L.twofold_horner(FAKE, 5000, FAKE, 10, out, None, None) == T.TF_EINVAL
    assert L.twofold_horner(FAKE, 3, FAKE, 0, out, None, None) == T.TF_OK


def test_host_mapped_query_without_device(L):
    """The host-mapping query never fails: NULL and plain host memory (and
    any pointer when no device is present) give 0."""
    import numpy as np
    assert L.twofold_host_mapped(None) == 0
    a = np.zeros(16)
    if not __import__("torch").cuda.is_available():
        assert L.twofold_host_mapped(ctypes.c_void_p(a.ctypes.data)) == 0


def test_plain_arith_mode(L):
    """The plain twin's division / root setting: -1 queries, 0 and 1 set and
    return the previous mode, anything else is TF_EINVAL and changes nothing."""
    prev = L.plain_arith(-1)
    assert prev == T.PLAIN_NATIVE
    try:
        assert L.plain_arith(T.PLAIN_INTEGER) == T.PLAIN_NATIVE
        assert L.plain_arith(-1) == T.PLAIN_INTEGER
        assert L.plain_arith(2) == T.TF_EINVAL
        assert L.plain_arith(-2) == T.TF_EINVAL
        assert L.plain_arith(-1) == T.PLAIN_INTEGER
        with pytest.raises(T.TwofoldError):
            T.plain_arith(7)
    finally:
        L.plain_arith(prev)


def test_batch_rejects_bad_jobs_and_configs(L):
    """Host-side checks of the mixed batch, before any device call."""
    J = T.tf_job * 2
    out = T.tf_out(FAKE, FAKE, None)
    good = J(T.tf_job(T.JOB_DOT, 0, 100, T.tf_in(FAKE, None), T.tf_in(FAKE, None), None, out),
             T.tf_job(T.JOB_HORNER, 5, 100, T.tf_in(FAKE, None), T.tf_in(None, None), FAKE, out))
    cfg = lambda *a: ctypes.byref(T.tf_batch_config(*a))
    plan = T.tf_batch_plan()
    assert L.twofold_batch_workspace_bytes(good, 2, None, None) > 0
    for c in [(3, 4096, 256, 0), (512, 4096, 256, 0), (32, 0, 256, 0), (32, 4096, 100, 0), (32, 4096, 256, -1)]:
        assert L.twofold_batch_workspace_bytes(good, 2, None, cfg(*c)) == 0, c
        assert L.twofold_batch_prepare(good, 2, None, cfg(*c), FAKE, 1 << 30, ctypes.byref(plan), None) == T.TF_EINVAL
    bad = J(*good)
    bad[0].kind = 9
    assert L.twofold_batch_prepare(bad, 2, None, None, FAKE, 1 << 30, ctypes.byref(plan), None) == T.TF_EINVAL
    bad = J(*good)
    bad[1].x = T.tf_in(FAKE, FAKE)                  # Horner points take no tails
    assert L.twofold_batch_prepare(bad, 2, None, None, FAKE, 1 << 30, ctypes.byref(plan), None) == T.TF_EINVAL
    bad = J(*good)
    bad[1].k = 5000
    assert L.twofold_batch_prepare(bad, 2, None, None, FAKE, 1 << 30, ctypes.byref(plan), None) == T.TF_EINVAL
    bad = J(*good)
    bad[0].x = T.tf_in(FAKE + 4, None)              # misaligned
    assert L.twofold_batch_prepare(bad, 2, None, None, FAKE, 1 << 30, ctypes.byref(plan), None) == T.TF_EINVAL
    bad = J(*good)
    bad[0].n = -1
    assert L.twofold_batch_prepare(bad, 2, None, None, FAKE, 1 << 30, ctypes.byref(plan), None) == T.TF_EINVAL
    assert L.twofold_batch_prepare(good, 2, None, None, FAKE, 64, ctypes.byref(plan), None) == T.TF_ENOSPC
    assert L.twofold_batch_prepare(good, 2, None, None, FAKE + 8, 1 << 30, ctypes.byref(plan), None) == T.TF_ENOSPC
    assert L.twofold_batch_launch(ctypes.byref(T.tf_batch_plan()), None) == T.TF_EINVAL   # not prepared


def test_server_rejects_bad_arguments(L):
    """Host-side checks of the request server (no device needed)."""
    h = ctypes.c_void_p()
    assert L.twofold_server_create(100, 16, None, None, ctypes.byref(h)) == T.TF_EINVAL      # arena too small
    assert L.twofold_server_create(1 << 20, 0, None, None, ctypes.byref(h)) == T.TF_EINVAL   # no batch slots
    bad = T.params(leaf=0)
    assert L.twofold_server_create(1 << 20, 16, ctypes.byref(bad), None, ctypes.byref(h)) == T.TF_EINVAL
    cfg = T.tf_batch_config(3, 4096, 256, 0)
    assert L.twofold_server_create(1 << 20, 16, None, ctypes.byref(cfg), ctypes.byref(h)) == T.TF_EINVAL
    assert L.twofold_server_create(1 << 20, 16, None, None, None) == T.TF_EINVAL
    r = T.tf_request()
    tid = ctypes.c_uint64()
    assert L.twofold_server_submit(None, ctypes.byref(r), ctypes.byref(tid)) == T.TF_EINVAL
    assert L.twofold_server_wait(None, 1, 0, None) == T.TF_EINVAL
    assert L.twofold_server_destroy(None) == T.TF_EINVAL
    assert L.twofold_server_inject_failures(None, 1) == T.TF_EINVAL
