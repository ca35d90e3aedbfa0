"""Python side of the request server (C ABI twofold_server_*): submit sum,
dot, Horner and elementwise requests with host arrays, wait for their
results.  The scheduler (admission by device memory, continuous batching
into mixed persistent batches, copies and kernels on a pool of streams) runs
in the library's own thread; this module only marshals arrays and keeps them
alive until their request is done.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import (JOB_DOT, JOB_EW, JOB_HORNER, JOB_SUM, _check, _pp, lib, tf_batch_config, tf_params, tf_request,
               tf_request_info, tf_server_stats)


def _host(a):
    """A contiguous float64 host array (numpy, or a CPU torch tensor)."""
    if a is None:
        return None
    if hasattr(a, "is_cuda"):
        if a.is_cuda:
            raise ValueError("server requests take host arrays")
        a = a.numpy()
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _pinned(n, dtype):
    """Page-locked host output buffer (the scheduler's copies stay asynchronous)."""
    import torch
    t = torch.empty(max(n, 1), dtype=dtype).pin_memory()
    return t.numpy()[:n] if n else t.numpy()[:0]


class Ticket:
    def __init__(self, server, tid, keep, out):
        self.server, self.id, self._keep, self.out = server, tid, keep, out
        self.info = None
        self.status = None


class Server:
    def __init__(self, mem_cap: int, max_batch_jobs: int = 4096, p: tf_params | None = None,
                 cfg: tf_batch_config | None = None):
        h = ctypes.c_void_p()
        _check(lib().twofold_server_create(mem_cap, max_batch_jobs, _pp(p),
                                           ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(h)),
               "twofold_server_create")
        self._h = h

    # -------------------------------------------------------------- submit
    def _submit(self, kind, n, ins, coefs=None, k=0, prog=None, nin=0, nout=1, keep=()):
        r = tf_request()
        r.kind, r.k, r.n = kind, k, n
        for i, a in enumerate(ins):
            r.inp[i] = None if a is None else a.ctypes.data
        r.coefs = None if coefs is None else coefs.ctypes.data
        if prog is not None:
            r.prog, r.nprog, r.nin = prog.ctypes.data, prog.shape[0], nin
        import torch
        out = (_pinned(nout, torch.float64), _pinned(nout, torch.float64), _pinned(nout, torch.uint8))
        r.out_hi, r.out_lo, r.out_flags = out[0].ctypes.data, out[1].ctypes.data, out[2].ctypes.data
        tid = ctypes.c_uint64()
        _check(lib().twofold_server_submit(self._h, ctypes.byref(r), ctypes.byref(tid)), "twofold_server_submit")
        return Ticket(self, tid.value, (ins, coefs, prog) + tuple(keep), out)

    def submit_sum(self, x, xl=None) -> Ticket:
        x, xl = _host(x), _host(xl)
        return self._submit(JOB_SUM, x.size, [x, xl])

    def submit_dot(self, x, y, xl=None, yl=None) -> Ticket:
        x, y, xl, yl = _host(x), _host(y), _host(xl), _host(yl)
        if y.size != x.size:
            raise ValueError("x and y must have the same length")
        return self._submit(JOB_DOT, x.size, [x, xl, y, yl])

    def submit_horner(self, coefs, x) -> Ticket:
        c, x = _host(coefs), _host(x)
        return self._submit(JOB_HORNER, x.size, [x], coefs=c, k=c.size - 1, nout=x.size)

    def submit_ew(self, prog, inputs) -> Ticket:
        """inputs: up to 4 (hi, lo-or-None) host arrays; the program as for twofold_ew."""
        pa = np.ascontiguousarray(np.asarray(prog, np.int32).reshape(-1, 4))
        ins = []
        for h, lo in inputs:
            ins += [_host(h), _host(lo)]
        n = ins[0].size
        return self._submit(JOB_EW, n, ins, prog=pa, nin=len(inputs), nout=n)

    # ---------------------------------------------------------------- wait
    def wait(self, t: Ticket, timeout_ms: int = -1):
        """(z0, z1, flags) of the request; raises TwofoldError on failure."""
        info = tf_request_info()
        st = lib().twofold_server_wait(self._h, t.id, timeout_ms, ctypes.byref(info))
        t.status = st
        if st == -4:                       # TF_ETIMEOUT: still running, ticket valid
            return None
        t.info = info
        _check(st, "twofold_server_wait")
        return t.out

    def inject_failures(self, every: int) -> None:
        """Fail every `every`-th batch the scheduler starts from now on,
        before any of its work runs (host-side fault injection for tests;
        0 turns it off).  Its requests complete with TF_ECUDA."""
        _check(lib().twofold_server_inject_failures(self._h, every), "twofold_server_inject_failures")

    def stats(self) -> dict:
        s = tf_server_stats()
        _check(lib().twofold_server_stats(self._h, ctypes.byref(s)), "twofold_server_stats")
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close(self):
        if self._h:
            _check(lib().twofold_server_destroy(self._h), "twofold_server_destroy")
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
