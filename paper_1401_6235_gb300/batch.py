"""Mixed persistent batches of sum, dot and Horner jobs (one kernel launch
per batch), their replay from a captured CUDA graph, and an autotuner that
picks the batch configuration (leaves per work item, points per item, CTA
size) by timing candidates on the device.

Every job's result is the one its single-job entry point returns, bit for
bit, for any configuration; the tuner only changes the speed.  Marshalling
only: the work runs in ``twofold_batch_launch`` (C ABI, include/twofold.h).
"""
from __future__ import annotations

import ctypes
import json
import math
import os

from . import (JOB_DOT, JOB_HORNER, JOB_SUM, _check, _dev, _pp, _stream, _torch, lib, tf_batch_config,
               tf_batch_plan, tf_in, tf_job, tf_out, tf_params)


class Job:
    """One job of a batch: the tensors it reads and the result tensors."""

    def __init__(self, kind, n, x, xl=None, y=None, yl=None, coefs=None, k=0, out=None):
        torch = _torch()
        self.kind, self.n, self.k = kind, n, k
        self.x, self.xl, self.y, self.yl, self.coefs = x, xl, y, yl, coefs
        m = n if kind == JOB_HORNER else 1
        dev = x.device if x is not None else torch.device("cuda")
        self.out = out if out is not None else (torch.empty(m, dtype=torch.float64, device=dev),
                                                torch.empty(m, dtype=torch.float64, device=dev),
                                                torch.empty(m, dtype=torch.uint8, device=dev))

    def struct(self) -> tf_job:
        j = tf_job()
        j.kind, j.k, j.n = self.kind, self.k, self.n
        j.x = tf_in(_dev(self.x, "x") if self.n else None, _dev(self.xl, "xl") if self.n else None)
        j.y = tf_in(_dev(self.y, "y") if self.y is not None and self.n else None,
                    _dev(self.yl, "yl") if self.yl is not None and self.n else None)
        j.coefs = _dev(self.coefs, "coefs") if self.coefs is not None else None
        j.out = tf_out(_dev(self.out[0]), _dev(self.out[1]), _dev(self.out[2]))
        return j

    def cost(self) -> float:
        return float(self.n) * (max(1, self.k) * 1.25 if self.kind == JOB_HORNER else 1.0)


def sum_job(x, xl=None, out=None) -> Job:
    return Job(JOB_SUM, x.numel(), x, xl, out=out)


def dot_job(x, y, xl=None, yl=None, out=None) -> Job:
    if y.numel() != x.numel():
        raise ValueError("x and y must have the same length")
    return Job(JOB_DOT, x.numel(), x, xl, y, yl, out=out)


def horner_job(coefs, x, out=None) -> Job:
    """p(x) = coefs[0] + coefs[1] x + ... with the degree k = len(coefs) - 1."""
    return Job(JOB_HORNER, x.numel(), x, coefs=coefs, k=coefs.numel() - 1, out=out)


def config(leaves_per_item=256, points_per_item=16384, threads=256, ctas_per_sm=0) -> tf_batch_config:
    return tf_batch_config(leaves_per_item, points_per_item, threads, ctas_per_sm)


class Batch:
    """A prepared batch: job tables in a device workspace and the host plan.

    ``launch()`` starts the persistent kernel (stream-ordered, no host work
    besides the launch); ``graph()`` captures one launch into a CUDA graph
    whose ``replay()`` runs the whole batch again."""

    def __init__(self, jobs, p: tf_params | None = None, cfg: tf_batch_config | None = None, stream=None):
        self.jobs = list(jobs)
        self.p, self.cfg = p, cfg
        n = len(self.jobs)
        self._arr = (tf_job * max(1, n))(*[j.struct() for j in self.jobs])
        cfgp = ctypes.byref(cfg) if cfg is not None else None
        nb = lib().twofold_batch_workspace_bytes(self._arr, n, _pp(p), cfgp)
        if n and nb == 0:
            raise ValueError("invalid batch (job kinds, sizes or configuration)")
        # the plan's tables live in this workspace for the batch's lifetime, so
        # it is the batch's own (not the shared scratch of the single calls)
        self.ws = _torch().empty(max(nb, 256), dtype=_torch().uint8, device="cuda")
        self.plan = tf_batch_plan()
        _check(lib().twofold_batch_prepare(self._arr, n, _pp(p), cfgp, _dev(self.ws), self.ws.numel(),
                                           ctypes.byref(self.plan), _stream(stream)), "twofold_batch_prepare")

    def launch(self, stream=None) -> None:
        _check(lib().twofold_batch_launch(ctypes.byref(self.plan), _stream(stream)), "twofold_batch_launch")

    def graph(self):
        """One launch captured into a torch CUDA graph (replay() reruns it)."""
        torch = _torch()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            self.launch(s)                      # warm launch outside the capture
            s.synchronize()
            with torch.cuda.graph(g, stream=s):
                self.launch(s)
        torch.cuda.current_stream().wait_stream(s)
        return g

    @property
    def outputs(self):
        return [j.out for j in self.jobs]


# ------------------------------------------------------------------ autotuner

def signature(jobs, p: tf_params | None = None) -> str:
    """A key for the tuning cache: per kind, the job count in each power-of-
    two size class (and the degree class for Horner), plus the leaf length."""
    hist = {}
    for j in jobs:
        key = (j.kind, int(math.log2(max(1, j.n))), int(math.log2(max(1, j.k))) if j.kind == JOB_HORNER else 0)
        hist[key] = hist.get(key, 0) + 1
    leaf = p.leaf if p is not None else 256
    return json.dumps({"leaf": leaf, "jobs": sorted([list(k) + [v] for k, v in hist.items()])})


def candidates():
    out = []
    for t in (128, 256, 512):
        for b in (32, 64, 128, 256, 512):
            if b > t:
                continue
            for pts in (4096, 16384, 65536):
                out.append((b, pts, t))
    return out


_CACHE: dict = {}


def _cache_path():
    return os.environ.get("TWOFOLD_TUNE_CACHE")


def _load_cache():
    path = _cache_path()
    if path and os.path.exists(path) and not _CACHE:
        with open(path) as f:
            _CACHE.update(json.load(f))


def _save_cache():
    path = _cache_path()
    if path:
        with open(path, "w") as f:
            json.dump(_CACHE, f, indent=1, sort_keys=True)


def time_batch(b: Batch, reps=5) -> float:
    """Milliseconds per launch (CUDA events, after two warm launches)."""
    torch = _torch()
    for _ in range(2):
        b.launch()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        b.launch()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(jobs, p: tf_params | None = None, cands=None, reps=5, verbose=False) -> tf_batch_config:
    """The fastest configuration for this job mix, measured on the current
    device; cached in memory by signature() (and in the JSON file named by
    $TWOFOLD_TUNE_CACHE when set)."""
    _load_cache()
    key = signature(jobs, p)
    if key in _CACHE:
        return config(*_CACHE[key]["cfg"])
    best, best_ms, log = None, float("inf"), []
    for b_, pts, t in (cands or candidates()):
        cfg = config(b_, pts, t)
        ms = time_batch(Batch(jobs, p, cfg), reps)
        log.append((b_, pts, t, ms))
        if verbose:
            print(f"  leaves/item {b_:4d} points/item {pts:6d} threads {t:4d}: {ms:.3f} ms")
        if ms < best_ms:
            best, best_ms = (b_, pts, t, 0), ms
    _CACHE[key] = {"cfg": list(best), "ms": best_ms, "tried": len(log)}
    _save_cache()
    return config(*best)
