"""Seeded synthetic inputs for the twofold workloads.

The only module that both the CPU oracle (tests, CPU baseline) and the CUDA
library's callers use.  It generates input arrays and, for ill-conditioned
dot products, their exact value; it holds none of the twofold method's
arithmetic.  All randomness is counter-based SplitMix64 (see ``synth.c``), so
any slice of any array can be regenerated on its own and generation is split
over host threads.

Workload recipes (sizes are parameters; defaults are the full workloads):

* ``dot_uniform``   x, y i.i.d. uniform[-1, 1], seed 0, x then y (dot, n=65536).
* ``ew_chain``      a, b, c: random sign x 10^U(-3,3); d: 10^U(-3,3);
                    tails uniform in +-1/2 ulp of the head (chain over 2^28).
* ``cond_dots``     4096 dots of 2^16 with condition 10^U(2,30) per dot.
* ``horner``        x uniform[0.9, 1.1]; coefficients of (x-1)^k, k in {5,10,20,30}.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_lib = None

_THREADS = max(1, min(16, os.cpu_count() or 1))
_CHUNK = 1 << 21


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so (plain C, no FP contraction)."""
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu99", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", src, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        d, i64, u64, p = ctypes.c_double, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
        L.synth_u64.argtypes = [u64, u64, u64]
        L.synth_u64.restype = u64
        L.synth_uniform.argtypes = [u64, u64, i64, i64, d, d, p]
        L.synth_loguniform.argtypes = [u64, u64, i64, i64, d, d, ctypes.c_int, p]
        L.synth_ulp_tails.argtypes = [u64, u64, i64, i64, p, p]
        L.synth_exact_dot.argtypes = [p, p, i64, p, p]
        L.synth_exact_sum.argtypes = [p, p, i64]
        L.synth_exact_sum.restype = d
        L.synth_cond_dot.argtypes = [u64, i64, d, p, p, p, p]
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _chunked(n: int, fn) -> None:
    spans = [(i, min(n, i + _CHUNK)) for i in range(0, n, _CHUNK)]
    if len(spans) <= 1:
        for s, e in spans:
            fn(s, e)
        return
    with ThreadPoolExecutor(_THREADS) as ex:
        list(ex.map(lambda se: fn(*se), spans))


def uniform(seed: int, stream: int, n: int, lo: float, hi: float, out=None) -> np.ndarray:
    out = np.empty(n, np.float64) if out is None else out
    L = lib()
    _chunked(n, lambda s, e: L.synth_uniform(seed, stream, s, e - s, lo, hi, _ptr(out) + 8 * s))
    return out


def uniform_slice(seed: int, stream: int, a: int, b: int, lo: float, hi: float) -> np.ndarray:
    """Elements [a, b) of the stream that uniform() draws from index 0 (the
    generator is counter-based, so any slice is regenerable on its own)."""
    out = np.empty(b - a, np.float64)
    L = lib()
    _chunked(b - a, lambda s, e: L.synth_uniform(seed, stream, a + s, e - s, lo, hi, _ptr(out) + 8 * s))
    return out


def loguniform(seed: int, stream: int, n: int, e_lo: float, e_hi: float, signed: bool,
               out=None) -> np.ndarray:
    out = np.empty(n, np.float64) if out is None else out
    L = lib()
    _chunked(n, lambda s, e: L.synth_loguniform(seed, stream, s, e - s, e_lo, e_hi, int(signed),
                                                 _ptr(out) + 8 * s))
    return out


def ulp_tails(seed: int, stream: int, heads: np.ndarray, out=None) -> np.ndarray:
    heads = np.ascontiguousarray(heads, np.float64)
    n = heads.size
    out = np.empty(n, np.float64) if out is None else out
    L = lib()
    _chunked(n, lambda s, e: L.synth_ulp_tails(seed, stream, s, e - s, _ptr(heads) + 8 * s,
                                                _ptr(out) + 8 * s))
    return out


# ----------------------------------------------------------------- workloads

def dot_uniform(n: int = 65536, seed: int = 0):
    """x, y i.i.d. uniform[-1, 1] (x is stream 0, y stream 1)."""
    return uniform(seed, 0, n, -1.0, 1.0), uniform(seed, 1, n, -1.0, 1.0)


EW_CHAIN_STREAMS = {"a0": 0, "b0": 1, "c0": 2, "d0": 3, "a1": 4, "b1": 5, "c1": 6, "d1": 7}


def ew_chain(n: int = 1 << 28, seed: int = 0, pinned=None) -> dict:
    """Inputs of z = sqrt((a*b + c)/d) over n twofolds.

    ``pinned``: optional callable (n) -> writable float64 ndarray used as the
    output buffer of each array (e.g. views of pinned host memory)."""
    alloc = pinned if pinned is not None else (lambda m: np.empty(m, np.float64))
    out = {}
    for k in ("a0", "b0", "c0"):
        out[k] = loguniform(seed, EW_CHAIN_STREAMS[k], n, -3.0, 3.0, True, out=alloc(n))
    out["d0"] = loguniform(seed, EW_CHAIN_STREAMS["d0"], n, -3.0, 3.0, False, out=alloc(n))
    for k in ("a", "b", "c", "d"):
        out[k + "1"] = ulp_tails(seed, EW_CHAIN_STREAMS[k + "1"], out[k + "0"], out=alloc(n))
    return out


def exact_dot(x: np.ndarray, y: np.ndarray):
    """(nearest double to the exact dot, exact condition number)."""
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    d = ctypes.c_double()
    c = ctypes.c_double()
    lib().synth_exact_dot(_ptr(x), _ptr(y), x.size, ctypes.byref(d), ctypes.byref(c))
    return d.value, c.value


def exact_sum(x: np.ndarray, xl: np.ndarray | None = None) -> float:
    x = np.ascontiguousarray(x, np.float64)
    if xl is not None:
        xl = np.ascontiguousarray(xl, np.float64)
    return lib().synth_exact_sum(_ptr(x), _ptr(xl) if xl is not None else None, x.size)


def cond_dot(seed: int, n: int, cond: float):
    """One ill-conditioned dot: (x, y, exact dot rounded to nearest, realised cond)."""
    x = np.empty(n, np.float64)
    y = np.empty(n, np.float64)
    d = ctypes.c_double()
    c = ctypes.c_double()
    lib().synth_cond_dot(seed, n, cond, _ptr(x), _ptr(y), ctypes.byref(d), ctypes.byref(c))
    return x, y, d.value, c.value


def cond_dots(njobs: int = 4096, n: int = 1 << 16, seed: int = 0, e_lo: float = 2.0,
              e_hi: float = 30.0, x=None, y=None):
    """``njobs`` dots of length n laid end to end; dot j has target condition
    10^U(e_lo, e_hi) (U from stream 9 of ``seed``, index j) and is built from
    seed ``seed * 2^20 + j``.  Returns x, y, offsets (njobs+1), exact dots,
    realised conditions and target conditions."""
    x = np.empty(njobs * n, np.float64) if x is None else x
    y = np.empty(njobs * n, np.float64) if y is None else y
    targets = 10.0 ** uniform(seed, 9, njobs, e_lo, e_hi)
    exact = np.empty(njobs)
    cond = np.empty(njobs)
    L = lib()

    def one(j):
        d = ctypes.c_double()
        c = ctypes.c_double()
        L.synth_cond_dot((seed << 20) + j, n, float(targets[j]), _ptr(x) + 8 * j * n,
                         _ptr(y) + 8 * j * n, ctypes.byref(d), ctypes.byref(c))
        exact[j] = d.value
        cond[j] = c.value

    with ThreadPoolExecutor(_THREADS) as ex:
        list(ex.map(one, range(njobs)))
    offs = np.arange(njobs + 1, dtype=np.int64) * n
    return x, y, offs, exact, cond, targets


def cond_dots_sized(sizes, conds, seed: int = 0, x=None, y=None):
    """Dots of the given lengths and target conditions laid end to end (dot j
    built from seed ``seed * 2^20 + j``): x, y, offsets, exact dots, realised
    conditions.  ``x``/``y``: optional output buffers (e.g. pinned memory)."""
    sizes = np.asarray(sizes, np.int64)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    x = np.empty(int(offs[-1]), np.float64) if x is None else x
    y = np.empty(int(offs[-1]), np.float64) if y is None else y
    exact = np.empty(sizes.size)
    cond = np.empty(sizes.size)
    L = lib()

    def one(j):
        d = ctypes.c_double()
        c = ctypes.c_double()
        L.synth_cond_dot((seed << 20) + j, int(sizes[j]), float(conds[j]), _ptr(x) + 8 * int(offs[j]),
                         _ptr(y) + 8 * int(offs[j]), ctypes.byref(d), ctypes.byref(c))
        exact[j] = d.value
        cond[j] = c.value

    with ThreadPoolExecutor(_THREADS) as ex:
        list(ex.map(one, range(sizes.size)))
    return x, y, offs, exact, cond


def binomial_coefs(k: int) -> np.ndarray:
    """Ascending coefficients a_0..a_k of (x-1)^k; exact in binary64 for k <= 30."""
    return np.array([math.comb(k, i) * (-1) ** (k - i) for i in range(k + 1)], np.float64)


def horner_points(n: int = 1 << 24, seed: int = 0, stream: int = 0) -> np.ndarray:
    return uniform(seed, stream, n, 0.9, 1.1)
