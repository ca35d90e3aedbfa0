"""CPU oracle for twofold fast arithmetic (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``twofold_oracle.c`` (plain
C, binary64, round-to-nearest, no FP contraction) with ctypes and numpy and
shares no code with the CUDA library in ``paper_1401_6235_gb300``.

Every function follows one algorithm of Latkin, "Twofold fast arithmetic"
(arXiv:1401.6235); the C source cites the algorithm above each function and
lists the readings taken where the paper is silent or misprinted.

Pinned by ``tests/test_oracle_*.py`` against exact rational arithmetic, the
paper's worked examples and printed application logs, closed forms and
special-case reductions.  The paper states no error bound for RTF1; its pin
is a bound derived from its own steps (the exact remainder of the
first-order root correction plus one rounding per step), checked against a
high-precision square root for coupled and non-coupled inputs, besides the
Root section's worked example.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

ADD, SUB, MUL, DIV, SQRT = 1, 2, 3, 4, 5
PADD, PSUB, PMUL, PDIV, PSQRT = 6, 7, 8, 9, 10     # coupled (Dekker emulation) operations
PANIC, NONFINITE = 1, 2
REL, ULP = 0, 1
DEFAULT_TAU = 2.0 ** -40

THREADS = max(1, min(16, os.cpu_count() or 1))
_CHUNK = 1 << 18

CFLAGS = ["-O2", "-std=gnu99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


class _TF(ctypes.Structure):
    _fields_ = [("z0", ctypes.c_double), ("z1", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FP contraction, no fast-math)."""
    srcs = [os.path.join(_HERE, f) for f in ("twofold_oracle.c", "twofold_oracle_f32.c")]
    if force or not os.path.exists(_SO) or any(os.path.getmtime(_SO) < os.path.getmtime(s) for s in srcs):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, *srcs, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        _lib = load(_SO)
    return _lib


def load(path: str) -> ctypes.CDLL:
    """Open an oracle shared object and declare its signatures."""
    L = ctypes.CDLL(path)
    d, i, i64, p = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
    pd = ctypes.POINTER(ctypes.c_double)
    for name in ("tfo_two_sum", "tfo_two_diff", "tfo_two_prod", "tfo_div_rem", "tfo_fast_two_sum"):
        getattr(L, name).argtypes = [d, d, pd, pd]
    L.tfo_sqrt_rem.argtypes = [d, pd, pd]
    for name in ("tfo_atf1", "tfo_stf1", "tfo_mtf1", "tfo_dtf1", "tfo_mpf1", "tfo_dpf1"):
        getattr(L, name).argtypes = [d, d, d, d]
        getattr(L, name).restype = _TF
    for name in ("tfo_atf11", "tfo_stf11", "tfo_mtf11", "tfo_dtf11"):
        getattr(L, name).argtypes = [d, d, d]
        getattr(L, name).restype = _TF
    L.tfo_dtf111.argtypes = [d, d]
    L.tfo_dtf111.restype = _TF
    L.tfo_rpf1.argtypes = [d, d]
    L.tfo_rpf1.restype = _TF
    L.tfo_rpf11.argtypes = [d]
    L.tfo_rpf11.restype = _TF
    L.tfo_rtf1.argtypes = [d, d]
    L.tfo_rtf1.restype = _TF
    L.tfo_op.argtypes = [i, d, d, i, d, d, i, pd, pd]
    L.tfo_flag.argtypes = [d, d, i, d, d]
    L.tfo_flag.restype = ctypes.c_ubyte
    L.tfo_ew.argtypes = [p, i, p, p, i, i64, i64, p, p, p, i, d, d]
    L.tfo_ew_plain.argtypes = [p, i, p, i, i64, i64, p]
    L.tfo_reduce.argtypes = [p, p, p, p, i64, i64, i, p, pd, pd]
    L.tfo_reduce_leaves.argtypes = [p, p, p, p, i64, i64, i, i64, i64, p]
    L.tfo_tree.argtypes = [p, i64, pd, pd]
    L.tfo_reduce_plain.argtypes = [p, p, i64, i64, i, p]
    L.tfo_reduce_plain.restype = d
    L.tfo_horner.argtypes = [p, i, p, i64, i64, p, p, p, i, d, d]
    L.tfo_horner_plain.argtypes = [p, i, p, i64, i64, p]
    f = ctypes.c_float
    pf = ctypes.POINTER(ctypes.c_float)
    for name in ("tfof_two_sum", "tfof_two_diff", "tfof_two_prod", "tfof_div_rem", "tfof_fast_two_sum"):
        getattr(L, name).argtypes = [f, f, pf, pf]
    L.tfof_sqrt_rem.argtypes = [f, pf, pf]
    L.tfof_op.argtypes = [i, f, f, i, f, f, i, pf, pf]
    L.tfof_flag.argtypes = [f, f, i, f, f]
    L.tfof_flag.restype = ctypes.c_ubyte
    L.tfof_ew.argtypes = [p, i, p, p, i, i64, i64, p, p, p, i, f, f]
    L.tfof_ew_plain.argtypes = [p, i, p, i, i64, i64, p]
    L.tfof_reduce_sum.argtypes = [p, p, i64, i64, pf, pf]
    L.tfof_reduce.argtypes = [p, p, p, p, i64, i64, i, pf, pf]
    L.tfof_reduce_plain.argtypes = [p, p, i64, i64, i]
    L.tfof_reduce_plain.restype = f
    return L


# ------------------------------------------------------------------ scalars

def _pair(fn, *args):
    a = ctypes.c_double()
    b = ctypes.c_double()
    fn(*args, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def two_sum(a, b):
    """Algorithm 1.2: a + b -> (s, t)."""
    return _pair(lib().tfo_two_sum, a, b)


def fast_two_sum(a, b):
    """Algorithm 1.1 (three operations, exact when |a| >= |b|): a + b -> (s, t)."""
    return _pair(lib().tfo_fast_two_sum, a, b)


def two_diff(a, b):
    """Algorithm 2.2 (signs read as Shewchuk's): a - b -> (d, t)."""
    return _pair(lib().tfo_two_diff, a, b)


def two_prod(a, b):
    """Algorithm 3: a * b -> (p, e)."""
    return _pair(lib().tfo_two_prod, a, b)


def div_rem(a, b):
    """Algorithm 4: a / b -> (q, r), a = q b + r."""
    return _pair(lib().tfo_div_rem, a, b)


def sqrt_rem(a):
    """Algorithm 5: sqrt(a) -> (c, d), a = c^2 + d."""
    return _pair(lib().tfo_sqrt_rem, a)


def _tf(r):
    return r.z0, r.z1


def atf1(x0, x1, y0, y1): return _tf(lib().tfo_atf1(x0, x1, y0, y1))
def atf11(x0, x1, y0): return _tf(lib().tfo_atf11(x0, x1, y0))
def stf1(x0, x1, y0, y1): return _tf(lib().tfo_stf1(x0, x1, y0, y1))
def stf11(x0, x1, y0): return _tf(lib().tfo_stf11(x0, x1, y0))
def mtf1(x0, x1, y0, y1): return _tf(lib().tfo_mtf1(x0, x1, y0, y1))
def mtf11(x0, x1, y0): return _tf(lib().tfo_mtf11(x0, x1, y0))
def dtf1(x0, x1, y0, y1): return _tf(lib().tfo_dtf1(x0, x1, y0, y1))
def dtf11(x0, x1, y0): return _tf(lib().tfo_dtf11(x0, x1, y0))
def dtf111(x0, y0): return _tf(lib().tfo_dtf111(x0, y0))
def mpf1(x0, x1, y0, y1): return _tf(lib().tfo_mpf1(x0, x1, y0, y1))
def dpf1(x0, x1, y0, y1): return _tf(lib().tfo_dpf1(x0, x1, y0, y1))
def rpf1(x0, x1): return _tf(lib().tfo_rpf1(x0, x1))
def rpf11(x0): return _tf(lib().tfo_rpf11(x0))
def rtf1(x0, x1): return _tf(lib().tfo_rtf1(x0, x1))


def op(code, x, y=None):
    """One twofold op with operand kinds: x, y are (hi, lo) tuples or plain
    floats (dotted).  Returns (z0, z1)."""
    def split(v):
        if v is None:
            return 0.0, 0.0, 1
        if isinstance(v, tuple):
            return float(v[0]), float(v[1]), 0
        return float(v), 0.0, 1
    x0, x1, xd = split(x)
    y0, y1, yd = split(y)
    return _pair(lib().tfo_op, code, x0, x1, xd, y0, y1, yd)


def flag(z0, z1, mode=REL, tau=DEFAULT_TAU, m=1.0):
    return int(lib().tfo_flag(z0, z1, mode, tau, m))


# ------------------------------------------------------------------ arrays

def _f64(a):
    return np.ascontiguousarray(a, np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data


def _par(n, fn, chunk=_CHUNK, threads=None):
    spans = [(s, min(n, s + chunk)) for s in range(0, n, chunk)]
    t = THREADS if threads is None else threads
    if len(spans) <= 1 or t <= 1:
        for s, e in spans:
            fn(s, e)
        return
    with ThreadPoolExecutor(t) as ex:
        list(ex.map(lambda se: fn(*se), spans))


def ew(prog, inputs, mode=REL, tau=DEFAULT_TAU, m=1.0, threads=None):
    """Run a program (list of (op, dst, a, b)) over twofold arrays.

    ``inputs``: list of (hi, lo) with lo None for a dotted input.
    Returns (z0, z1, flags)."""
    prog_a = np.ascontiguousarray(np.asarray(prog, np.int32).reshape(-1, 4))
    his = [_f64(h) for h, _ in inputs]
    los = [None if lo is None else _f64(lo) for _, lo in inputs]
    n = his[0].size if his else 0
    hp = (ctypes.c_void_p * len(his))(*[_ptr(h) for h in his])
    lp = (ctypes.c_void_p * len(los))(*[_ptr(lo) for lo in los])
    z0 = np.empty(n)
    z1 = np.empty(n)
    fl = np.empty(n, np.uint8)
    L = lib()
    _par(n, lambda s, e: L.tfo_ew(_ptr(prog_a), prog_a.shape[0], hp, lp, len(his), s, e,
                                  _ptr(z0), _ptr(z1), _ptr(fl), mode, tau, m), threads=threads)
    return z0, z1, fl


def ew_plain(prog, his, threads=None):
    prog_a = np.ascontiguousarray(np.asarray(prog, np.int32).reshape(-1, 4))
    his = [_f64(h) for h in his]
    n = his[0].size if his else 0
    hp = (ctypes.c_void_p * len(his))(*[_ptr(h) for h in his])
    out = np.empty(n)
    L = lib()
    _par(n, lambda s, e: L.tfo_ew_plain(_ptr(prog_a), prog_a.shape[0], hp, len(his), s, e,
                                        _ptr(out)), threads=threads)
    return out


def reduce_leaves(x, xl=None, y=None, yl=None, L=256, threads=None):
    """Leaf results (m x 2 array of z0, z1) of the blocked order."""
    is_dot = y is not None
    x = _f64(x)
    xl = None if xl is None else _f64(xl)
    y = None if y is None else _f64(y)
    yl = None if yl is None else _f64(yl)
    n = x.size
    m = (n + L - 1) // L
    out = np.empty((m, 2))
    lb = lib()
    _par(m, lambda s, e: lb.tfo_reduce_leaves(_ptr(x), _ptr(xl), _ptr(y), _ptr(yl), n, L,
                                              int(is_dot), s, e, _ptr(out) + 16 * s),
         chunk=max(1, _CHUNK // L), threads=threads)
    return out


def tree(nodes):
    """The bottom-up pairwise ATF1 tree over given (z0, z1) nodes."""
    nodes = np.array(nodes, np.float64).reshape(-1, 2).copy()
    a = ctypes.c_double()
    b = ctypes.c_double()
    lib().tfo_tree(_ptr(nodes), nodes.shape[0], ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def reduce(x, xl=None, y=None, yl=None, L=256, threads=None):
    """Twofold sum (y None) or dot of the arrays in the blocked order: (z0, z1)."""
    return tree(reduce_leaves(x, xl, y, yl, L, threads))


def reduce_plain(x, y=None, L=256):
    x = _f64(x)
    y = None if y is None else _f64(y)
    n = x.size
    work = np.empty(max(1, (n + L - 1) // L))
    return lib().tfo_reduce_plain(_ptr(x), _ptr(y), n, L, int(y is not None), _ptr(work))


def horner(coefs, x, mode=REL, tau=DEFAULT_TAU, m=1.0, threads=None):
    a = _f64(coefs)
    x = _f64(x)
    n = x.size
    z0 = np.empty(n)
    z1 = np.empty(n)
    fl = np.empty(n, np.uint8)
    L = lib()
    _par(n, lambda s, e: L.tfo_horner(_ptr(a), a.size - 1, _ptr(x), s, e, _ptr(z0), _ptr(z1),
                                      _ptr(fl), mode, tau, m), threads=threads)
    return z0, z1, fl


def horner_plain(coefs, x, threads=None):
    a = _f64(coefs)
    x = _f64(x)
    n = x.size
    out = np.empty(n)
    L = lib()
    _par(n, lambda s, e: L.tfo_horner_plain(_ptr(a), a.size - 1, _ptr(x), s, e, _ptr(out)),
         threads=threads)
    return out


def flags(z0, z1, mode=REL, tau=DEFAULT_TAU, m=1.0):
    z0 = np.atleast_1d(np.asarray(z0, np.float64))
    z1 = np.atleast_1d(np.asarray(z1, np.float64))
    return np.array([flag(a, b, mode, tau, m) for a, b in zip(z0, z1)], np.uint8)


# ---------------------------------------------------------- batched helpers

def dot_batched(x, xl, y, yl, offs, L=256, mode=REL, tau=DEFAULT_TAU, m=1.0, threads=None):
    """Independent dots over [offs[j], offs[j+1]): (z0[], z1[], flags[])."""
    offs = np.asarray(offs, np.int64)
    nj = offs.size - 1
    z0 = np.empty(nj)
    z1 = np.empty(nj)

    def one(j):
        a, b = int(offs[j]), int(offs[j + 1])
        z0[j], z1[j] = reduce(x[a:b], None if xl is None else xl[a:b],
                              y[a:b], None if yl is None else yl[a:b], L, threads=1)

    t = THREADS if threads is None else threads
    with ThreadPoolExecutor(t) as ex:
        list(ex.map(one, range(nj)))
    return z0, z1, flags(z0, z1, mode, tau, m)


def sum_batched(x, xl, offs, L=256, mode=REL, tau=DEFAULT_TAU, m=1.0, threads=None):
    offs = np.asarray(offs, np.int64)
    nj = offs.size - 1
    z0 = np.empty(nj)
    z1 = np.empty(nj)

    def one(j):
        a, b = int(offs[j]), int(offs[j + 1])
        z0[j], z1[j] = reduce(x[a:b], None if xl is None else xl[a:b], L=L, threads=1)

    t = THREADS if threads is None else threads
    with ThreadPoolExecutor(t) as ex:
        list(ex.map(one, range(nj)))
    return z0, z1, flags(z0, z1, mode, tau, m)


def horner_batched(coefs, coef_offs, ks, x, x_offs, mode=REL, tau=DEFAULT_TAU, m=1.0,
                   threads=None):
    """Job j: coefficients coefs[coef_offs[j] : coef_offs[j]+ks[j]+1] over
    points x[x_offs[j] : x_offs[j+1]].  Returns concatenated (z0, z1, flags)."""
    x = _f64(x)
    n = x.size
    z0 = np.empty(n)
    z1 = np.empty(n)
    fl = np.empty(n, np.uint8)
    for j in range(len(ks)):
        a = coefs[coef_offs[j]: coef_offs[j] + ks[j] + 1]
        s, e = int(x_offs[j]), int(x_offs[j + 1])
        z0[s:e], z1[s:e], fl[s:e] = horner(a, x[s:e], mode, tau, m, threads)
    return z0, z1, fl


# ------------------------------------------------------------ binary32 basis

STICKY = 4           # flag mode bit: OR the flags of every intermediate result (R12)
DEFAULT_TAU32 = 2.0 ** -18


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _pair32(fn, *args):
    a, b = ctypes.c_float(), ctypes.c_float()
    fn(*args, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def two_sum32(a, b): return _pair32(lib().tfof_two_sum, a, b)
def two_diff32(a, b): return _pair32(lib().tfof_two_diff, a, b)
def two_prod32(a, b): return _pair32(lib().tfof_two_prod, a, b)
def div_rem32(a, b): return _pair32(lib().tfof_div_rem, a, b)
def sqrt_rem32(a): return _pair32(lib().tfof_sqrt_rem, a)
def fast_two_sum32(a, b): return _pair32(lib().tfof_fast_two_sum, a, b)


def op32(code, x, y=None):
    """One binary32 twofold op (operands as in op()); returns (z0, z1) as floats
    holding binary32 values."""
    def split(v):
        if v is None:
            return 0.0, 0.0, 1
        if isinstance(v, tuple):
            return float(v[0]), float(v[1]), 0
        return float(v), 0.0, 1
    x0, x1, xd = split(x)
    y0, y1, yd = split(y)
    return _pair32(lib().tfof_op, code, x0, x1, xd, y0, y1, yd)


def flag32(z0, z1, mode=REL, tau=DEFAULT_TAU32, m=1.0):
    return int(lib().tfof_flag(z0, z1, mode, tau, m))


def ew32(prog, inputs, mode=REL, tau=DEFAULT_TAU32, m=1.0, threads=None):
    """binary32 twofold program (inputs: (hi, lo-or-None) float32 arrays)."""
    prog_a = np.ascontiguousarray(np.asarray(prog, np.int32).reshape(-1, 4))
    his = [_f32(h) for h, _ in inputs]
    los = [None if lo is None else _f32(lo) for _, lo in inputs]
    n = his[0].size if his else 0
    hp = (ctypes.c_void_p * len(his))(*[_ptr(h) for h in his])
    lp = (ctypes.c_void_p * len(los))(*[_ptr(lo) for lo in los])
    z0 = np.empty(n, np.float32)
    z1 = np.empty(n, np.float32)
    fl = np.empty(n, np.uint8)
    L = lib()
    _par(n, lambda s, e: L.tfof_ew(_ptr(prog_a), prog_a.shape[0], hp, lp, len(his), s, e, _ptr(z0), _ptr(z1),
                                   _ptr(fl), mode, tau, m), threads=threads)
    return z0, z1, fl


def ew32_plain(prog, his, threads=None):
    prog_a = np.ascontiguousarray(np.asarray(prog, np.int32).reshape(-1, 4))
    his = [_f32(h) for h in his]
    n = his[0].size if his else 0
    hp = (ctypes.c_void_p * len(his))(*[_ptr(h) for h in his])
    out = np.empty(n, np.float32)
    L = lib()
    _par(n, lambda s, e: L.tfof_ew_plain(_ptr(prog_a), prog_a.shape[0], hp, len(his), s, e, _ptr(out)),
         threads=threads)
    return out


def reduce_sum32(x, xl=None, L=256):
    """binary32 twofold sum in the blocked pairwise order (R8)."""
    x = _f32(x)
    xl = None if xl is None else _f32(xl)
    return _pair32(lib().tfof_reduce_sum, _ptr(x), _ptr(xl), x.size, L)


def reduce32(x, xl=None, y=None, yl=None, L=256):
    """binary32 twofold sum (y None) or dot in the blocked pairwise order (R8)."""
    x = _f32(x)
    xl = None if xl is None else _f32(xl)
    y = None if y is None else _f32(y)
    yl = None if yl is None else _f32(yl)
    return _pair32(lib().tfof_reduce, _ptr(x), _ptr(xl), _ptr(y), _ptr(yl), x.size, L, int(y is not None))


def reduce32_plain(x, y=None, L=256):
    """Plain binary32 twin of reduce32 (the same leaves and tree)."""
    x = _f32(x)
    y = None if y is None else _f32(y)
    return lib().tfof_reduce_plain(_ptr(x), _ptr(y), x.size, L, int(y is not None))
