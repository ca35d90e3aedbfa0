"""GB300 twofold arithmetic: Python binding of libtwofold.so.

Twofold fast arithmetic (Latkin, arXiv:1401.6235) carries z ~ z0 + z1: z0 is
the plain IEEE binary64 result, z1 estimates its error, and a per-result
flag byte signals when z1 is large relative to z0.  All arithmetic runs in
the CUDA kernels of ``libtwofold.so`` (C ABI declared in include/twofold.h);
this module only marshals torch tensors (device memory, streams) into
pointers and sizes.  There is no CPU fallback: importing works without a
GPU, but every call needs the built library and CUDA tensors (the
elementwise calls also take pinned host tensors that the device maps, whose
bytes the kernels then move across the host link themselves).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtwofold.so")

TF_OK, TF_EINVAL, TF_ENOSPC, TF_ECUDA, TF_ETIMEOUT, TF_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
ADD, SUB, MUL, DIV, SQRT = 1, 2, 3, 4, 5
PADD, PSUB, PMUL, PDIV, PSQRT = 6, 7, 8, 9, 10      # coupled (Dekker emulation) operations
PANIC, NONFINITE = 1, 2
PANIC_REL, PANIC_ULP, PANIC_STICKY = 0, 1, 4
KIND_SUM, KIND_DOT = 1, 2
MAX_PROG, MAX_INPUTS, MAX_REGS = 32, 12, 32

#: the elementwise chain z = sqrt((a*b + c)/d) over inputs a, b, c, d (registers 0..3)
CHAIN_SQRT_MAD_DIV = [(MUL, 4, 0, 1), (ADD, 5, 4, 2), (DIV, 6, 5, 3), (SQRT, 7, 6, 6)]


class TwofoldError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} ({status})")


class tf_in(ctypes.Structure):
    _fields_ = [("hi", ctypes.c_void_p), ("lo", ctypes.c_void_p)]


class tf_out(ctypes.Structure):
    _fields_ = [("hi", ctypes.c_void_p), ("lo", ctypes.c_void_p), ("flags", ctypes.c_void_p)]


class tf_in_f32(ctypes.Structure):
    _fields_ = [("hi", ctypes.c_void_p), ("lo", ctypes.c_void_p)]


class tf_out_f32(ctypes.Structure):
    _fields_ = [("hi", ctypes.c_void_p), ("lo", ctypes.c_void_p), ("flags", ctypes.c_void_p)]


class tf_params(ctypes.Structure):
    _fields_ = [("panic_mode", ctypes.c_int32), ("leaf", ctypes.c_int32),
                ("panic_tau", ctypes.c_double), ("panic_ulps", ctypes.c_double)]


class tf_job(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("k", ctypes.c_int32), ("n", ctypes.c_int64), ("x", tf_in),
                ("y", tf_in), ("coefs", ctypes.c_void_p), ("out", tf_out)]


class tf_batch_config(ctypes.Structure):
    _fields_ = [("leaves_per_item", ctypes.c_int32), ("points_per_item", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32)]


class tf_batch_plan(ctypes.Structure):
    _fields_ = [("opaque", ctypes.c_int64 * 16)]


class tf_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("k", ctypes.c_int32), ("n", ctypes.c_int64),
                ("inp", ctypes.c_void_p * 8), ("coefs", ctypes.c_void_p), ("prog", ctypes.c_void_p),
                ("nprog", ctypes.c_int32), ("nin", ctypes.c_int32), ("out_hi", ctypes.c_void_p),
                ("out_lo", ctypes.c_void_p), ("out_flags", ctypes.c_void_p)]


class tf_request_info(ctypes.Structure):
    _fields_ = [("submitted_ns", ctypes.c_int64), ("admitted_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64),
                ("status", ctypes.c_int32), ("batch_jobs", ctypes.c_int32)]


class tf_server_stats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("failed", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("batched_jobs", ctypes.c_int64), ("arena_bytes", ctypes.c_int64), ("peak_bytes", ctypes.c_int64),
                ("pending", ctypes.c_int64), ("max_inflight", ctypes.c_int32), ("inflight", ctypes.c_int32)]


JOB_SUM, JOB_DOT, JOB_HORNER, JOB_EW = 1, 2, 3, 4


def params(panic_mode: int = PANIC_REL, leaf: int = 256, panic_tau: float = 2.0 ** -40,
           panic_ulps: float = 4096.0) -> tf_params:
    return tf_params(panic_mode, leaf, panic_tau, panic_ulps)


# Every symbol the header declares, with its ctypes signature.
_P, _I32, _I64, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
_IN, _OUT, _PP = tf_in, tf_out, ctypes.POINTER(tf_params)
SIGNATURES = {
    "twofold_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "twofold_version": ([], ctypes.c_int),
    "twofold_host_mapped": ([_P], ctypes.c_int),
    "twofold_ew": ([_P, _I32, _P, _I32, _I64, _OUT, _PP, _P], ctypes.c_int),
    "plain_ew": ([_P, _I32, _P, _I32, _I64, _P, _P], ctypes.c_int),
    "plain_arith": ([_I32], ctypes.c_int),
    "twofold_ew_f32": ([_P, _I32, _P, _I32, _I64, tf_out_f32, _PP, _P], ctypes.c_int),
    "twofold_ew_jit": ([_I32, ctypes.POINTER(_I64), ctypes.POINTER(_I64)], ctypes.c_int),
    "plain_ew_f32": ([_P, _I32, _P, _I32, _I64, _P, _P], ctypes.c_int),
    "twofold_sum_f32": ([tf_in_f32, _I64, tf_out_f32, _PP, _P, _SZ, _P], ctypes.c_int),
    "twofold_dot_f32": ([tf_in_f32, tf_in_f32, _I64, tf_out_f32, _PP, _P, _SZ, _P], ctypes.c_int),
    "plain_sum_f32": ([_P, _I64, _P, _PP, _P, _SZ, _P], ctypes.c_int),
    "plain_dot_f32": ([_P, _P, _I64, _P, _PP, _P, _SZ, _P], ctypes.c_int),
    "twofold_workspace_bytes": ([_I32, _I64, _I32, _PP], _SZ),
    "twofold_sum": ([_IN, _I64, _OUT, _PP, _P, _SZ, _P], ctypes.c_int),
    "twofold_dot": ([_IN, _IN, _I64, _OUT, _PP, _P, _SZ, _P], ctypes.c_int),
    "twofold_sum_batched": ([_IN, _P, _I32, _OUT, _PP, _P, _SZ, _P], ctypes.c_int),
    "twofold_dot_batched": ([_IN, _IN, _P, _I32, _OUT, _PP, _P, _SZ, _P], ctypes.c_int),
    "plain_sum": ([_P, _I64, _P, _PP, _P, _SZ, _P], ctypes.c_int),
    "plain_dot": ([_P, _P, _I64, _P, _PP, _P, _SZ, _P], ctypes.c_int),
    "plain_dot_batched": ([_P, _P, _P, _I32, _P, _PP, _P, _SZ, _P], ctypes.c_int),
    "twofold_dot_noalloc": ([_IN, _IN, _I64, _OUT, _PP, _P], ctypes.c_int),
    "twofold_combine": ([_P, _P, _I64, _OUT, _PP, _P, _SZ, _P], ctypes.c_int),
    "twofold_horner": ([_P, _I32, _P, _I64, _OUT, _PP, _P], ctypes.c_int),
    "twofold_horner_workspace_bytes": ([_I32], _SZ),
    "twofold_horner_batched": ([_P, _P, _P, _I32, _P, _P, _OUT, _PP, _P, _SZ, _P], ctypes.c_int),
    "plain_horner": ([_P, _I32, _P, _I64, _P, _P], ctypes.c_int),
    "plain_horner_batched": ([_P, _P, _P, _I32, _P, _P, _P, _P, _SZ, _P], ctypes.c_int),
    "twofold_batch_workspace_bytes": ([_P, _I32, _PP, ctypes.POINTER(tf_batch_config)], _SZ),
    "twofold_batch_prepare": ([_P, _I32, _PP, ctypes.POINTER(tf_batch_config), _P, _SZ,
                               ctypes.POINTER(tf_batch_plan), _P], ctypes.c_int),
    "twofold_batch_launch": ([ctypes.POINTER(tf_batch_plan), _P], ctypes.c_int),
    "twofold_batch": ([_P, _I32, _PP, ctypes.POINTER(tf_batch_config), _P, _SZ, _P], ctypes.c_int),
    "twofold_server_create": ([_SZ, _I32, _PP, ctypes.POINTER(tf_batch_config), ctypes.POINTER(_P)], ctypes.c_int),
    "twofold_server_submit": ([_P, ctypes.POINTER(tf_request), ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "twofold_server_wait": ([_P, ctypes.c_uint64, _I32, ctypes.POINTER(tf_request_info)], ctypes.c_int),
    "twofold_server_stats": ([_P, ctypes.POINTER(tf_server_stats)], ctypes.c_int),
    "twofold_server_destroy": ([_P], ctypes.c_int),
    "twofold_server_inject_failures": ([_P, _I32], ctypes.c_int),
    "twofold_pipe_probe": ([_I32, _I64, _I32, _I32, _P, _P], ctypes.c_int),
    "twofold_wait_timeouts": ([ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "twofold_inject_pair_drop": ([_I32], ctypes.c_int),
}

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library.  Raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run __graft_entry__.build() "
                               "(the twofold path has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().twofold_strerror(status).decode()


def _check(status: int, where: str) -> None:
    if status != TF_OK:
        raise TwofoldError(status, where)


# ------------------------------------------------------------ marshalling

def _torch():
    import torch
    return torch


def _dev(t, name="tensor", host_ok=False):
    """Device pointer of a contiguous CUDA float64/uint8 tensor (or None).
    With host_ok, a pinned host tensor that the device maps at the same
    address is accepted too (the kernels access it across the host link)."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.is_cuda:
        return t.data_ptr()
    if host_ok and t.is_pinned() and lib().twofold_host_mapped(ctypes.c_void_p(t.data_ptr())) == 1:
        return t.data_ptr()
    raise ValueError(f"{name} must be a CUDA tensor{' or device-mapped pinned host tensor' if host_ok else ''} "
                     "(the twofold path has no CPU fallback)")


def _stream(stream):
    torch = _torch()
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _pp(p):
    return None if p is None else ctypes.byref(p)


_ws_cache = {}


def workspace(nbytes: int, device=None):
    """A cached uint8 CUDA workspace of at least nbytes (grown on demand).
    Calls on one stream may share it; concurrent streams need their own."""
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    buf = _ws_cache.get(dev)
    if buf is None or buf.numel() < nbytes:
        buf = torch.empty(max(nbytes, 1 << 16), dtype=torch.uint8, device=dev)
        _ws_cache[dev] = buf
    return buf


def _outputs(n, device, out):
    torch = _torch()
    if out is not None:
        return out
    if device.type == "cpu":        # host-buffer form: pinned, device-mapped outputs
        return (torch.empty(n, dtype=torch.float64).pin_memory(), torch.empty(n, dtype=torch.float64).pin_memory(),
                torch.empty(n, dtype=torch.uint8).pin_memory())
    return (torch.empty(n, dtype=torch.float64, device=device),
            torch.empty(n, dtype=torch.float64, device=device),
            torch.empty(n, dtype=torch.uint8, device=device))


def _prog_array(prog):
    a = np.ascontiguousarray(np.asarray(prog, np.int32).reshape(-1, 4))
    return a


# ------------------------------------------------------------ entry points

def twofold_ew(prog, inputs, out=None, p: tf_params | None = None, stream=None):
    """Evaluate program ``prog`` (rows (op, dst, a, b)) over twofold inputs.

    inputs: list of (hi, lo) CUDA float64 tensors, lo None for dotted input
    (or pinned host tensors that the device maps: the kernel then reads and
    writes host memory across the link).  Returns (z0, z1, flags) tensors
    (or fills ``out``)."""
    pa = _prog_array(prog)
    n = inputs[0][0].numel()
    ins = (tf_in * len(inputs))(*[tf_in(_dev(h, "hi", True), _dev(lo, "lo", True)) for h, lo in inputs])
    for h, lo in inputs:
        if h.numel() != n or (lo is not None and lo.numel() != n):
            raise ValueError("inputs must all have the same length")
    hi, lo_, fl = _outputs(n, inputs[0][0].device, out)
    o = tf_out(_dev(hi, "out hi", True), _dev(lo_, "out lo", True), _dev(fl, "flags", True))
    _check(lib().twofold_ew(pa.ctypes.data, pa.shape[0], ins, len(inputs), n, o, _pp(p),
                            _stream(stream)), "twofold_ew")
    return hi, lo_, fl


def plain_ew(prog, his, out=None, stream=None):
    torch = _torch()
    pa = _prog_array(prog)
    n = his[0].numel()
    ptrs = (ctypes.c_void_p * len(his))(*[_dev(h, "input", True) for h in his])
    if out is None:
        out = (torch.empty(n, dtype=torch.float64).pin_memory() if his[0].device.type == "cpu"
               else torch.empty(n, dtype=torch.float64, device=his[0].device))
    _check(lib().plain_ew(pa.ctypes.data, pa.shape[0], ptrs, len(his), n, _dev(out, "out", True),
                          _stream(stream)), "plain_ew")
    return out


def _outputs_f32(n, device, out):
    torch = _torch()
    if out is not None:
        return out
    if device.type == "cpu":
        return (torch.empty(n, dtype=torch.float32).pin_memory(), torch.empty(n, dtype=torch.float32).pin_memory(),
                torch.empty(n, dtype=torch.uint8).pin_memory())
    return (torch.empty(n, dtype=torch.float32, device=device), torch.empty(n, dtype=torch.float32, device=device),
            torch.empty(n, dtype=torch.uint8, device=device))


def twofold_ew_f32(prog, inputs, out=None, p: tf_params | None = None, stream=None):
    """twofold_ew over binary32 twofolds: inputs are (hi, lo) float32 tensors
    (lo None for dotted input); returns (z0, z1, flags)."""
    pa = _prog_array(prog)
    n = inputs[0][0].numel()
    for h, lo in inputs:
        if h.numel() != n or (lo is not None and lo.numel() != n):
            raise ValueError("inputs must all have the same length")
    ins = (tf_in_f32 * len(inputs))(*[tf_in_f32(_dev(h, "hi", True), _dev(lo, "lo", True)) for h, lo in inputs])
    hi, lo_, fl = _outputs_f32(n, inputs[0][0].device, out)
    o = tf_out_f32(_dev(hi, "out hi", True), _dev(lo_, "out lo", True), _dev(fl, "flags", True))
    _check(lib().twofold_ew_f32(pa.ctypes.data, pa.shape[0], ins, len(inputs), n, o, _pp(p), _stream(stream)),
           "twofold_ew_f32")
    return hi, lo_, fl


def plain_ew_f32(prog, his, out=None, stream=None):
    torch = _torch()
    pa = _prog_array(prog)
    n = his[0].numel()
    ptrs = (ctypes.c_void_p * len(his))(*[_dev(h, "input", True) for h in his])
    if out is None:
        out = (torch.empty(n, dtype=torch.float32).pin_memory() if his[0].device.type == "cpu"
               else torch.empty(n, dtype=torch.float32, device=his[0].device))
    _check(lib().plain_ew_f32(pa.ctypes.data, pa.shape[0], ptrs, len(his), n, _dev(out, "out", True),
                              _stream(stream)), "plain_ew_f32")
    return out


def _red32(kind, x, y, n, out, p, ws):
    if ws is None:
        ws = workspace(max(256, lib().twofold_workspace_bytes(kind, n, 1, _pp(p))))
    return ws


def twofold_sum_f32(x, xl=None, out=None, p: tf_params | None = None, ws=None, stream=None):
    """Twofold sum of binary32 twofolds (float32 CUDA tensors) in the blocked
    pairwise order; returns (z0, z1, flags), 1-element tensors."""
    n = x.numel()
    if xl is not None and xl.numel() != n:
        raise ValueError("x and its tails must have the same length")
    ws = _red32(KIND_SUM, x, None, n, out, p, ws)
    hi, lo, fl = _outputs_f32(1, x.device, out)
    _check(lib().twofold_sum_f32(tf_in_f32(_dev(x, "x"), _dev(xl, "xl")), n,
                                 tf_out_f32(_dev(hi), _dev(lo), _dev(fl)), _pp(p), _dev(ws), ws.numel(),
                                 _stream(stream)), "twofold_sum_f32")
    return hi, lo, fl


def twofold_dot_f32(x, y, xl=None, yl=None, out=None, p: tf_params | None = None, ws=None, stream=None):
    """Twofold dot of binary32 twofolds (float32 CUDA tensors); returns (z0, z1, flags)."""
    n = x.numel()
    if y.numel() != n or (xl is not None and xl.numel() != n) or (yl is not None and yl.numel() != n):
        raise ValueError("x, y and their tails must have the same length")
    ws = _red32(KIND_DOT, x, y, n, out, p, ws)
    hi, lo, fl = _outputs_f32(1, x.device, out)
    _check(lib().twofold_dot_f32(tf_in_f32(_dev(x, "x"), _dev(xl, "xl")), tf_in_f32(_dev(y, "y"), _dev(yl, "yl")),
                                 n, tf_out_f32(_dev(hi), _dev(lo), _dev(fl)), _pp(p), _dev(ws), ws.numel(),
                                 _stream(stream)), "twofold_dot_f32")
    return hi, lo, fl


def plain_sum_f32(x, out=None, p: tf_params | None = None, ws=None, stream=None):
    torch = _torch()
    n = x.numel()
    ws = _red32(KIND_SUM, x, None, n, out, p, ws)
    out = torch.empty(1, dtype=torch.float32, device=x.device) if out is None else out
    _check(lib().plain_sum_f32(_dev(x, "x"), n, _dev(out), _pp(p), _dev(ws), ws.numel(), _stream(stream)),
           "plain_sum_f32")
    return out


def plain_dot_f32(x, y, out=None, p: tf_params | None = None, ws=None, stream=None):
    torch = _torch()
    n = x.numel()
    if y.numel() != n:
        raise ValueError("x and y must have the same length")
    ws = _red32(KIND_DOT, x, y, n, out, p, ws)
    out = torch.empty(1, dtype=torch.float32, device=x.device) if out is None else out
    _check(lib().plain_dot_f32(_dev(x, "x"), _dev(y, "y"), n, _dev(out), _pp(p), _dev(ws), ws.numel(),
                               _stream(stream)), "plain_dot_f32")
    return out


def jit_mode(mode: int = -1):
    """Set the runtime-specialisation mode of the elementwise calls (0 off,
    1 automatic for n >= 2^20, 2 always; -1 only queries).  Returns
    (previous mode, kernels built, builds failed)."""
    b, f = ctypes.c_int64(), ctypes.c_int64()
    prev = lib().twofold_ew_jit(mode, ctypes.byref(b), ctypes.byref(f))
    if prev < 0:
        raise TwofoldError(prev, "twofold_ew_jit")
    return prev, b.value, f.value


PLAIN_NATIVE, PLAIN_INTEGER = 0, 1


def plain_arith(mode: int = -1) -> int:
    """Select the arithmetic of the plain binary64 twins: PLAIN_NATIVE
    (CUDA's operations, the initial mode) or PLAIN_INTEGER (the library's
    integer-pipe division and root in plain_ew, multiplication in
    plain_horner: the same bits); -1 only queries.  Returns the previous
    mode."""
    prev = lib().plain_arith(mode)
    if prev < 0:
        raise TwofoldError(prev, "plain_arith")
    return prev


def _red_out(njobs, device, out):
    return _outputs(njobs, device, out)


def twofold_sum(x, xl=None, out=None, p: tf_params | None = None, ws=None, stream=None):
    """Twofold sum in the blocked pairwise order; returns (z0, z1, flags),
    1-element tensors.  Inputs and outputs may be CUDA tensors or pinned host
    tensors the device maps (the kernels then cross the host link)."""
    n = x.numel()
    nb = lib().twofold_workspace_bytes(KIND_SUM, n, 1, _pp(p))
    ws = workspace(nb) if ws is None else ws
    hi, lo, fl = _red_out(1, x.device, out)
    _check(lib().twofold_sum(tf_in(_dev(x, "x", True), _dev(xl, "xl", True)), n,
                             tf_out(_dev(hi, "out", True), _dev(lo, "out", True), _dev(fl, "flags", True)),
                             _pp(p), _dev(ws), ws.numel(), _stream(stream)), "twofold_sum")
    return hi, lo, fl


def twofold_dot(x, y, xl=None, yl=None, out=None, p: tf_params | None = None, ws=None, stream=None):
    """Twofold dot (as twofold_sum: CUDA or device-mapped pinned host tensors)."""
    n = x.numel()
    if y.numel() != n:
        raise ValueError("x and y must have the same length")
    nb = lib().twofold_workspace_bytes(KIND_DOT, n, 1, _pp(p))
    ws = workspace(nb) if ws is None else ws
    hi, lo, fl = _red_out(1, x.device, out)
    _check(lib().twofold_dot(tf_in(_dev(x, "x", True), _dev(xl, "xl", True)),
                             tf_in(_dev(y, "y", True), _dev(yl, "yl", True)), n,
                             tf_out(_dev(hi, "out", True), _dev(lo, "out", True), _dev(fl, "flags", True)),
                             _pp(p), _dev(ws), ws.numel(), _stream(stream)), "twofold_dot")
    return hi, lo, fl


def twofold_combine(z0, z1, out=None, p: tf_params | None = None, ws=None, stream=None):
    """The pairwise tree over partial results (device float64 tensors of the
    same length): the end of a sum or dot split into aligned 2^k-leaf blocks."""
    m = z0.numel()
    if z1.numel() != m:
        raise ValueError("z0 and z1 must have the same length")
    ws = workspace(max(256, 2 * ((8 * m + 255) // 256 * 256))) if ws is None else ws
    hi, lo, fl = _red_out(1, z0.device, out)
    _check(lib().twofold_combine(_dev(z0), _dev(z1), m, tf_out(_dev(hi), _dev(lo), _dev(fl)), _pp(p), _dev(ws),
                                 ws.numel(), _stream(stream)), "twofold_combine")
    return hi, lo, fl


def twofold_dot_noalloc(x, y, xl=None, yl=None, out=None, p: tf_params | None = None, stream=None):
    """twofold_dot without a workspace: the library's static device scratch
    holds the partials (for callers that cannot allocate at the call).
    Calls that overlap on the GPU share that scratch and race."""
    n = x.numel()
    if y.numel() != n:
        raise ValueError("x and y must have the same length")
    hi, lo, fl = _red_out(1, x.device, out)
    _check(lib().twofold_dot_noalloc(tf_in(_dev(x), _dev(xl)), tf_in(_dev(y), _dev(yl)), n,
                                     tf_out(_dev(hi), _dev(lo), _dev(fl)), _pp(p), _stream(stream)),
           "twofold_dot_noalloc")
    return hi, lo, fl


def _offs(offs):
    a = np.ascontiguousarray(np.asarray(offs, np.int64))
    return a, a.size - 1


def twofold_sum_batched(x, offs, xl=None, out=None, p: tf_params | None = None, ws=None, stream=None):
    oa, nj = _offs(offs)
    nb = lib().twofold_workspace_bytes(KIND_SUM, int(oa[-1]), nj, _pp(p))
    ws = workspace(nb) if ws is None else ws
    hi, lo, fl = _red_out(nj, x.device, out)
    _check(lib().twofold_sum_batched(tf_in(_dev(x), _dev(xl)), oa.ctypes.data, nj,
                                     tf_out(_dev(hi), _dev(lo), _dev(fl)), _pp(p), _dev(ws), ws.numel(),
                                     _stream(stream)), "twofold_sum_batched")
    return hi, lo, fl


def twofold_dot_batched(x, y, offs, xl=None, yl=None, out=None, p: tf_params | None = None, ws=None,
                        stream=None):
    oa, nj = _offs(offs)
    nb = lib().twofold_workspace_bytes(KIND_DOT, int(oa[-1]), nj, _pp(p))
    ws = workspace(nb) if ws is None else ws
    hi, lo, fl = _red_out(nj, x.device, out)
    _check(lib().twofold_dot_batched(tf_in(_dev(x), _dev(xl)), tf_in(_dev(y), _dev(yl)), oa.ctypes.data,
                                     nj, tf_out(_dev(hi), _dev(lo), _dev(fl)), _pp(p), _dev(ws),
                                     ws.numel(), _stream(stream)), "twofold_dot_batched")
    return hi, lo, fl


def plain_sum(x, out=None, p: tf_params | None = None, ws=None, stream=None):
    torch = _torch()
    n = x.numel()
    ws = workspace(lib().twofold_workspace_bytes(KIND_SUM, n, 1, _pp(p))) if ws is None else ws
    out = torch.empty(1, dtype=torch.float64, device=x.device) if out is None else out
    _check(lib().plain_sum(_dev(x), n, _dev(out), _pp(p), _dev(ws), ws.numel(), _stream(stream)),
           "plain_sum")
    return out


def plain_dot(x, y, out=None, p: tf_params | None = None, ws=None, stream=None):
    torch = _torch()
    n = x.numel()
    ws = workspace(lib().twofold_workspace_bytes(KIND_DOT, n, 1, _pp(p))) if ws is None else ws
    out = torch.empty(1, dtype=torch.float64, device=x.device) if out is None else out
    _check(lib().plain_dot(_dev(x), _dev(y), n, _dev(out), _pp(p), _dev(ws), ws.numel(),
                           _stream(stream)), "plain_dot")
    return out


def plain_dot_batched(x, y, offs, out=None, p: tf_params | None = None, ws=None, stream=None):
    torch = _torch()
    oa, nj = _offs(offs)
    ws = workspace(lib().twofold_workspace_bytes(KIND_DOT, int(oa[-1]), nj, _pp(p))) if ws is None else ws
    out = torch.empty(nj, dtype=torch.float64, device=x.device) if out is None else out
    _check(lib().plain_dot_batched(_dev(x), _dev(y), oa.ctypes.data, nj, _dev(out), _pp(p), _dev(ws),
                                   ws.numel(), _stream(stream)), "plain_dot_batched")
    return out


def twofold_horner(coef, x, out=None, p: tf_params | None = None, stream=None):
    """Twofold Horner of ascending dotted coefficients ``coef`` (CUDA float64,
    k+1 values) at points ``x`` (CUDA or device-mapped pinned host tensor);
    returns (z0, z1, flags)."""
    n = x.numel()
    hi, lo, fl = _outputs(n, x.device, out)
    _check(lib().twofold_horner(_dev(coef), coef.numel() - 1, _dev(x, "x", True), n,
                                tf_out(_dev(hi, "out", True), _dev(lo, "out", True), _dev(fl, "flags", True)),
                                _pp(p), _stream(stream)), "twofold_horner")
    return hi, lo, fl


def twofold_horner_batched(coefs, coef_offs, ks, x, x_offs, out=None, p: tf_params | None = None,
                           ws=None, stream=None):
    co = np.ascontiguousarray(np.asarray(coef_offs, np.int32))
    kk = np.ascontiguousarray(np.asarray(ks, np.int32))
    xo = np.ascontiguousarray(np.asarray(x_offs, np.int64))
    nj = kk.size
    ws = workspace(lib().twofold_horner_workspace_bytes(nj)) if ws is None else ws
    hi, lo, fl = _outputs(x.numel(), x.device, out)
    _check(lib().twofold_horner_batched(_dev(coefs), co.ctypes.data, kk.ctypes.data, nj, _dev(x, "x", True),
                                        xo.ctypes.data, tf_out(_dev(hi, "out", True), _dev(lo, "out", True),
                                                               _dev(fl, "flags", True)), _pp(p),
                                        _dev(ws), ws.numel(), _stream(stream)), "twofold_horner_batched")
    return hi, lo, fl


def plain_horner(coef, x, out=None, stream=None):
    torch = _torch()
    out = torch.empty(x.numel(), dtype=torch.float64, device=x.device) if out is None else out
    _check(lib().plain_horner(_dev(coef), coef.numel() - 1, _dev(x), x.numel(), _dev(out),
                              _stream(stream)), "plain_horner")
    return out


def plain_horner_batched(coefs, coef_offs, ks, x, x_offs, out=None, ws=None, stream=None):
    torch = _torch()
    co = np.ascontiguousarray(np.asarray(coef_offs, np.int32))
    kk = np.ascontiguousarray(np.asarray(ks, np.int32))
    xo = np.ascontiguousarray(np.asarray(x_offs, np.int64))
    nj = kk.size
    ws = workspace(lib().twofold_horner_workspace_bytes(nj)) if ws is None else ws
    out = torch.empty(x.numel(), dtype=torch.float64, device=x.device) if out is None else out
    _check(lib().plain_horner_batched(_dev(coefs), co.ctypes.data, kk.ctypes.data, nj, _dev(x),
                                      xo.ctypes.data, _dev(out), _dev(ws), ws.numel(), _stream(stream)),
           "plain_horner_batched")
    return out


# ------------------------------------------------------------ pipe-rate probes

PROBE_DADD, PROBE_DMUL, PROBE_DFMA, PROBE_FFMA = 0, 1, 2, 3
PROBE_IMAD, PROBE_SHF, PROBE_MULHI64, PROBE_MUFU, PROBE_I2F = 4, 5, 6, 7, 8
PROBE_CHAIN_LDS, PROBE_CHAIN_AHEAD, PROBE_LATENCY = 9, 10, 0x100
#: lane instructions per thread per loop iteration of a probe (8 chains x 16 rounds)
PROBE_OPS_PER_ITER = 128


def pipe_probe(op: int, iters: int, blocks: int, threads: int, rec=None, stream=None):
    """One launch of the pipe-rate probe (measurement only): returns the
    int64 CUDA tensor of 4 stamps per CTA (SM id, start clock, end clock,
    digest)."""
    torch = _torch()
    rec = torch.empty(4 * blocks, dtype=torch.int64, device="cuda") if rec is None else rec
    _check(lib().twofold_pipe_probe(op, iters, blocks, threads, _dev(rec), _stream(stream)), "twofold_pipe_probe")
    return rec


def wait_timeouts() -> int:
    """Bounded device-side waits that ran out on the current device (see
    twofold_wait_timeouts); 0 in a healthy run."""
    c = ctypes.c_uint64()
    _check(lib().twofold_wait_timeouts(ctypes.byref(c)), "twofold_wait_timeouts")
    return int(c.value)


def inject_pair_drop(chunk: int) -> int:
    """Failure injection for tests (twofold_inject_pair_drop): the latency
    schedule's producers skip chunk `chunk` (-1: off); returns the previous
    setting."""
    r = lib().twofold_inject_pair_drop(chunk)
    if r < -1:
        _check(r, "twofold_inject_pair_drop")
    return r
