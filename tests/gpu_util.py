"""Helpers for the GPU parity tests: device transfer and bitwise comparison
with NaNs canonicalised (the one allowed difference: NaN payloads)."""
import numpy as np

from tests.fp import canon


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    return t.detach().cpu().numpy()


def assert_bits(gpu, ref, what="", idx=None):
    g = canon(host(gpu) if not isinstance(gpu, np.ndarray) else gpu)
    r = canon(ref)
    if idx is not None:
        g = g[idx]
    if not np.array_equal(g, r):
        bad = np.nonzero(g != r)[0]
        i = bad[0]
        raise AssertionError(f"{what}: {bad.size} mismatches, first at {i}: "
                             f"gpu={g[i]:#018x} oracle={r[i]:#018x}")


def assert_flags(gpu, ref, what="", idx=None):
    g = host(gpu) if not isinstance(gpu, np.ndarray) else gpu
    if idx is not None:
        g = g[idx]
    if not np.array_equal(g, ref):
        bad = np.nonzero(g != ref)[0]
        raise AssertionError(f"{what}: {bad.size} flag mismatches, first at {bad[0]}: "
                             f"gpu={g[bad[0]]} oracle={ref[bad[0]]}")


SPECIAL = np.array([0.0, -0.0, 1.0, -1.0, 2.0, 0.5, 3.0, -7.25, 0.1, -1e-300, 1e300, -1e300,
                    2.0 ** -1074, -(2.0 ** -1074), 2.0 ** -1022, 2.2250738585072009e-308,
                    1.7976931348623157e308, -1.7976931348623157e308, 1.0 + 2.0 ** -52,
                    1.0 - 2.0 ** -53, np.inf, -np.inf, np.nan, 4.0, 1e-160, 3.0e155])
