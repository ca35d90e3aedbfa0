"""The benchmark's output contract on the CPU: the JSON line built from a
workload's result carries every key the contract asks for, with the
roofline arithmetic of both bounds; and the reference arm (the CPU oracle
on a bounded sample) prints its line and exits 0."""
import json
import os
import subprocess
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "e2e", "gpu_launches", "clocks", "roofline"}


def fake(bound):
    res = {"metric": "m", "value": 2.0, "unit": "GB/s", "ms_per_step": 4.0, "config": {"workload": "w"},
           "e2e": {"value": 1.0, "unit": "GB/s", "h2d_bytes_per_step": 8, "d2h_bytes_per_step": 8},
           "gpu_launches": 3, "clocks": {"sm_mhz": 2000.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 9},
           "_kernel_ms": 4.0, "_ops": 8e9, "_bytes": 4e9, "_units": 1 << 28,
           "_sample": lambda: {"value": 1.0, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": "s"}}
    if bound == "hbm":
        res["_bound"] = "hbm"
        res["_dtype"] = "f32"
    return res


RATES = {"dadd": 1.7, "shf": 64.0, "imad": 64.0, "ffma": 128.0}


@pytest.mark.parametrize("bound", ["alu", "hbm"])
def test_line_has_the_contract_keys(bound):
    args = types.SimpleNamespace(workload="ew_chain", steps=3, warmup=3, no_cpu_baseline=False)
    line = bench.build_line(fake(bound), args, 1, 152, 6784.5, "measured", RATES)
    assert KEYS <= set(line), KEYS - set(line)
    assert "cpu_baseline" in line and line["cpu_baseline"]["kind"] == "oracle"
    r = line["roofline"]
    assert r["bound"] == bound and set(r) >= {"achieved", "peak", "unit", "frac", "traffic"}
    if bound == "alu":
        # the binding pipe: the largest floor of the chain kernel's committed per-element counts
        per, _, src = bench.PIPE_LOAD["ew_chain"]
        assert os.path.exists(os.path.join(ROOT, src))
        units, hz = 1 << 28, 152 * 2000.0 * 1e6
        floors = {p: per[p] * units / (RATES[bench.PIPE_PROBE[p]] * hz) * 1e3 for p in per}
        assert r["pipe"] == max(floors, key=floors.get)
        assert r["floors_ms"] == pytest.approx(floors)
        assert r["peak"] == pytest.approx(RATES[bench.PIPE_PROBE[r["pipe"]]] * hz / 1e12)
        assert r["achieved"] == pytest.approx(per[r["pipe"]] * units / 4e-3 / 1e12)
        assert r["frac"] == pytest.approx(max(floors.values()) / 4.0)
        a = r["fp64_algorithmic"]
        assert a["frac"] == pytest.approx(bench.ALG_FP64["ew_chain"] * units / 4e-3 / (1.7 * hz))
    else:
        assert r["achieved"] == pytest.approx(4e9 / 4e-3 / 1e9) and r["peak"] == 6784.5
        assert line["dtype"] == "f32"
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert not any(k.startswith("_") for k in line)
    json.dumps(line)


def test_reference_arm_prints_its_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--n", "65536"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_peak_measurement_line_has_no_roofline():
    """The pipe-rate workload measures the peaks themselves: its line keeps
    the contract's keys with a null roofline and no HBM block."""
    res = fake("alu")
    res.update({"_kernel_ms": 0.0, "_ops": 0, "_bytes": 0, "_units": None, "_sample": None, "_bound": "none",
                "e2e": None})
    args = types.SimpleNamespace(workload="fp64_peak", steps=3, warmup=3, no_cpu_baseline=False)
    line = bench.build_line(res, args, 1, 152, 6784.5, "measured")
    assert KEYS <= set(line) and line["roofline"] is None and "hbm" not in line
    json.dumps(line)


def test_probe_rate_from_stamps():
    """Lane operations per SM clock from per-CTA stamps: per SM, the CTAs'
    operations over the first start to the last end; median over SMs."""
    import numpy as np
    threads, iters = 256, 10
    ops = threads * iters * 128
    st = np.array([[0, 100, 100 + ops // 2, 0], [0, 150, 100 + ops, 0],       # SM 0: 2 CTAs over `ops` clocks
                   [3, 0, ops, 0],                                              # SM 3: 1 CTA over `ops` clocks
                   [5, 10, 10 + ops // 4, 0]], np.int64)                        # SM 5: 1 CTA over ops/4 clocks
    r = bench.probe_rate(st, threads, iters)
    assert r["sms"] == 3 and r["min"] == pytest.approx(1.0) and r["max"] == pytest.approx(4.0)
    assert r["op_per_clk_sm"] == pytest.approx(2.0)
