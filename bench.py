"""Benchmark of the twofold hot path on GB300.

Default workload: the elementwise twofold chain z = sqrt((a*b + c)/d) over
n = 2^28 twofolds (a, b, c: random sign x 10^U(-3,3), d: 10^U(-3,3), tails
uniform in +-1/2 ulp), one twofold_ew launch per step, beside its plain
binary64 twin with CUDA's division and root (slowdown_vs_plain) and with
the library's integer-pipe ones (slowdown_vs_plain_int).  Other workloads
(--workload): dot (one n = 65536 dot), cond_dots (4096 ill-conditioned dots
of 2^16 in one batched launch), horner (k in {5,10,20,30} x 2^24 points in
one batched launch, and as a persistent batch), batch_mix (2000 uneven
jobs in one persistent launch vs one call each), serve (the request server
under Poisson arrivals), ew_chain_f32 / dot_f32 (the binary32 basis),
criteria (the paper's cached / uncached slowdown criteria) and dot_sharded
(one dot split over the ranks).

Prints ONE JSON line on rank 0.  `value` is whole-job throughput with
inputs resident in HBM; `e2e` is the same metric through the public API
with HOST buffers every step: either copied in and out around the call, or
pinned host buffers the device maps, which the kernel reads and writes
across the host link itself (`e2e.how` says which).  `--impl reference`
times the CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0
# The binary64 kernels are bound by the SM's execution pipes, not by HBM.
# Their roofline: per pipe, the lane-instruction slots a unit of work takes
# on that pipe (warp instructions executed on it x 32 / units, from one ncu
# capture of the kernel, named beside) over the pipe's rate, which bench.py
# measures live with the pipe-rate probes (lane ops per SM clock, the probe
# named in PIPE_PROBE) times SMs times the sampled SM clock.  The pipe with
# the largest floor is the bound; frac = that floor / the measured time.
# "issue" counts every issued instruction against the issue limit (the FP32
# fma probe, which runs at the issue rate).
PIPE_PROBE = {"fp64": "dadd", "alu": "shf", "fmaheavy": "imad", "issue": "ffma"}
PIPE_LOAD = {
    "ew_chain": ({"fp64": 21.00, "alu": 612.04, "fmaheavy": 286.65, "issue": 1106.22}, "element",
                 "profiles/tf_jit_ew_chain_n2e28.md"),
    "horner": ({"fp64": 4.000, "alu": 129.40, "fmaheavy": 36.64, "issue": 194.72}, "point step",
               "profiles/horner_kernel_k5-30_2e24.md"),
    "cond_dots": ({"fp64": 3.607, "alu": 128.06, "fmaheavy": 35.17, "issue": 188.85}, "element",
                  "profiles/reduce_blocks_cond_dots_4096x2e16.md"),
}

# Algorithmic unit costs (bytes and basic FP64 operations per result).
EW_BYTES = 8 * 8 + 2 * 8 + 1            # 4 twofold inputs, twofold output, flag byte
EW_PLAIN_BYTES = 4 * 8 + 8
EW32_BYTES = 8 * 4 + 2 * 4 + 1          # the binary32 chain: 4 twofold inputs, twofold output, flag
EW32_PLAIN_BYTES = 4 * 4 + 4
# basic ops of the chain: MTF1 8, ATF1 8, DTF1 6 (2 div), RTF1 20 (2 sqrt, 1 div), flag 1
EW_OPS = 8 + 8 + 6 + 20 + 1
DOT_BYTES = 16                           # dotted x_i, y_i
DOT_OPS = 2 + 8                          # Two-Product + ATF1 per element
HORNER_BYTES = 8 + 16 + 1                # x in, twofold out, flag
HORNER_OPS_PER_STEP = 4 + 7              # MTF1.1 + ATF1.1


# DRAM bytes per launch of the timed kernel from one ncu capture (summaries in
# profiles/), scaled by the units a launch processes; None where the kernel
# changed after its counters were taken.
TRAFFIC_PER_UNIT = {
    "ew_chain": ((284.63e6 + 87.02e6) * 64 / (1 << 28), "profiles/tf_jit_ew_chain_n2e28.md"),
    "ew_chain_f32": ((536.909e6 + 128.039e6) * 16 / (1 << 28), "profiles/tf_jit_ew_chain_f32_n2e28.md"),
    "horner": (784.21e6 * 2 / (1 << 26), "profiles/horner_kernel_k5-30_2e24.md"),
    "cond_dots": ((268.59e6 + 3.30e6) / (1 << 24), "profiles/reduce_blocks_cond_dots_4096x2e16.md"),
    "dot": (1.109248e6 / 65536, "profiles/reduce_lat_pair_dot_n65536.md"),
    "dot_f32": ((536.895e6 + 3.582e6) / (1 << 26), "profiles/red32_blocks_dot_f32_2e28.md"),
}

# FP64 instructions per unit that the paper's algorithms themselves need
# (the chain: MTF1 3 add + 3 mul, ATF1 3 add, DTF1 2 add + 1 fma, RTF1 5 add;
# a Horner step: MTF1.1 1 mul + 1 add, ATF1.1 2 add; a dotted dot element:
# ATF1 3 add, the Two-Product on the integer pipes), the rest of their
# arithmetic running on the integer pipes with the same bits.
ALG_FP64 = {"ew_chain": 17, "horner": 4, "cond_dots": 3, "dot": 3}   # (the kernels issue a few more, see PIPE_LOAD)


def measured_peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during timing."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        clk, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                clk.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not clk:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(clk), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(clk)}


# ----------------------------------------------------------------- timing

def time_steps(step, steps, warmup, dist_on):
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if dist_on:
        import torch.distributed as dist
        dist.barrier()
    s = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(steps):
        step()
    e1.record(s)
    torch.cuda.synchronize()
    if dist_on:
        import torch.distributed as dist
        dist.barrier()
    ms = e0.elapsed_time(e1)
    if dist_on:
        from paper_1401_6235_gb300.dist import max_over_ranks
        ms = max_over_ranks(ms, device="cuda")
    return ms


def graph_throughput(call, reps):
    """`reps` back-to-back calls captured in one CUDA graph, replayed 3 times:
    mean microseconds per call and calls per second (launch cost removed)."""
    import torch
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(3):
            call()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(reps):
            call()
    g.replay()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / (3 * reps)
    return {"calls_in_graph": reps, "replays": 3, "us_per_call": us, "calls_per_s": 1e6 / us}


# ------------------------------------------------------------- pipe rates

PROBES = {"dadd": 0, "dmul": 1, "dfma": 2, "ffma": 3, "imad": 4, "shf": 5, "mulhi64": 6, "mufu": 7, "i2f": 8}


def probe_rate(stamps, threads, iters, ops_per_iter=128):
    """Lane operations per SM clock from the probe's per-CTA stamps (rows of
    SM id, start clock, end clock, digest): per SM, the operations of its
    CTAs over the span from their first start to their last end; returns the
    median over SMs, the spread and the number of SMs seen."""
    st = np.asarray(stamps, np.int64).reshape(-1, 4)
    rates = []
    for s in np.unique(st[:, 0]):
        r = st[st[:, 0] == s]
        span = int(r[:, 2].max() - r[:, 1].min())
        if span > 0:
            rates.append(len(r) * threads * iters * ops_per_iter / span)
    rates = np.asarray(rates)
    return {"op_per_clk_sm": float(np.median(rates)), "min": float(rates.min()), "max": float(rates.max()),
            "sms": int(rates.size)}


def measure_pipes(names=tuple(PROBES), target_cycles=4e6, blocks_per_sm=4, threads=256, reps=3):
    """Issue rate of each probed instruction kind on this GPU (lane ops per
    SM clock, the best of `reps` launches of ~target_cycles SM clocks; all
    CTAs resident at once)."""
    import torch
    import paper_1401_6235_gb300 as T
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = sms * blocks_per_sm
    rec = torch.empty(4 * blocks, dtype=torch.int64, device="cuda")
    out = {}
    for name in names:
        op = PROBES[name]
        T.pipe_probe(op, 4, blocks, threads, rec)                  # calibration launch
        torch.cuda.synchronize()
        cal = probe_rate(rec.cpu().numpy(), threads, 4)["op_per_clk_sm"]
        iters = max(8, int(target_cycles * cal / (blocks_per_sm * threads * T.PROBE_OPS_PER_ITER)))
        best = None
        for _ in range(reps):
            T.pipe_probe(op, iters, blocks, threads, rec)
            torch.cuda.synchronize()
            r = probe_rate(rec.cpu().numpy(), threads, iters)
            if best is None or r["op_per_clk_sm"] > best["op_per_clk_sm"]:
                best = r
        best["iters"] = iters
        out[name] = best
    return out


def measure_latencies(names=("dadd", "dmul", "dfma", "imad"), target_cycles=1e6):
    """Dependent-chain latency in SM clocks: one warp per SM runs one chain
    per thread (32 lanes over the measured lane rate)."""
    import torch
    import paper_1401_6235_gb300 as T
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    rec = torch.empty(4 * sms, dtype=torch.int64, device="cuda")
    out = {}
    for name in names:
        op = PROBES[name] | T.PROBE_LATENCY
        T.pipe_probe(op, 2, sms, 32, rec)
        torch.cuda.synchronize()
        cal = probe_rate(rec.cpu().numpy(), 32, 2)["op_per_clk_sm"]
        iters = max(4, int(target_cycles * cal / (32 * T.PROBE_OPS_PER_ITER)))
        T.pipe_probe(op, iters, sms, 32, rec)
        torch.cuda.synchronize()
        r = probe_rate(rec.cpu().numpy(), 32, iters)
        out[name] = {"cycles": 32.0 / r["op_per_clk_sm"], "iters": iters}
    # a short reduction's critical loop: one 16-byte load and two dependent
    # adds per element, in the compiler's order and in the fixed order of the
    # CTA-pair reduction's chains
    for key, form, what in (
            ("chain_lds_element", T.PROBE_CHAIN_LDS,
             "clocks per element of acc = (acc + e) + t with (e, t) loaded from shared memory"),
            ("chain_ahead_element", T.PROBE_CHAIN_AHEAD,
             "the same, loads and adds in a fixed order: the next 8 elements' loads after the first add of the 8 before")):
        op = form | T.PROBE_LATENCY
        T.pipe_probe(op, 1, sms, 32, rec)
        torch.cuda.synchronize()
        iters = max(2, int(target_cycles / (256 * 150)))
        T.pipe_probe(op, iters, sms, 32, rec)
        torch.cuda.synchronize()
        r = probe_rate(rec.cpu().numpy(), 32, iters, ops_per_iter=256)
        out[key] = {"cycles": 32.0 / r["op_per_clk_sm"], "iters": iters, "what": what}
    return out


def workload_fp64_peak(args, rank, world, dist_on):
    """The issue rates that bound the binary64 kernels, measured on this
    GPU: binary64 add / multiply / fma, binary32 fma (issue limit), integer
    multiply-add, funnel shift (integer ALU), 64-bit high multiply, root
    seed and integer-to-float conversion, each as lane operations per SM
    clock, and the same times SMs times the sampled SM clock; and the
    dependent-chain latency of binary64 add / multiply / fma and integer
    multiply-add in SM clocks."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    measure_pipes(("dadd",), target_cycles=1e6, reps=1)              # warm-up
    with ClockSampler(args.smi_index) as cs:
        t0 = time.perf_counter()
        rates = measure_pipes()
        wall = time.perf_counter() - t0
        lat = measure_latencies()
    clk = cs.summary()
    mhz = clk["sm_mhz"] or 2070.0
    for r in rates.values():
        r["gops"] = r["op_per_clk_sm"] * sms * mhz * 1e6 / 1e9
    return {
        "metric": "FP64 pipe issue rate (binary64 add, lane ops per SM clock)",
        "value": rates["dadd"]["op_per_clk_sm"], "unit": "op/clk/SM", "ms_per_step": wall * 1e3 / len(rates),
        "pipes": rates, "latency_cycles": lat, "sms": sms,
        "config": {"workload": "pipe-rate probes: 8 independent register chains per thread, 128 instructions per "
                               "loop iteration, 4 CTAs x 256 threads per SM, best of 3 launches of ~4e6 SM clocks",
                   "l2": "registers only (no memory traffic)", "parallelism": f"replicas x{world}"},
        "e2e": None, "gpu_launches": len(PROBES) * 4 + 1, "clocks": clk,
        "_kernel_ms": 0.0, "_ops": 0, "_bytes": 0, "_units": None, "_sample": None, "_bound": "none",
    }


# --------------------------------------------------------------- workloads

def workload_ew(args, rank, world, dist_on):
    import torch
    import paper_1401_6235_gb300 as T
    import synth
    n = args.n or (1 << 28)
    prog = T.CHAIN_SQRT_MAD_DIV
    pin = lambda m: torch.empty(m, dtype=torch.float64).pin_memory().numpy()
    host = synth.ew_chain(n, seed=rank, pinned=pin)
    keys = ["a0", "a1", "b0", "b1", "c0", "c1", "d0", "d1"]
    g = {k: torch.from_numpy(host[k]).to("cuda", non_blocking=True) for k in keys}
    ins = [(g["a0"], g["a1"]), (g["b0"], g["b1"]), (g["c0"], g["c1"]), (g["d0"], g["d1"])]
    out = (torch.empty(n, dtype=torch.float64, device="cuda"), torch.empty(n, dtype=torch.float64, device="cuda"),
           torch.empty(n, dtype=torch.uint8, device="cuda"))
    pout = torch.empty(n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()

    def step():
        T.twofold_ew(prog, ins, out=out)

    def pstep():
        T.plain_ew(prog, [h for h, _ in ins], out=pout)

    with ClockSampler(args.smi_index) as cs:
        ms = time_steps(step, args.steps, args.warmup, dist_on)
    plain_ms = time_steps(pstep, args.steps, args.warmup, dist_on)
    # the plain twin again with the integer-pipe division and root that the
    # twofold kernel uses (the same bits): the fastest plain chain here
    plain_int = time_plain_integer(T, pstep, args, dist_on)

    # end to end through the public call with HOST buffers: the inputs live in
    # pinned host memory that the device maps, and the chain kernel reads them
    # and writes z0, z1 and flags back across the host link every step (the
    # link's copy engines peak lower than these direct accesses here, and a
    # chunked copy pipeline measured slower)
    del pout
    hins = [(torch.from_numpy(host[k + "0"]), torch.from_numpy(host[k + "1"])) for k in "abcd"]
    hout = (torch.empty(n, dtype=torch.float64).pin_memory(), torch.empty(n, dtype=torch.float64).pin_memory(),
            torch.empty(n, dtype=torch.uint8).pin_memory())

    def e2e_step():
        T.twofold_ew(prog, hins, out=hout)

    e2e_steps = max(3, args.steps // 4)
    e2e_ms = time_steps(e2e_step, e2e_steps, max(1, args.warmup // 2), dist_on)

    per = ms / args.steps
    gbs = EW_BYTES * n * world / (per * 1e-3) / 1e9
    res = {
        "metric": "twofold GB/s (elementwise chain sqrt((a*b+c)/d), 81 B/elt)",
        "value": gbs, "unit": "GB/s", "ms_per_step": per,
        "plain_ms_per_step": plain_ms / args.steps,
        "slowdown_vs_plain": per / (plain_ms / args.steps),
        "plain_int_ms_per_step": plain_int, "slowdown_vs_plain_int": per / plain_int,
        "mega_ops": n * world / (per * 1e-3) / 1e6,
        "config": {"workload": "ew_chain sqrt((a*b+c)/d)", "n": n, "bytes_per_elt": EW_BYTES,
                   "inputs": "a,b,c sign*10^U(-3,3), d 10^U(-3,3), tails U(+-1/2 ulp), seed = rank",
                   "l2": "inputs (16 GiB) larger than L2; no flush needed",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": EW_BYTES * n * world / (e2e_ms / e2e_steps * 1e-3) / 1e9, "unit": "GB/s",
                "ms_per_step": e2e_ms / e2e_steps, "how": "pinned host inputs and outputs, device-mapped",
                "h2d_bytes_per_step": 64 * n, "d2h_bytes_per_step": 17 * n},
        "gpu_launches": args.steps,
        "clocks": cs.summary(),
        "_kernel_ms": per, "_ops": EW_OPS * n, "_bytes": EW_BYTES * n, "_units": n,
        "_sample": lambda: cpu_sample_ew(n),
    }
    return res


def cpu_sample_ew(n):
    import oracle as O
    import paper_1401_6235_gb300 as T
    import synth
    m = min(n, 1 << 26)
    d = synth.ew_chain(m, seed=0)
    ins = [(d[k + "0"], d[k + "1"]) for k in "abcd"]
    reps = 4
    t = time.perf_counter()
    for _ in range(reps):
        O.ew(T.CHAIN_SQRT_MAD_DIV, ins)
    dt = (time.perf_counter() - t) / reps
    return {"value": EW_BYTES * m / dt / 1e9, "unit": "GB/s", "cores": O.THREADS, "kind": "oracle",
            "sample": f"first {m} elements of the chain workload (seed 0), {reps} passes, {dt:.2f} s wall each "
                      f"(~{reps * dt * O.THREADS:.0f} core-seconds in all)"}


def time_plain_integer(T, call, args, dist_on):
    """The plain twin timed again with the integer-pipe routines of
    plain_arith (the same bits); returns ms per step."""
    prev = T.plain_arith(T.PLAIN_INTEGER)
    try:
        return time_steps(call, args.steps, args.warmup, dist_on) / args.steps
    finally:
        T.plain_arith(prev)


def workload_dot(args, rank, world, dist_on):
    import torch
    import paper_1401_6235_gb300 as T
    import synth
    n = args.n or 65536
    x, y = synth.dot_uniform(n, seed=0)
    gx, gy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    ws = T.workspace(T.lib().twofold_workspace_bytes(T.KIND_DOT, n, 1, None))
    out = (torch.empty(1, dtype=torch.float64, device="cuda"), torch.empty(1, dtype=torch.float64, device="cuda"),
           torch.empty(1, dtype=torch.uint8, device="cuda"))
    step = lambda: T.twofold_dot(gx, gy, out=out, ws=ws)
    with ClockSampler(args.smi_index) as cs:
        ms = time_steps(step, args.steps, args.warmup, dist_on)
    pout = torch.empty(1, dtype=torch.float64, device="cuda")
    plain_ms = time_steps(lambda: T.plain_dot(gx, gy, out=pout, ws=ws), args.steps, args.warmup, dist_on)
    hx, hy = torch.from_numpy(x).pin_memory(), torch.from_numpy(y).pin_memory()
    hres = torch.empty(3, dtype=torch.float64).pin_memory()

    def e2e_step():
        gx.copy_(hx, non_blocking=True)
        gy.copy_(hy, non_blocking=True)
        T.twofold_dot(gx, gy, out=out, ws=ws)
        hres[0:1].copy_(out[0], non_blocking=True)
        hres[1:2].copy_(out[1], non_blocking=True)

    e2e_ms = time_steps(e2e_step, args.steps, args.warmup, dist_on)
    # the same call on the pinned host buffers themselves (the device maps them;
    # the kernel reads x, y and writes the result across the host link)
    hout = (torch.empty(1, dtype=torch.float64).pin_memory(), torch.empty(1, dtype=torch.float64).pin_memory(),
            torch.empty(1, dtype=torch.uint8).pin_memory())
    mapped_ms = time_steps(lambda: T.twofold_dot(hx, hy, out=hout, ws=ws), args.steps, args.warmup, dist_on)
    graph = graph_throughput(lambda: T.twofold_dot(gx, gy, out=out, ws=ws), 1000)
    per = ms / args.steps
    return {
        "metric": "twofold dot latency (n=65536)", "value": per * 1e3, "unit": "us",
        "higher_is_better": False, "ms_per_step": per,
        "plain_ms_per_step": plain_ms / args.steps, "slowdown_vs_plain": per / (plain_ms / args.steps),
        "gbs": DOT_BYTES * n / (per * 1e-3) / 1e9,
        "config": {"workload": "dot n=65536 uniform[-1,1] seed 0, L=256", "n": n,
                   "l2": "input (1 MiB) L2-resident after warm-up (latency-bound workload)",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": min(e2e_ms, mapped_ms) / args.steps * 1e3, "unit": "us", "h2d_bytes_per_step": 16 * n,
                "d2h_bytes_per_step": 16 if e2e_ms <= mapped_ms else 17,
                "how": "copies to device buffers" if e2e_ms <= mapped_ms else "pinned host buffers, device-mapped",
                "copies_us": e2e_ms / args.steps * 1e3, "mapped_us": mapped_ms / args.steps * 1e3},
        "graph": graph,
        "latency_floor": dot_latency_floor(cs.summary().get("sm_mhz"), per * 1e3),
        "gpu_launches": 2 * args.steps, "clocks": cs.summary(),    # leaves kernel + final tree
        "_kernel_ms": per, "_ops": DOT_OPS * n, "_bytes": DOT_BYTES * n, "_units": n, "_bound": "latency",
        "_sample": lambda: cpu_sample_dot(n),
    }


def dot_latency_floor(sm_mhz, us):
    """The order's own floor for one leaf: the z1 accumulator of a 256-element
    leaf takes two dependent binary64 adds per element, 64 cycles each on this
    GPU (measured), whatever else runs in parallel."""
    mhz = sm_mhz or 2070.0
    floor = 2 * 256 * 64 / mhz
    return {"floor_us": floor, "frac": floor / us, "what": "512 dependent FP64 adds x 64 cycles at the sampled "
            "SM clock (the z1 chain of one 256-element leaf); launch, terms and tree levels come on top"}


def cpu_sample_dot(n):
    import oracle as O
    import synth
    x, y = synth.dot_uniform(n, seed=0)
    reps = 200
    t = time.perf_counter()
    for _ in range(reps):
        O.reduce(x, None, y, None)
    dt = (time.perf_counter() - t) / reps
    return {"value": dt * 1e6, "unit": "us", "cores": 1, "kind": "oracle",
            "sample": f"the whole n={n} dot, mean of {reps} runs"}


def workload_cond_dots(args, rank, world, dist_on):
    import torch
    import paper_1401_6235_gb300 as T
    import synth
    n = 1 << 16
    nj = max(1, args.n // n) if args.n else 4096
    x, y, offs, exact, cond, _ = synth.cond_dots(nj, n, seed=rank)
    gx, gy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    ws = T.workspace(T.lib().twofold_workspace_bytes(T.KIND_DOT, nj * n, nj, None))
    out = (torch.empty(nj, dtype=torch.float64, device="cuda"), torch.empty(nj, dtype=torch.float64, device="cuda"),
           torch.empty(nj, dtype=torch.uint8, device="cuda"))
    step = lambda: T.twofold_dot_batched(gx, gy, offs, out=out, ws=ws)
    with ClockSampler(args.smi_index) as cs:
        ms = time_steps(step, args.steps, args.warmup, dist_on)
    pout = torch.empty(nj, dtype=torch.float64, device="cuda")
    plain_ms = time_steps(lambda: T.plain_dot_batched(gx, gy, offs, out=pout, ws=ws), args.steps, args.warmup,
                          dist_on)
    del pout
    # end to end: the inputs copied in from pinned host memory and the
    # results read back, every step.  The jobs go in chunks over two streams,
    # so the copy of a chunk overlaps the dots of the one before (the jobs
    # are independent: the same bits as one call over all of them)
    hx, hy = torch.from_numpy(x).pin_memory(), torch.from_numpy(y).pin_memory()
    hres = tuple(torch.empty(nj, dtype=t.dtype).pin_memory() for t in out)
    offs_a = np.asarray(offs, np.int64)
    nchunk = 8 if nj % 8 == 0 else 1
    per_c = nj // nchunk
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    chunk_elems = max(int(offs_a[(c + 1) * per_c] - offs_a[c * per_c]) for c in range(nchunk))
    # one workspace per stream (T.workspace would hand both the same cached buffer)
    wss = [torch.empty(T.lib().twofold_workspace_bytes(T.KIND_DOT, chunk_elems, per_c, None), dtype=torch.uint8,
                       device="cuda") for _ in streams]

    def e2e_step():
        cur = torch.cuda.current_stream()
        for st in streams:
            st.wait_stream(cur)
        for c in range(nchunk):
            a, b = c * per_c, (c + 1) * per_c
            e0, e1 = int(offs_a[a]), int(offs_a[b])
            with torch.cuda.stream(streams[c % 2]):
                gx[e0:e1].copy_(hx[e0:e1], non_blocking=True)
                gy[e0:e1].copy_(hy[e0:e1], non_blocking=True)
                T.twofold_dot_batched(gx[e0:e1], gy[e0:e1], offs_a[a:b + 1] - e0, out=tuple(t[a:b] for t in out),
                                      ws=wss[c % 2])
                for h, d in zip(hres, out):
                    h[a:b].copy_(d[a:b], non_blocking=True)
        for st in streams:
            cur.wait_stream(st)

    ref = tuple(t.cpu() for t in out)
    e2e_steps = max(3, args.steps // 4)
    e2e_ms = time_steps(e2e_step, e2e_steps, 3, dist_on) / e2e_steps
    torch.cuda.synchronize()
    e2e_same = all(torch.equal(h.view(torch.uint8), r.view(torch.uint8)) for h, r in zip(hres, ref))
    if not e2e_same:
        raise RuntimeError("the chunked end-to-end step changed the bits of the batched call")
    per = ms / args.steps
    return {
        "metric": f"batched twofold dots jobs/s ({nj} x 2^16)", "value": nj * world / (per * 1e-3),
        "e2e": {"value": nj * world / (e2e_ms * 1e-3), "unit": "jobs/s", "ms_per_step": e2e_ms,
                "how": f"inputs copied from pinned host memory, results read back, each step; {nchunk} chunks of "
                       f"jobs over two streams (copies overlap the dots)", "same_bits_as_one_call": bool(e2e_same),
                "h2d_bytes_per_step": 16 * nj * n, "d2h_bytes_per_step": 17 * nj},
        "unit": "jobs/s", "ms_per_step": per, "plain_ms_per_step": plain_ms / args.steps,
        "slowdown_vs_plain": per / (plain_ms / args.steps), "gbs": DOT_BYTES * nj * n / (per * 1e-3) / 1e9,
        "config": {"workload": f"{nj} ill-conditioned dots x 2^16, cond 10^U(2,30)", "n": nj * n,
                   "l2": f"inputs ({nj * n * 16 / 2**30:g} GiB) larger than L2", "parallelism": f"replicas x{world}"},
        "gpu_launches": args.steps, "clocks": cs.summary(),
        "_kernel_ms": per, "_ops": DOT_OPS * nj * n, "_bytes": DOT_BYTES * nj * n, "_units": nj * n,
        "_sample": None,
    }


def workload_horner(args, rank, world, dist_on):
    import torch
    import paper_1401_6235_gb300 as T
    import synth
    ks = [5, 10, 20, 30]
    npts = args.n or (1 << 24)
    coefs = np.concatenate([synth.binomial_coefs(k) for k in ks])
    coff = np.concatenate([[0], np.cumsum([k + 1 for k in ks])[:-1]]).astype(np.int32)
    x = np.concatenate([synth.horner_points(npts, seed=rank, stream=j) for j in range(len(ks))])
    xoff = (np.arange(len(ks) + 1) * npts).astype(np.int64)
    gc, gxx = torch.from_numpy(coefs).cuda(), torch.from_numpy(x).cuda()
    out = (torch.empty(x.size, dtype=torch.float64, device="cuda"),
           torch.empty(x.size, dtype=torch.float64, device="cuda"),
           torch.empty(x.size, dtype=torch.uint8, device="cuda"))
    step = lambda: T.twofold_horner_batched(gc, coff, ks, gxx, xoff, out=out)
    with ClockSampler(args.smi_index) as cs:
        ms = time_steps(step, args.steps, args.warmup, dist_on)
    pout = torch.empty(x.size, dtype=torch.float64, device="cuda")
    plain_ms = time_steps(lambda: T.plain_horner_batched(gc, coff, ks, gxx, xoff, out=pout), args.steps,
                          args.warmup, dist_on)
    plain_int = time_plain_integer(T, lambda: T.plain_horner_batched(gc, coff, ks, gxx, xoff, out=pout), args,
                                   dist_on)
    del pout
    # the same four jobs as one persistent mixed batch (autotuned points per
    # item and CTA size), replayed from a captured CUDA graph
    from paper_1401_6235_gb300 import batch as Bt
    bout = [torch.empty_like(t) for t in out]
    jobs = [Bt.horner_job(gc[int(coff[j]):int(coff[j]) + ks[j] + 1], gxx[int(xoff[j]):int(xoff[j + 1])],
                          out=tuple(t[int(xoff[j]):int(xoff[j + 1])] for t in bout)) for j in range(len(ks))]
    cfg = Bt.tune(jobs)
    graph = Bt.Batch(jobs, cfg=cfg).graph()
    batch_ms = time_steps(graph.replay, args.steps, args.warmup, dist_on) / args.steps
    same = all(torch.equal(u.view(torch.uint8), v.view(torch.uint8)) for u, v in zip(out, bout))
    del bout, jobs, graph
    # end to end: points in pinned host memory and the results written to pinned
    # host memory by the kernel itself (device-mapped), every step
    hx = torch.from_numpy(x).pin_memory()
    hout = (torch.empty(x.size, dtype=torch.float64).pin_memory(), torch.empty(x.size, dtype=torch.float64).pin_memory(),
            torch.empty(x.size, dtype=torch.uint8).pin_memory())
    e2e_steps = max(3, args.steps // 4)
    e2e_ms = time_steps(lambda: T.twofold_horner_batched(gc, coff, ks, hx, xoff, out=hout), e2e_steps, 3,
                        dist_on) / e2e_steps
    per = ms / args.steps
    steps_total = sum(ks) * npts
    return {
        "metric": "batched twofold Horner points/s (k=5,10,20,30 x 2^24)", "value": x.size * world / (per * 1e-3),
        "unit": "points/s", "ms_per_step": per, "plain_ms_per_step": plain_ms / args.steps,
        "slowdown_vs_plain": per / (plain_ms / args.steps), "plain_int_ms_per_step": plain_int,
        "slowdown_vs_plain_int": per / plain_int,
        "e2e": {"value": x.size * world / (e2e_ms * 1e-3), "unit": "points/s", "ms_per_step": e2e_ms,
                "how": "pinned host points and results, device-mapped", "h2d_bytes_per_step": 8 * x.size,
                "d2h_bytes_per_step": 17 * x.size},
        "persistent_batch": {"ms_per_step": batch_ms, "points_s": x.size * world / (batch_ms * 1e-3),
                             "config": {"points_per_item": cfg.points_per_item, "threads": cfg.threads},
                             "same_bits_as_batched_call": bool(same), "how": "twofold_batch, autotuned, graph replay"},
        "config": {"workload": "Horner (x-1)^k expanded, k in {5,10,20,30}, 2^24 points each, x~U[0.9,1.1]",
                   "n": int(x.size), "l2": "inputs 512 MiB larger than L2", "parallelism": f"replicas x{world}"},
        "gpu_launches": args.steps, "clocks": cs.summary(),
        "_kernel_ms": per, "_ops": HORNER_OPS_PER_STEP * steps_total + len(ks) * npts,
        "_bytes": HORNER_BYTES * x.size, "_units": x.size, "_pipe_units": steps_total, "_sample": None,
    }


def workload_batch_mix(args, rank, world, dist_on):
    """Thousands of uneven sum / dot / Horner jobs: one persistent launch of
    the mixed batch (replayed from a CUDA graph, configuration chosen by the
    autotuner) against one entry-point call per job, on the same data, with
    the results compared bit for bit."""
    import torch
    import paper_1401_6235_gb300 as T
    from paper_1401_6235_gb300 import batch as B
    import synth
    rng = np.random.default_rng(1000 + rank)
    nj = args.n or 2000
    kinds = rng.choice([T.JOB_DOT, T.JOB_SUM, T.JOB_HORNER], size=nj, p=[0.5, 0.25, 0.25])
    sizes = np.floor(10.0 ** rng.uniform(3, 6, nj)).astype(np.int64)
    degs = rng.integers(8, 31, nj)
    red = kinds != T.JOB_HORNER
    n_red, n_h = int(sizes[red].sum()), int(sizes[~red].sum())
    x, y = synth.dot_uniform(n_red, seed=rank)
    pts = synth.horner_points(n_h, seed=rank, stream=7)
    gx, gy, gp = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), torch.from_numpy(pts).cuda()
    coef = {k: torch.from_numpy(synth.binomial_coefs(k)).cuda() for k in range(8, 31)}
    jobs, a, b = [], 0, 0
    for kind, n, k in zip(kinds, sizes, degs):
        n = int(n)
        if kind == T.JOB_HORNER:
            jobs.append(B.horner_job(coef[int(k)], gp[b:b + n]))
            b += n
        elif kind == T.JOB_DOT:
            jobs.append(B.dot_job(gx[a:a + n], gy[a:a + n]))
            a += n
        else:
            jobs.append(B.sum_job(gx[a:a + n]))
            a += n
    cands = [(32, 4096, 128), (64, 16384, 256), (256, 16384, 256), (256, 4096, 256), (128, 65536, 512),
             (512, 65536, 512)]
    cfg = B.tune(jobs, cands=cands, reps=3)
    batch = B.Batch(jobs, cfg=cfg)
    g = batch.graph()
    with ClockSampler(args.smi_index) as cs:
        ms = time_steps(g.replay, args.steps, args.warmup, dist_on)
    got = [tuple(t.clone() for t in j.out) for j in jobs]
    # the same jobs, one entry-point call each (workspaces allocated up front)
    wsz = max(T.lib().twofold_workspace_bytes(T.KIND_DOT, int(n), 1, None) for n in sizes)
    ws = T.workspace(max(wsz, 256))

    def per_job():
        for j in jobs:
            if j.kind == T.JOB_DOT:
                T.twofold_dot(j.x, j.y, out=j.out, ws=ws)
            elif j.kind == T.JOB_SUM:
                T.twofold_sum(j.x, out=j.out, ws=ws)
            else:
                T.twofold_horner(j.coefs, j.x, out=j.out)

    pj_ms = time_steps(per_job, max(3, args.steps // 4), args.warmup, dist_on)
    torch.cuda.synchronize()
    same = all(torch.equal(u.view(torch.uint8), v.view(torch.uint8)) for o, j in zip(got, jobs)
               for u, v in zip(o, j.out))
    per = ms / args.steps
    pj = pj_ms / max(3, args.steps // 4)
    n_dot = int(sizes[kinds == T.JOB_DOT].sum())
    n_sum = n_red - n_dot
    hsteps = int((sizes[~red] * degs[~red]).sum())
    return {
        "metric": f"mixed batch jobs/s ({nj} jobs: dot 50%, sum 25%, Horner k 8-30 25%; sizes 10^U(3,6))",
        "value": nj * world / (per * 1e-3), "unit": "jobs/s", "ms_per_step": per,
        "per_job_launches": {"value": nj * world / (pj * 1e-3), "unit": "jobs/s", "ms_per_step": pj,
                             "launches_per_step": int(nj + (kinds != T.JOB_HORNER).sum())},
        "speedup_vs_per_job": pj / per, "same_bits_as_per_job": bool(same),
        "tuned_config": {"leaves_per_item": cfg.leaves_per_item, "points_per_item": cfg.points_per_item,
                         "threads": cfg.threads},
        "config": {"workload": "mixed sum/dot/Horner batch, x,y ~ U[-1,1], Horner x ~ U[0.9,1.1], binomial "
                               "coefficients", "jobs": nj, "elements": n_red, "points": n_h,
                   "l2": f"inputs ({(16 * n_red + 8 * n_h) / 2**30:.1f} GiB) larger than L2",
                   "parallelism": f"replicas x{world}"},
        "gpu_launches": args.steps, "clocks": cs.summary(),
        "_kernel_ms": per, "_ops": DOT_OPS * n_dot + 8 * n_sum + HORNER_OPS_PER_STEP * hsteps,
        "_bytes": DOT_BYTES * n_dot + 8 * n_sum + HORNER_BYTES * n_h, "_units": nj, "_sample": None,
    }


def workload_serve(args, rank, world, dist_on):
    """A Poisson stream of mixed requests (dot 40 %, sum 20 %, Horner k 8-30
    20 %, elementwise chain 20 %; sizes 10^U(3,7); dots of condition
    10^U(0,20)) through the request server at several arrival rates:
    achieved jobs/s and p50 / p99 latency from submission to completion,
    against a one-worker server that runs each request alone (copy in,
    single-job call, copy out, synchronise) on the same arrival times (its
    queue is replayed from measured service times)."""
    import torch
    import paper_1401_6235_gb300 as T
    from paper_1401_6235_gb300.serve import Server
    import synth
    rng = np.random.default_rng(2000 + rank)
    nreq = args.n or 100000
    rates = getattr(args, "serve_rates", None) or [2000.0, 4000.0, 8000.0, 16000.0]
    secs = getattr(args, "serve_seconds", None) or 8.0
    per_rate = [min(nreq, int(secs * r)) for r in rates[:-1]] + [nreq]    # ~secs of arrivals below the top rate
    pool = 1 << 24
    pin = lambda m: torch.empty(m, dtype=torch.float64).pin_memory().numpy()
    xy = synth.ew_chain(pool, seed=rank, pinned=pin)              # 8 pinned pools of 2^24 doubles
    hx = synth.horner_points(pool, seed=rank, stream=5)
    coef = {k: synth.binomial_coefs(k) for k in range(8, 31)}
    kinds = rng.choice(["dot", "sum", "horner", "ew"], size=nreq, p=[0.4, 0.2, 0.2, 0.2])
    sizes = np.floor(10.0 ** rng.uniform(3, 7, nreq)).astype(np.int64)
    offs = (rng.random(nreq) * (pool - sizes)).astype(np.int64)
    degs = rng.integers(8, 31, nreq)
    # dot requests: one of 128 ill-conditioned dots built up front (sizes 10^U(3,7), conditions 10^U(0,20))
    ndots = 128
    dsz = np.floor(10.0 ** rng.uniform(3, 7, ndots)).astype(np.int64)
    dx, dy = pin(int(dsz.sum())), pin(int(dsz.sum()))
    _, _, doffs, _, dcond = synth.cond_dots_sized(dsz, 10.0 ** rng.uniform(0, 20, ndots), seed=7 + rank, x=dx, y=dy)
    dsel = rng.integers(0, ndots, nreq)
    sizes = np.where(kinds == "dot", dsz[dsel], sizes)

    def args_of(i):
        a, n = int(offs[i]), int(sizes[i])
        sl = slice(a, a + n)
        if kinds[i] == "dot":
            d = slice(int(doffs[dsel[i]]), int(doffs[dsel[i] + 1]))
            return ("dot", dx[d], dy[d])
        if kinds[i] == "sum":
            return ("sum", xy["c0"][sl])
        if kinds[i] == "horner":
            return ("horner", coef[int(degs[i])], hx[sl])
        return ("ew", [(xy[c + "0"][sl], xy[c + "1"][sl]) for c in "abcd"])

    reqs = [args_of(i) for i in range(nreq)]
    # requests built up front (ctypes structs, outputs in shared pinned scratch: the
    # timed loop only submits), so that the client can offer rates above the server's
    import ctypes
    prog = np.ascontiguousarray(np.asarray(T.CHAIN_SQRT_MAD_DIV, np.int32))
    oh, ol = pin(pool), pin(pool)
    of = torch.empty(pool, dtype=torch.uint8).pin_memory().numpy()
    kind_id = {"dot": T.JOB_DOT, "sum": T.JOB_SUM, "horner": T.JOB_HORNER, "ew": T.JOB_EW}
    structs = []
    for r in reqs:
        q = T.tf_request()
        q.kind = kind_id[r[0]]
        if r[0] == "dot":
            q.n, q.inp[0], q.inp[2] = r[1].size, r[1].ctypes.data, r[2].ctypes.data
        elif r[0] == "sum":
            q.n, q.inp[0] = r[1].size, r[1].ctypes.data
        elif r[0] == "horner":
            q.n, q.k, q.coefs, q.inp[0] = r[2].size, r[1].size - 1, r[1].ctypes.data, r[2].ctypes.data
        else:
            q.n = r[1][0][0].size
            for i, (h, lo) in enumerate(r[1]):
                q.inp[2 * i], q.inp[2 * i + 1] = h.ctypes.data, lo.ctypes.data
            q.prog, q.nprog, q.nin = prog.ctypes.data, prog.shape[0], 4
        q.out_hi, q.out_lo, q.out_flags = oh.ctypes.data, ol.ctypes.data, of.ctypes.data
        structs.append(q)
    L = T.lib()
    submit_c, wait_c = L.twofold_server_submit, L.twofold_server_wait

    sweep, arrivals = [], []
    with Server(mem_cap=32 << 30, max_batch_jobs=4096) as srv:
        h = srv._h
        tid = ctypes.c_uint64()
        info = T.tf_request_info()
        # warm the server, the allocator and the kernels: the first 50 requests
        # and the largest of each kind (a large elementwise request builds the
        # specialised chain kernel, ~0.2-0.9 s on first use)
        warm = list(range(min(50, nreq)))
        for kd in ("dot", "sum", "horner", "ew"):
            idx = np.flatnonzero(kinds == kd)
            if idx.size:
                warm.append(int(idx[np.argmax(sizes[idx])]))
        for i in warm:
            submit_c(h, ctypes.byref(structs[i]), ctypes.byref(tid))
            wait_c(h, tid.value, -1, ctypes.byref(info))
        for rate, nr in zip(rates, per_rate):
            arrive = np.cumsum(rng.exponential(1.0 / rate, nr))
            arrivals.append(arrive)
            ids = np.empty(nr, np.uint64)
            t0 = time.perf_counter()
            for i, q in enumerate(structs[:nr]):
                while time.perf_counter() - t0 < arrive[i]:
                    pass
                st_ = submit_c(h, ctypes.byref(q), ctypes.byref(tid))
                if st_ != 0:
                    raise RuntimeError(f"submit: {T.strerror(st_)}")
                ids[i] = tid.value
            sub_s = time.perf_counter() - t0
            rec = np.empty((nr, 3))
            for i in range(nr):
                if wait_c(h, int(ids[i]), -1, ctypes.byref(info)) != 0:
                    raise RuntimeError("request failed")
                rec[i] = (info.submitted_ns, info.done_ns, info.batch_jobs)
            lat = (rec[:, 1] - rec[:, 0]) * 1e-6
            span = (rec[:, 1].max() - rec[:, 0].min()) * 1e-9
            sweep.append({"rate": rate, "requests": nr, "offered_jobs_s": nr / sub_s, "jobs_s": nr / span,
                          "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                          "mean_batch": float(rec[:, 2].mean())})
        stats = srv.stats()

    # one request at a time: copy in, single-job call, copy out, synchronise
    ws = T.workspace(T.lib().twofold_workspace_bytes(T.KIND_DOT, pool, 1, None))
    service = np.empty(nreq)
    for i, r in enumerate(reqs):
        t = time.perf_counter()
        if r[0] == "dot":
            o = T.twofold_dot(torch.from_numpy(r[1]).cuda(non_blocking=True),
                              torch.from_numpy(r[2]).cuda(non_blocking=True), ws=ws)
        elif r[0] == "sum":
            o = T.twofold_sum(torch.from_numpy(r[1]).cuda(non_blocking=True), ws=ws)
        elif r[0] == "horner":
            o = T.twofold_horner(torch.from_numpy(r[1]).cuda(non_blocking=True),
                                 torch.from_numpy(r[2]).cuda(non_blocking=True))
        else:
            o = T.twofold_ew(T.CHAIN_SQRT_MAD_DIV, [(torch.from_numpy(h).cuda(non_blocking=True),
                                                     torch.from_numpy(lo).cuda(non_blocking=True)) for h, lo in r[1]])
        [t_.cpu() for t_ in o]
        torch.cuda.synchronize()
        service[i] = time.perf_counter() - t
    for row, arrive in zip(sweep, arrivals):       # the per-job server on the same arrival times
        nr = arrive.size
        done = np.empty(nr)
        free = 0.0
        for i in range(nr):
            free = max(arrive[i], free) + service[i]
            done[i] = free
        lat = (done - arrive) * 1e3
        row["per_job"] = {"jobs_s": nr / (done[-1] - arrive[0]), "p50_ms": float(np.percentile(lat, 50)),
                          "p99_ms": float(np.percentile(lat, 99))}
    top = sweep[-1]
    moved = sum(16 * int(sizes[i]) if kinds[i] == "dot" else 8 * int(sizes[i]) if kinds[i] == "sum" else
                25 * int(sizes[i]) if kinds[i] == "horner" else 81 * int(sizes[i]) for i in range(nreq))
    return {
        "metric": "served twofold jobs/s at the highest offered rate (Poisson, mixed kinds), p50/p99 latency",
        "value": top["jobs_s"], "unit": "jobs/s", "ms_per_step": 1e3 / top["jobs_s"],
        "sweep": sweep, "server": {k: stats[k] for k in ("batches", "batched_jobs", "peak_bytes", "max_inflight")},
        "config": {"workload": f"Poisson streams of {per_rate} requests (one per rate): dot 40%, sum 20%, Horner k "
                               "8-30 20%, chain 20%; sizes 10^U(3,7); dots drawn from 128 ill-conditioned dots "
                               "(cond 10^U(0,20)); other inputs slices of pinned host pools; memory cap 32 GiB",
                   "rates": rates, "dot_cond_range": [float(dcond.min()), float(dcond.max())],
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": top["jobs_s"], "unit": "jobs/s", "h2d_bytes_per_step": int(moved / nreq),
                "d2h_bytes_per_step": None},
        "gpu_launches": None, "clocks": {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0},
        "_kernel_ms": 1e3 / top["jobs_s"], "_ops": 0, "_bytes": moved / nreq, "_units": None, "_sample": None,
    }


def workload_ew_f32(args, rank, world, dist_on):
    """The chain sqrt((a*b + c)/d) over binary32 twofolds (the paper's float
    basis): heads float(v), tails float(v - head) of the binary64 chain
    inputs, 41 B per element (plain twin 20 B).  On this GPU the binary32
    arithmetic runs on the wide FP32 pipe, so the kernel is bound by HBM."""
    import torch
    import paper_1401_6235_gb300 as T
    import synth
    n = args.n or (1 << 28)
    prog = T.CHAIN_SQRT_MAD_DIV
    g = {k: (torch.empty(n, dtype=torch.float32, device="cuda"), torch.empty(n, dtype=torch.float32, device="cuda"))
         for k in "abcd"}
    chunk = 1 << 24
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        d = synth.ew_chain(e - s, seed=rank * 1000 + s // chunk)
        for k in "abcd":
            h = d[k + "0"].astype(np.float32)
            g[k][0][s:e].copy_(torch.from_numpy(h))
            g[k][1][s:e].copy_(torch.from_numpy((d[k + "0"] - h.astype(np.float64)).astype(np.float32)))
    ins = [g[k] for k in "abcd"]
    out = (torch.empty(n, dtype=torch.float32, device="cuda"), torch.empty(n, dtype=torch.float32, device="cuda"),
           torch.empty(n, dtype=torch.uint8, device="cuda"))
    pout = torch.empty(n, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    with ClockSampler(args.smi_index) as cs:
        ms = time_steps(lambda: T.twofold_ew_f32(prog, ins, out=out), args.steps, args.warmup, dist_on)
    plain_ms = time_steps(lambda: T.plain_ew_f32(prog, [h for h, _ in ins], out=pout), args.steps, args.warmup,
                          dist_on)
    del pout
    # end to end: the same call on pinned host inputs and outputs that the
    # device maps (the kernel moves every byte across the host link)
    hins = [(t[0].cpu().pin_memory(), t[1].cpu().pin_memory()) for t in ins]
    hout = (torch.empty(n, dtype=torch.float32).pin_memory(), torch.empty(n, dtype=torch.float32).pin_memory(),
            torch.empty(n, dtype=torch.uint8).pin_memory())
    e2e_steps = max(3, args.steps // 8)
    e2e_ms = time_steps(lambda: T.twofold_ew_f32(prog, hins, out=hout), e2e_steps, 3, dist_on) / e2e_steps
    per = ms / args.steps
    nbytes = EW32_BYTES * n
    return {
        "e2e": {"value": nbytes * world / (e2e_ms * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": e2e_ms,
                "how": "pinned host inputs and outputs, device-mapped", "h2d_bytes_per_step": 32 * n,
                "d2h_bytes_per_step": 9 * n},
        "metric": "twofold GB/s, binary32 basis (elementwise chain sqrt((a*b+c)/d), 41 B/elt)",
        "value": nbytes * world / (per * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": per,
        "plain_ms_per_step": plain_ms / args.steps, "slowdown_vs_plain": per / (plain_ms / args.steps),
        "plain_gbs": EW32_PLAIN_BYTES * n * world / (plain_ms / args.steps * 1e-3) / 1e9,
        "config": {"workload": "ew_chain binary32 sqrt((a*b+c)/d)", "n": n, "bytes_per_elt": EW32_BYTES,
                   "inputs": "the binary64 chain inputs as binary32 twofolds (head float(v), tail float(v-head))",
                   "l2": "inputs (8 GiB) larger than L2; no flush needed", "parallelism": f"replicas x{world}"},
        "gpu_launches": args.steps, "clocks": cs.summary(),
        "_kernel_ms": per, "_ops": 0, "_bytes": nbytes, "_units": n, "_sample": None,
        "_bound": "hbm", "_dtype": "f32",
    }


def workload_dot_f32(args, rank, world, dist_on):
    """A binary32 twofold dot of 2^28 dotted elements (the paper's float
    basis; inputs 2 GiB, beyond L2), against its plain binary32 twin: the
    FP32 pipe is wide here, so the bound is HBM (8 B per element)."""
    import torch
    import paper_1401_6235_gb300 as T
    import synth
    n = args.n or (1 << 28)
    gx = torch.from_numpy(synth.uniform(rank, 0, n, -1.0, 1.0).astype(np.float32)).cuda()
    gy = torch.from_numpy(synth.uniform(rank, 1, n, -1.0, 1.0).astype(np.float32)).cuda()
    ws = T.workspace(T.lib().twofold_workspace_bytes(T.KIND_DOT, n, 1, None))
    out = (torch.empty(1, dtype=torch.float32, device="cuda"), torch.empty(1, dtype=torch.float32, device="cuda"),
           torch.empty(1, dtype=torch.uint8, device="cuda"))
    pout = torch.empty(1, dtype=torch.float32, device="cuda")
    with ClockSampler(args.smi_index) as cs:
        ms = time_steps(lambda: T.twofold_dot_f32(gx, gy, out=out, ws=ws), args.steps, args.warmup, dist_on)
    plain_ms = time_steps(lambda: T.plain_dot_f32(gx, gy, out=pout, ws=ws), args.steps, args.warmup, dist_on)
    # end to end: the inputs copied in from pinned host memory and the result read back, every step
    hx, hy = gx.cpu().pin_memory(), gy.cpu().pin_memory()
    hres = tuple(torch.empty(1, dtype=t.dtype).pin_memory() for t in out)

    def e2e_step():
        gx.copy_(hx, non_blocking=True)
        gy.copy_(hy, non_blocking=True)
        T.twofold_dot_f32(gx, gy, out=out, ws=ws)
        for h, d in zip(hres, out):
            h.copy_(d, non_blocking=True)

    e2e_steps = max(3, args.steps // 4)
    e2e_ms = time_steps(e2e_step, e2e_steps, 3, dist_on) / e2e_steps
    per = ms / args.steps
    return {
        "metric": "binary32 twofold dot GB/s (2^28 dotted elements, 8 B/elt)", "value": 8 * n * world / (per * 1e-3) / 1e9,
        "unit": "GB/s", "ms_per_step": per, "plain_ms_per_step": plain_ms / args.steps,
        "slowdown_vs_plain": per / (plain_ms / args.steps),
        "config": {"workload": "dot_f32 x, y uniform[-1,1] float, seed = rank, L=256", "n": n,
                   "l2": "inputs (2 GiB) larger than L2; no flush needed", "parallelism": f"replicas x{world}"},
        "e2e": {"value": 8 * n * world / (e2e_ms * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": e2e_ms,
                "how": "inputs copied from pinned host memory, result read back, each step",
                "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 9},
        "gpu_launches": 2 * args.steps, "clocks": cs.summary(),
        "_kernel_ms": per, "_ops": 0, "_bytes": 8 * n, "_units": n, "_bound": "hbm", "_dtype": "f32",
        "_sample": None,
    }


def workload_dot_sharded(args, rank, world, dist_on):
    """One twofold dot split across the ranks (one GPU each): 2^28 dotted
    elements per rank on aligned 2^k-leaf shards, each rank reducing its
    shard, the 16-byte partials all-gathered and the tree finished on every
    rank (twofold_combine); the result is the one-GPU result bit for bit.
    Per-rank work is fixed, so scaling is weak."""
    import torch
    import paper_1401_6235_gb300 as T
    import synth
    from paper_1401_6235_gb300.dist import reduce_sharded, shard_plan
    per_rank = args.n or (1 << 28)
    n_total = per_rank * world
    a, b = shard_plan(n_total, 256, world)[rank]
    gx = torch.from_numpy(synth.uniform_slice(7, 0, a, b, -1.0, 1.0)).cuda()
    gy = torch.from_numpy(synth.uniform_slice(7, 1, a, b, -1.0, 1.0)).cuda()
    ws = T.workspace(T.lib().twofold_workspace_bytes(T.KIND_DOT, b - a, 1, None))
    local_out = tuple(torch.empty(1, dtype=dt, device="cuda") for dt in (torch.float64, torch.float64, torch.uint8))
    cws = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    cout = tuple(torch.empty(1, dtype=dt, device="cuda") for dt in (torch.float64, torch.float64, torch.uint8))

    def step():
        if dist_on:
            return reduce_sharded(lambda: T.twofold_dot(gx, gy, out=local_out, ws=ws)[:2],
                                  lambda u, v: T.twofold_combine(u, v, out=cout, ws=cws), n_total, 256, rank, world,
                                  gx.device)
        z0, z1, _ = T.twofold_dot(gx, gy, out=local_out, ws=ws)
        return T.twofold_combine(z0, z1, out=cout, ws=cws)

    with ClockSampler(args.smi_index) as cs:
        ms = time_steps(step, args.steps, args.warmup, dist_on)
    per = ms / args.steps
    return {
        "metric": "sharded twofold dot, elements/s (2^28 dotted elements per GPU)",
        "value": n_total / (per * 1e-3), "unit": "elements/s", "ms_per_step": per,
        "config": {"workload": "one dot over all ranks, x,y ~ U[-1,1] seed 7, aligned 2^k-leaf shards, L=256",
                   "n_total": n_total, "l2": f"inputs ({16 * (b - a) / 2**30:g} GiB per GPU) larger than L2",
                   "parallelism": f"sharded x{world}"},
        "e2e": None, "gpu_launches": 3 * args.steps, "clocks": cs.summary(),   # leaves, tree, combine
        "_kernel_ms": per, "_ops": DOT_OPS * (b - a), "_bytes": DOT_BYTES * (b - a), "_units": b - a,
        "_sample": None,
    }


def workload_criteria(args, rank, world, dist_on):
    """The paper's speed criteria for twofolds: at most 2x the plain
    arithmetic's time on data outside the caches and 10x inside them.  The
    chain sqrt((a*b+c)/d): GPU kernels at n = 100 and 10^4 (launch-bound),
    2^20 (inputs L2-resident) and 2^26 (inputs 4 GiB, beyond L2), each
    twofold time over its plain twin's; the host side (the oracle, as it
    stands, 1 thread and all threads) at n = 100, 10^4 and 2^26."""
    import torch
    import paper_1401_6235_gb300 as T
    import synth
    prog = T.CHAIN_SQRT_MAD_DIV
    sizes = [100, 10 ** 4, 1 << 20, 1 << 26]
    rows = []
    for n in sizes:
        d = synth.ew_chain(n, seed=3)
        g = [(torch.from_numpy(d[k + "0"]).cuda(), torch.from_numpy(d[k + "1"]).cuda()) for k in "abcd"]
        out = (torch.empty(n, dtype=torch.float64, device="cuda"), torch.empty(n, dtype=torch.float64, device="cuda"),
               torch.empty(n, dtype=torch.uint8, device="cuda"))
        pout = torch.empty(n, dtype=torch.float64, device="cuda")
        reps = max(10, min(2000, (1 << 27) // n))
        tf = time_steps(lambda: T.twofold_ew(prog, g, out=out), reps, args.warmup, dist_on) / reps
        pl = time_steps(lambda: T.plain_ew(prog, [h for h, _ in g], out=pout), reps, args.warmup, dist_on) / reps
        prev_mode = T.plain_arith(T.PLAIN_INTEGER)
        try:
            pli = time_steps(lambda: T.plain_ew(prog, [h for h, _ in g], out=pout), reps, args.warmup,
                             dist_on) / reps
        finally:
            T.plain_arith(prev_mode)
        rows.append({"n": n, "where": "L2" if n <= (1 << 20) else "HBM", "twofold_us": tf * 1e3,
                     "plain_us": pl * 1e3, "slowdown": tf / pl,
                     "plain_int_us": pli * 1e3, "slowdown_vs_plain_int": tf / pli,
                     "criterion": "2x" if n > (1 << 20) else "10x", "met": tf / pl <= (2.0 if n > (1 << 20) else 10.0)})
        del g, out, pout
    top = rows[-1]
    return {
        "metric": "twofold / plain time, chain sqrt((a*b+c)/d), n = 2^26 (paper criterion: <= 2x uncached)",
        "value": top["slowdown"], "unit": "x", "higher_is_better": False, "ms_per_step": top["twofold_us"] * 1e-3,
        "gpu": rows,
        "config": {"workload": "ew_chain sqrt((a*b+c)/d) at n = 100, 1e4, 2^20, 2^26 (seed 3)",
                   "l2": "n <= 2^20 L2-resident (the cached criterion), 2^26 beyond L2",
                   "parallelism": f"replicas x{world}"},
        "e2e": None, "gpu_launches": None,
        "clocks": {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0},
        "_kernel_ms": top["twofold_us"] * 1e-3, "_ops": EW_OPS * sizes[-1], "_bytes": EW_BYTES * sizes[-1],
        "_units": sizes[-1], "_sample": cpu_criteria,
    }


def cpu_criteria():
    """The oracle's twofold / plain slowdown on the host cores."""
    import oracle as O
    import paper_1401_6235_gb300 as T
    import synth
    prog = T.CHAIN_SQRT_MAD_DIV
    rows = []
    for n, threads in [(100, 1), (10 ** 4, 1), (1 << 26, 1), (1 << 26, O.THREADS)]:
        d = synth.ew_chain(n, seed=3)
        ins = [(d[k + "0"], d[k + "1"]) for k in "abcd"]
        his = [h for h, _ in ins]
        reps = max(1, min(2000, (1 << 20) // n))
        t = time.perf_counter()
        for _ in range(reps):
            O.ew(prog, ins, threads=threads)
        tf = (time.perf_counter() - t) / reps
        t = time.perf_counter()
        for _ in range(reps):
            O.ew_plain(prog, his, threads=threads)
        pl = (time.perf_counter() - t) / reps
        rows.append({"n": n, "threads": threads, "twofold_s": tf, "plain_s": pl, "slowdown": tf / pl,
                     "criterion": "2x" if n > (1 << 20) else "10x"})
    top = rows[-1]
    return {"value": top["slowdown"], "unit": "x", "cores": O.THREADS, "kind": "oracle",
            "sample": "the chain at n = 100, 1e4 (1 thread) and 2^26 (1 thread, all threads): twofold over plain "
                      "time of the oracle as it stands", "rows": rows}


WORKLOADS = {"ew_chain": workload_ew, "dot": workload_dot, "cond_dots": workload_cond_dots,
             "horner": workload_horner, "batch_mix": workload_batch_mix, "serve": workload_serve,
             "ew_chain_f32": workload_ew_f32, "criteria": workload_criteria,
             "dot_f32": workload_dot_f32, "dot_sharded": workload_dot_sharded, "fp64_peak": workload_fp64_peak}


# -------------------------------------------------------------- reference

def run_reference(args, rank, world):
    """The CPU oracle, as it stands, on a bounded sample per step."""
    if rank != 0:
        return
    import oracle as O
    import paper_1401_6235_gb300 as T
    import synth
    m = args.n or (1 << 23)
    d = synth.ew_chain(m, seed=0)
    ins = [(d[k + "0"], d[k + "1"]) for k in "abcd"]
    for _ in range(args.warmup):
        O.ew(T.CHAIN_SQRT_MAD_DIV, ins)
    t = time.perf_counter()
    for _ in range(args.steps):
        O.ew(T.CHAIN_SQRT_MAD_DIV, ins)
    dt = (time.perf_counter() - t) / args.steps
    v = EW_BYTES * m / dt / 1e9
    print(json.dumps({
        "impl": "reference",
        "metric": "twofold GB/s (elementwise chain sqrt((a*b+c)/d), 81 B/elt)",
        "value": v, "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "ew_chain sqrt((a*b+c)/d)", "n": m,
                   "sample": f"{m} elements of the 2^28 workload per step (CPU oracle)"},
        "cpu_baseline": {"value": v, "unit": "GB/s", "cores": O.THREADS, "kind": "oracle",
                         "sample": f"{m} elements per step"},
        "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------------------- line

def pipe_roofline(wl, pipe_units, kms, rates, sms, mhz):
    """Per-pipe floors of the dominant kernel (PIPE_LOAD x units over the
    measured pipe rates at the sampled clock) and the roofline of the
    binding pipe; None where the kernel has no committed counts."""
    load = PIPE_LOAD.get(wl)
    if not load or not rates or not pipe_units or kms <= 0:
        return None
    per, unit_of_work, src = load
    hz = sms * mhz * 1e6
    floors = {p: slots * pipe_units / (rates[PIPE_PROBE[p]] * hz) * 1e3 for p, slots in per.items()
              if rates.get(PIPE_PROBE[p])}
    bound = max(floors, key=floors.get)
    achieved = per[bound] * pipe_units / (kms * 1e-3) / 1e12
    peak = rates[PIPE_PROBE[bound]] * hz / 1e12
    r = {"bound": "alu", "pipe": bound, "achieved": achieved, "peak": peak, "unit": "Tinst/s",
         "frac": achieved / peak, "floors_ms": floors, "kernel_ms": kms,
         "load_per_unit": per, "unit_of_work": unit_of_work, "load_source": src,
         "pipe_rates": {p: rates[PIPE_PROBE[p]] for p in per if rates.get(PIPE_PROBE[p])},
         "what": "lane instructions of the binding pipe per second (ncu count per unit x units / kernel time) vs "
                 "its rate measured in this run by the pipe-rate probes (lane ops per SM clock x SMs x sampled "
                 "clock); frac = the pipe's floor / the kernel time"}
    alg = ALG_FP64.get(wl)
    if alg and rates.get("dadd"):
        fp64_peak = rates["dadd"] * hz / 1e12
        a = alg * pipe_units / (kms * 1e-3) / 1e12
        r["fp64_algorithmic"] = {"per_unit": alg, "achieved": a, "peak": fp64_peak, "frac": a / fp64_peak,
                                 "what": "FP64 instructions the paper's algorithms need per unit, per second, vs "
                                         "the measured FP64 rate"}
    return r


def build_line(res, args, world, sms, hbm, src, rates=None):
    """The JSON line of a workload's result dict: the contract's keys, the
    roofline of the dominant kernel (alu: its binding execution pipe, per
    pipe_roofline; hbm: algorithmic bytes against the measured copy
    bandwidth) and the CPU baseline sample."""
    res = dict(res)
    sample = res.pop("_sample")
    kms, ops, nbytes = res.pop("_kernel_ms"), res.pop("_ops"), res.pop("_bytes")
    units = res.pop("_units", None)
    pipe_units = res.pop("_pipe_units", units)
    tr = TRAFFIC_PER_UNIT.get(args.workload)
    traffic = round(tr[0] * units) if tr and units else None
    clk = res["clocks"]["sm_mhz"] or 2070.0
    bound = res.pop("_bound", "alu")
    if bound == "none" or kms <= 0:                # a measurement of the peaks themselves
        res["roofline"] = None
    elif bound == "latency":                       # one short reduction: its dependent chain bounds it
        f = res["latency_floor"]
        res["roofline"] = {"bound": "latency", "pipe": "fp64 dependent adds", "achieved": f["floor_us"] / f["frac"],
                           "floor": f["floor_us"], "unit": "us", "frac": f["frac"], "traffic": traffic,
                           "traffic_source": tr[1] if traffic else None, "what": f["what"]}
    elif bound == "hbm":
        gbs = nbytes / (kms * 1e-3) / 1e9
        res["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                           "traffic": traffic, "traffic_source": tr[1] if traffic else None,
                           "what": f"algorithmic bytes per launch / launch time vs the {src} copy bandwidth"}
    else:
        r = pipe_roofline(args.workload, pipe_units, kms, rates, sms, clk) if ops else None
        if r is not None:
            r["traffic"] = traffic
            r["traffic_source"] = tr[1] if traffic else None
        res["roofline"] = r
    if kms > 0:
        res["hbm"] = {"achieved": nbytes / (kms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                      "frac": nbytes / (kms * 1e-3) / 1e9 / hbm, "peak_source": src}
    if sample is not None and not args.no_cpu_baseline and world == 1:    # rank 0 at N = 1 only
        res["cpu_baseline"] = sample()
    line = {"metric": res.pop("metric"), "value": res.pop("value"), "unit": res.pop("unit"),
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res.pop("ms_per_step"), "higher_is_better": res.pop("higher_is_better", True),
            "scaling": "weak", "vs_baseline": None, "dtype": res.pop("_dtype", "f64"), "data": "synthetic"}
    line.update(res)
    return line


# ------------------------------------------------------------ sub-results

SUB_KEEP = ("metric", "value", "unit", "ms_per_step", "plain_ms_per_step", "slowdown_vs_plain",
            "plain_int_ms_per_step", "slowdown_vs_plain_int", "graph", "latency_floor", "persistent_batch",
            "per_job_launches", "speedup_vs_per_job", "same_bits_as_per_job", "tuned_config", "sweep", "e2e",
            "clocks", "gbs")


def subresult(name, fn, args, over, rank, world, dist_on, sms, hbm, src, rates):
    """One other workload of the hot path, shortened, for the default line:
    its headline figures and its roofline, built as its own line would be."""
    import types
    a = types.SimpleNamespace(**vars(args))
    a.workload = name
    for k, v in over.items():
        setattr(a, k, v)
    a.no_cpu_baseline = True
    t0 = time.perf_counter()
    res = fn(a, rank, world, dist_on)
    line = build_line(res, a, world, sms, hbm, src, rates)
    out = {k: line[k] for k in SUB_KEEP if k in line}
    out.update({"steps": a.steps, "config": line["config"], "roofline": line.get("roofline"),
                "hbm_frac": (line.get("hbm") or {}).get("frac"), "wall_s": time.perf_counter() - t0})
    return out


# The other measured rows, run after the chain in the default line: the
# 65536-element dot, the 4096 ill-conditioned dots, the batched Horner, the
# mixed persistent batch and a shortened serving sweep.
SUBRESULTS = [
    ("dot", {"steps": 200, "warmup": 20, "n": 0}),
    ("cond_dots", {"steps": 10, "warmup": 3, "n": 0}),
    ("horner", {"steps": 10, "warmup": 3, "n": 0}),
    ("batch_mix", {"steps": 10, "warmup": 3, "n": 0}),
    ("serve", {"steps": 1, "warmup": 3, "n": 10000, "serve_rates": [2000.0, 8000.0], "serve_seconds": 2.0}),
]


# ------------------------------------------------------------------- main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="ew_chain", choices=sorted(WORKLOADS))
    ap.add_argument("--n", type=int, default=0, help="override the problem size (testing)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-subresults", action="store_true",
                    help="default workload only: skip the other rows' shortened runs")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    dist_on = world > 1
    torch.cuda.set_device(local)
    if dist_on:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    args.smi_index = int(vis.split(",")[local]) if vis and vis.split(",")[local].isdigit() else local

    import __graft_entry__ as entry
    import paper_1401_6235_gb300 as T
    entry.build() if not os.path.exists(T.LIB_PATH) else None

    # the pipe rates of this GPU, for the roofline of pipe-bound kernels
    rates = None
    if args.workload in PIPE_LOAD:
        m = measure_pipes(tuple(sorted(set(PIPE_PROBE.values()))), target_cycles=2e6, reps=2)
        rates = {k: v["op_per_clk_sm"] for k, v in m.items()}
    res = WORKLOADS[args.workload](args, rank, world, dist_on)
    hbm, src = measured_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    subs = {}
    if args.workload == "ew_chain" and not args.no_subresults and not args.n:
        m = measure_pipes(tuple(sorted(set(PIPE_PROBE.values()))), target_cycles=2e6, reps=2)
        r2 = {k: v["op_per_clk_sm"] for k, v in m.items()}
        for name, over in SUBRESULTS:
            subs[name] = subresult(name, WORKLOADS[name], args, over, rank, world, dist_on, sms, hbm, src, r2)
            torch.cuda.empty_cache()
    if rank == 0:
        line = build_line(res, args, world, sms, hbm, src, rates)
        if subs:
            line["subresults"] = subs
        print(json.dumps(line), flush=True)
    if dist_on:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
