"""The pipe-rate probe (twofold_pipe_probe), whose measured rates are the
peaks of the bench line's roofline: every launch configuration stamps every
CTA, the rates come out in the ranges GB300's pipes allow (binary64 add at
most the FP64 pipe's nominal 2 lanes per SM clock, integer mad and funnel
shift at most 64, binary32 fma at most 128), the latency form of a binary64
add takes tens of clocks, and bad arguments are rejected before launch."""
import numpy as np
import pytest

import bench
import paper_1401_6235_gb300 as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    import __graft_entry__ as e
    e.build()
    return torch


def test_stamps_cover_every_cta(torch):
    blocks, threads = 300, 64
    rec = T.pipe_probe(T.PROBE_DADD, 3, blocks, threads)
    torch.cuda.synchronize()
    st = rec.cpu().numpy().reshape(-1, 4)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert st.shape == (blocks, 4)
    assert ((st[:, 0] >= 0) & (st[:, 0] < sms)).all()
    assert (st[:, 2] > st[:, 1]).all()


def test_rates_within_the_pipes_limits(torch):
    r = bench.measure_pipes(("dadd", "dfma", "imad", "shf", "ffma"), target_cycles=5e5, reps=1)
    assert 0.5 < r["dadd"]["op_per_clk_sm"] <= 2.05
    assert 0.5 < r["dfma"]["op_per_clk_sm"] <= 2.05
    assert 16 < r["imad"]["op_per_clk_sm"] <= 64.5
    assert 16 < r["shf"]["op_per_clk_sm"] <= 64.5
    assert 32 < r["ffma"]["op_per_clk_sm"] <= 128.5
    lat = bench.measure_latencies(("dadd", "imad"), target_cycles=2e5)
    assert 8 < lat["dadd"]["cycles"] < 500 and 1 < lat["imad"]["cycles"] < 50
    # two dependent adds per element: at least twice the add's latency
    assert 2 * lat["dadd"]["cycles"] * 0.95 < lat["chain_lds_element"]["cycles"] < 1000
    assert 2 * lat["dadd"]["cycles"] * 0.95 < lat["chain_ahead_element"]["cycles"] < 1000


def test_bad_arguments_are_rejected(torch):
    rec = torch.empty(16, dtype=torch.int64, device="cuda")
    L = T.lib()
    assert L.twofold_pipe_probe(99, 1, 4, 64, rec.data_ptr(), None) == T.TF_EINVAL
    assert L.twofold_pipe_probe(T.PROBE_FFMA | T.PROBE_LATENCY, 1, 4, 64, rec.data_ptr(), None) == T.TF_EINVAL
    assert L.twofold_pipe_probe(T.PROBE_DADD, 1, 4, 48, rec.data_ptr(), None) == T.TF_EINVAL
    assert L.twofold_pipe_probe(T.PROBE_DADD, 1, 4, 64, None, None) == T.TF_EINVAL
