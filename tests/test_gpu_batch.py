"""GPU parity of the mixed persistent batch (C ABI twofold_batch_*): every
job of a mix of sums, dots and Horner evaluations (empty, tiny, ragged, split
into many items, with and without tails, degrees 0..40) equals the oracle and
its single-job entry point bit for bit, under several configurations; a
prepared plan launched again, and replayed from a captured CUDA graph, gives
the same bits; the autotuner's choice too."""
import numpy as np
import pytest

import oracle as O
import paper_1401_6235_gb300 as T
import synth
from paper_1401_6235_gb300 import batch as B
from tests.fp import rand_tails
from tests.gpu_util import assert_bits, assert_flags, dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as e
    e.build()


def make_mix(seed, njobs=60, big=True):
    """Jobs and their oracle results."""
    rng = np.random.default_rng(seed)
    jobs, ref = [], []
    sizes = [0, 1, 2, 255, 256, 257, 4097, 65536, 100003]
    if big:
        sizes += [1 << 20, 3_000_001]
    for j in range(njobs):
        kind = [T.JOB_SUM, T.JOB_DOT, T.JOB_HORNER][j % 3]
        n = int(sizes[rng.integers(len(sizes))]) if j % 7 else int(rng.integers(0, 300000))
        if kind == T.JOB_HORNER:
            k = int(rng.integers(0, 41))
            a = synth.binomial_coefs(min(k, 30)) if k <= 30 else rng.standard_normal(k + 1)
            x = synth.horner_points(n, seed=seed * 1000 + j)
            jobs.append(B.horner_job(dev(a), dev(x)))
            ref.append(O.horner(a, x))
            continue
        x, y = synth.dot_uniform(n, seed=seed * 1000 + j)
        xl = rand_tails(np.random.default_rng(j), x, 30, 60) if (j % 4 == 1 and n) else None
        if kind == T.JOB_SUM:
            jobs.append(B.sum_job(dev(x), None if xl is None else dev(xl)))
            e0, e1 = O.reduce(x, xl, L=256)
        else:
            jobs.append(B.dot_job(dev(x), dev(y), None if xl is None else dev(xl)))
            e0, e1 = O.reduce(x, xl, y, None, L=256)
        ref.append(([e0], [e1], [O.flag(e0, e1)]))
    return jobs, ref


def check(jobs, ref, what):
    for i, (j, r) in enumerate(zip(jobs, ref)):
        if j.kind == T.JOB_HORNER and j.n == 0:
            continue
        assert_bits(j.out[0], r[0], f"{what} job {i} z0")
        assert_bits(j.out[1], r[1], f"{what} job {i} z1")
        assert_flags(j.out[2], r[2], f"{what} job {i} flags")


@pytest.mark.parametrize("cfg", [None, (32, 4096, 128), (256, 65536, 512), (1, 1000, 256), (64, 16384, 256, 1)])
def test_mixed_batch_equals_oracle(cfg):
    jobs, ref = make_mix(1)
    b = B.Batch(jobs, cfg=None if cfg is None else B.config(*cfg))
    b.launch()
    check(jobs, ref, f"cfg {cfg}")


def test_batch_equals_single_job_calls():
    jobs, _ = make_mix(2, njobs=30, big=False)
    B.Batch(jobs, cfg=B.config(64, 4096, 256)).launch()
    for i, j in enumerate(jobs):
        if j.kind == T.JOB_SUM:
            s = T.twofold_sum(j.x, j.xl)
        elif j.kind == T.JOB_DOT:
            s = T.twofold_dot(j.x, j.y, j.xl, j.yl)
        else:
            if j.n == 0:
                continue
            s = T.twofold_horner(j.coefs, j.x)
        for u, v in zip(j.out, s):
            assert np.array_equal(u.cpu().numpy().view(np.uint8), v.cpu().numpy().view(np.uint8)), i


def test_jobs_on_unaligned_views():
    """Dotted sum and dot jobs that are views into one buffer at even and odd
    element offsets (16-byte and one-element leaf walks in one launch)."""
    rng = np.random.default_rng(31)
    x, y = synth.dot_uniform(2_000_003, seed=31)
    gx, gy = dev(x), dev(y)
    jobs, ref, a = [], [], 0
    for j, n in enumerate([100003, 65536, 1, 257, 300000, 4097, 1 << 20, 77]):
        a += int(rng.integers(0, 3))
        if j % 2:
            jobs.append(B.dot_job(gx[a:a + n], gy[a + 1:a + 1 + n]))
            e0, e1 = O.reduce(x[a:a + n], None, y[a + 1:a + 1 + n], None, L=256)
        else:
            jobs.append(B.sum_job(gx[a:a + n]))
            e0, e1 = O.reduce(x[a:a + n], None, L=256)
        ref.append(([e0], [e1], [O.flag(e0, e1)]))
        a += n
    B.Batch(jobs).launch()
    check(jobs, ref, "views")


def test_relaunch_and_graph_replay():
    """The kernel leaves its counters zeroed: the same plan launched again,
    and replayed from a captured graph, gives the same bits."""
    import torch
    jobs, ref = make_mix(3, njobs=40, big=False)
    b = B.Batch(jobs, cfg=B.config(32, 4096, 256))
    for _ in range(3):
        for j in jobs:
            for t in j.out:
                t.fill_(7)
        b.launch()
        check(jobs, ref, "relaunch")
    g = b.graph()
    for _ in range(3):
        for j in jobs:
            for t in j.out:
                t.fill_(7)
        g.replay()
        torch.cuda.synchronize()
        check(jobs, ref, "graph replay")


def test_two_prepared_batches_stay_independent():
    """Each prepared plan keeps its tables in its own workspace: preparing a
    second batch (and running single-job calls) leaves the first intact."""
    jobs_a, ref_a = make_mix(5, njobs=30, big=False)
    jobs_b, ref_b = make_mix(6, njobs=30, big=False)
    a = B.Batch(jobs_a, cfg=B.config(32, 4096, 256))
    b = B.Batch(jobs_b, cfg=B.config(32, 4096, 256))
    T.twofold_dot(jobs_b[1].x, jobs_b[1].y)                 # the shared scratch of the single calls
    for _ in range(2):
        for j in jobs_a + jobs_b:
            for t in j.out:
                t.fill_(7)
        a.launch()
        b.launch()
        check(jobs_a, ref_a, "batch a")
        check(jobs_b, ref_b, "batch b")


def test_panic_params_and_leaf():
    """tf_params (leaf, ULP panic mode) apply to every job of the batch."""
    x, y = synth.dot_uniform(50001, seed=9)
    p = T.params(panic_mode=T.PANIC_ULP, panic_ulps=0.25, leaf=100)
    j = B.dot_job(dev(x), dev(y))
    s = B.sum_job(dev(x))
    B.Batch([j, s], p=p, cfg=B.config(16, 4096, 128)).launch()
    e0, e1 = O.reduce(x, None, y, None, L=100)
    assert_bits(j.out[0], [e0], "z0")
    assert_bits(j.out[1], [e1], "z1")
    assert_flags(j.out[2], [O.flag(e0, e1, O.ULP, m=0.25)], "flag")
    e0, e1 = O.reduce(x, None, L=100)
    assert_bits(s.out[0], [e0], "sum z0")


def test_autotuner_choice_is_exact():
    jobs, ref = make_mix(4, njobs=24, big=False)
    cfg = B.tune(jobs, cands=[(32, 4096, 128), (256, 16384, 256)], reps=2)
    assert (cfg.leaves_per_item, cfg.points_per_item, cfg.threads) in [(32, 4096, 128), (256, 16384, 256)]
    assert B.tune(jobs) is not None                  # cached by signature
    B.Batch(jobs, cfg=cfg).launch()
    check(jobs, ref, "tuned")
