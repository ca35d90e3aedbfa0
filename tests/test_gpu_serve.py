"""The request server (C ABI twofold_server_*): every request's results are
the single-job entry point's bits on the same inputs, whether it runs alone
or in a mix submitted concurrently from several threads; admission by
device memory completes a stream of requests larger than the arena, and a
request larger than the whole arena fails with TF_ENOSPC."""
import threading

import numpy as np
import pytest

import oracle as O
import paper_1401_6235_gb300 as T
import synth
from paper_1401_6235_gb300.serve import Server
from tests.fp import rand_tails
from tests.gpu_util import assert_bits, assert_flags, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as e
    e.build()


def make_requests(seed, count=48):
    """(kind, args) with host arrays, and the single-job device reference."""
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        kind = ["sum", "dot", "horner", "ew"][i % 4]
        n = int([0, 1, 257, 5000, 65536, 300001][rng.integers(6)]) if kind != "horner" or i % 8 else 0
        if kind == "horner":
            k = int(rng.integers(0, 31))
            a = synth.binomial_coefs(k)
            x = synth.horner_points(n, seed=seed * 100 + i)
            reqs.append((kind, (a, x)))
        elif kind == "ew":
            d = synth.ew_chain(n, seed=seed * 100 + i)
            reqs.append((kind, ([(d[c + "0"], d[c + "1"]) for c in "abcd"],)))
        else:
            x, y = synth.dot_uniform(n, seed=seed * 100 + i)
            xl = rand_tails(np.random.default_rng(i), x, 30, 60) if (i % 3 == 0 and n) else None
            reqs.append((kind, (x, xl, y)))
    return reqs


def submit(srv, kind, args):
    if kind == "sum":
        return srv.submit_sum(args[0], args[1])
    if kind == "dot":
        return srv.submit_dot(args[0], args[2], args[1])
    if kind == "horner":
        return srv.submit_horner(args[0], args[1])
    return srv.submit_ew(T.CHAIN_SQRT_MAD_DIV, args[0])


def single_job(kind, args):
    if kind == "sum":
        x, xl, _ = args
        return [host(t) for t in T.twofold_sum(dev(x), None if xl is None else dev(xl))]
    if kind == "dot":
        x, xl, y = args
        return [host(t) for t in T.twofold_dot(dev(x), dev(y), None if xl is None else dev(xl))]
    if kind == "horner":
        a, x = args
        if x.size == 0:
            return [np.empty(0), np.empty(0), np.empty(0, np.uint8)]
        return [host(t) for t in T.twofold_horner(dev(a), dev(x))]
    ins = [(dev(h), dev(lo)) for h, lo in args[0]]
    if ins[0][0].numel() == 0:
        return [np.empty(0), np.empty(0), np.empty(0, np.uint8)]
    return [host(t) for t in T.twofold_ew(T.CHAIN_SQRT_MAD_DIV, ins)]


def same(a, b, what):
    for u, v, name in zip(a, b, ("z0", "z1", "flags")):
        assert u.shape == v.shape, (what, name, u.shape, v.shape)
        if name == "flags":
            assert np.array_equal(u, v), (what, name)
        else:
            assert_bits(u, v, f"{what} {name}")


def test_results_alone_and_in_a_concurrent_mix():
    reqs = make_requests(1)
    ref = [single_job(k, a) for k, a in reqs]
    with Server(mem_cap=256 << 20, max_batch_jobs=64) as srv:
        alone = []
        for k, a in reqs:                       # one at a time
            t = submit(srv, k, a)
            alone.append([np.copy(o) for o in srv.wait(t)])
        # the same requests from four threads at once
        tickets = [None] * len(reqs)

        def client(c):
            for i in range(c, len(reqs), 4):
                tickets[i] = submit(srv, *reqs[i])
        th = [threading.Thread(target=client, args=(c,)) for c in range(4)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        mixed = [[np.copy(o) for o in srv.wait(t)] for t in tickets]
        st = srv.stats()
    for i, (r, a, m) in enumerate(zip(ref, alone, mixed)):
        same(a, r, f"alone {i} {reqs[i][0]}")
        same(m, r, f"mixed {i} {reqs[i][0]}")
    assert st["completed"] == 2 * len(reqs) and st["failed"] == 0
    assert st["batched_jobs"] == 2 * len(reqs)


def test_oracle_parity_of_served_dot_and_chain():
    x, y = synth.dot_uniform(100003, seed=3)
    d = synth.ew_chain(20011, seed=4)
    ins = [(d[c + "0"], d[c + "1"]) for c in "abcd"]
    with Server(mem_cap=64 << 20) as srv:
        t1 = srv.submit_dot(x, y)
        t2 = srv.submit_ew(T.CHAIN_SQRT_MAD_DIV, ins)
        z = srv.wait(t1)
        w = srv.wait(t2)
    e0, e1 = O.reduce(x, None, y, None)
    assert_bits(z[0], [e0], "dot z0")
    assert_bits(z[1], [e1], "dot z1")
    assert_flags(z[2], [O.flag(e0, e1)], "dot flag")
    r0, r1, rf = O.ew(T.CHAIN_SQRT_MAD_DIV, ins)
    assert_bits(w[0], r0, "chain z0")
    assert_bits(w[1], r1, "chain z1")
    assert_flags(w[2], rf, "chain flags")


def test_admission_by_memory():
    """An 8 MiB arena and 40 dots of 4 MiB of inputs each: at most one runs at
    a time, all complete with the right bits; a request larger than the arena
    fails with TF_ENOSPC and the server keeps serving."""
    n = 1 << 18
    xs = [synth.dot_uniform(n, seed=50 + i) for i in range(40)]
    with Server(mem_cap=8 << 20, max_batch_jobs=16) as srv:
        ts = [srv.submit_dot(x, y) for x, y in xs]
        big = srv.submit_sum(np.ones(2 << 20))
        after = srv.submit_sum(np.ones(1000))
        res = [srv.wait(t) for t in ts]
        with pytest.raises(T.TwofoldError) as ei:
            srv.wait(big)
        assert ei.value.status == T.TF_ENOSPC
        assert srv.wait(after)[0][0] == 1000.0
        st = srv.stats()
    assert st["peak_bytes"] <= 8 << 20
    for (x, y), z in zip(xs[:5], res[:5]):
        e0, e1 = O.reduce(x, None, y, None)
        assert_bits(z[0], [e0], "z0")
        assert_bits(z[1], [e1], "z1")


def test_batches_stay_within_a_quarter_of_the_arena():
    """A long queue of 1 MiB requests in a 64 MiB arena: no batch takes more
    than 16 MiB of request buffers, so several batches are in flight."""
    xs = [np.full(1 << 17, float(i)) for i in range(200)]
    with Server(mem_cap=64 << 20, max_batch_jobs=4096) as srv:
        ts = [srv.submit_sum(x) for x in xs]
        res = [srv.wait(t) for t in ts]
        st = srv.stats()
    assert max(t.info.batch_jobs for t in ts) <= 15
    assert st["completed"] == 200
    for i, z in enumerate(res):
        assert z[0][0] == float(i) * (1 << 17) and z[1][0] == 0.0


def test_wait_rejects_unknown_ticket():
    with Server(mem_cap=1 << 20) as srv:
        t = srv.submit_sum(np.ones(10))
        srv.wait(t)
        assert T.lib().twofold_server_wait(srv._h, t.id, 0, None) == T.TF_EINVAL    # already collected


def test_wait_timeout_keeps_the_ticket():
    """A wait that runs out returns TF_ETIMEOUT and leaves the ticket valid:
    a later wait collects the result (a 2^26-element chain, whose inputs
    take milliseconds to cross the host link)."""
    n = 1 << 26
    d = synth.ew_chain(n, seed=12)
    ins = [(d[c + "0"], d[c + "1"]) for c in "abcd"]
    with Server(mem_cap=8 << 30) as srv:
        t = srv.submit_ew(T.CHAIN_SQRT_MAD_DIV, ins)
        first = srv.wait(t, timeout_ms=0)
        assert first is None and t.status == T.TF_ETIMEOUT
        z = srv.wait(t)
        assert t.status == T.TF_OK
    idx = np.r_[0:1000, n - 1000:n]
    r0, r1, rf = O.ew(T.CHAIN_SQRT_MAD_DIV, [(h[idx], lo[idx]) for h, lo in ins])
    assert_bits(z[0][idx], r0, "z0")
    assert_bits(z[1][idx], r1, "z1")
    assert_flags(z[2][idx], rf, "flags")


def test_injected_batch_failures_are_reported_and_the_server_recovers():
    """Host-side fault injection (no device fault): with every second batch
    failed before it runs, requests submitted one at a time (one batch each)
    alternate between TF_ECUDA and the oracle's bits; the failures are
    counted, their memory comes back, and with injection off every later
    request completes correctly."""
    x, y = synth.dot_uniform(65537, seed=21)
    e0, e1 = O.reduce(x, None, y, None)
    with Server(mem_cap=16 << 20) as srv:
        srv.inject_failures(2)
        outcomes = []
        for _ in range(6):
            t = srv.submit_dot(x, y)
            try:
                z = srv.wait(t)
                assert_bits(z[0], [e0], "z0")
                assert_bits(z[1], [e1], "z1")
                outcomes.append(T.TF_OK)
            except T.TwofoldError as err:
                assert err.status == T.TF_ECUDA
                outcomes.append(err.status)
        assert outcomes == [T.TF_OK, T.TF_ECUDA] * 3, outcomes
        st = srv.stats()
        assert st["failed"] == 3 and st["completed"] == 3, st
        srv.inject_failures(0)
        for _ in range(4):
            z = srv.wait(srv.submit_dot(x, y))
            assert_bits(z[0], [e0], "z0 after")
            assert_bits(z[1], [e1], "z1 after")
        st = srv.stats()
        assert st["failed"] == 3 and st["completed"] == 7, st
    with pytest.raises(T.TwofoldError):
        Server(mem_cap=1 << 20).inject_failures(-1)
