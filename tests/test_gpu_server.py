"""Batched and served forms: many source configurations in one persistent
launch.  Each request's random streams are keyed by its seed and primary ids
only, and integer tallies commute, so a request's tallies must equal the
single-run path's bit for bit -- alone, in a mixed batch, under admission by
a small HBM budget, and when submitted while other requests are running."""
import time

import numpy as np
import pytest

from paper_2503_10263_gb300 import inputs
from tests import parity

pytestmark = pytest.mark.gpu

INT_KEYS = ("spectrum", "time_fx", "cross_pos", "cross_neg", "recomb", "ledger", "chan_count")
FLOAT_KEYS = ("density", "current", "field")


@pytest.fixture(scope="module")
def karl():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_10263_gb300 import karl as k
    return k


def _requests(n=8, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        col = rng.uniform(0.1, 1.0) * 5e21
        length = rng.uniform(2.0, 10.0)
        nd = int(rng.integers(50, 1500))
        n0 = inputs.parabolic_n0(col, length)
        prob = inputs._problem(f"r{i}", length, 1000,
                               inputs.parabolic_segment_means(n0, length, 1000), full=True)
        out.append((prob, inputs.decay_primaries(prob, nd, 100 + i), 7000 + i))
    return out


def _single(karl, prob, prims, seed, prec):
    return karl.Context(prob).run(prims, seed=seed, precision=prec, per_primary=False)


def _same(a, b):
    for k in INT_KEYS:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    for k in FLOAT_KEYS:
        np.testing.assert_allclose(a[k], b[k], rtol=1e-12, atol=0, err_msg=k)


@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
def test_batch_equals_single_runs(karl, prec_name):
    prec = karl.FP32 if prec_name == "fp32" else karl.FP64
    reqs = _requests()
    srv = karl.Server(reqs[0][0], precision=prec, hbm_budget_bytes=4 << 30, timeout_s=120)
    ids = [srv.submit(p, pr, s) for p, pr, s in reqs]
    srv.run_all()
    st = srv.stats()
    assert st.kernel_launches == 1                # the whole batch in one persistent launch
    for (p, pr, s), rid in zip(reqs, ids):
        done, t = srv.poll(rid)
        assert done
        assert parity.ledger_balances(t["ledger"])
        _same(t, _single(karl, p, pr, s, prec))
    srv.close()


def test_alone_and_in_the_mix(karl):
    reqs = _requests(6, seed=9)
    p, pr, s = reqs[2]
    alone = karl.Server(p, hbm_budget_bytes=1 << 30, timeout_s=120)
    rid = alone.submit(p, pr, s)
    alone.run_all()
    _, ta = alone.poll(rid)
    alone.close()
    mix = karl.Server(p, hbm_budget_bytes=2 << 30, timeout_s=120)
    ids = [mix.submit(q, qr, qs) for q, qr, qs in reqs]
    mix.run_all()
    _, tm = mix.poll(ids[2])
    mix.close()
    _same(ta, tm)


def test_admission_by_footprint(karl):
    reqs = _requests(6, seed=11)
    # budget for about two requests at a time: the rest wait and join later
    srv = karl.Server(reqs[0][0], hbm_budget_bytes=48 << 20, timeout_s=120)
    ids = [srv.submit(p, pr, s) for p, pr, s in reqs]
    st0 = srv.stats()
    assert st0.waiting > 0
    srv.run_all()
    for (p, pr, s), rid in zip(reqs, ids):
        done, t = srv.poll(rid)
        assert done
        _same(t, _single(karl, p, pr, s, karl.FP64))
    assert srv.stats().arena_bytes_peak <= 48 << 20
    srv.close()


def test_served_requests_join_the_running_launch(karl):
    reqs = _requests(8, seed=5)
    srv = karl.Server(reqs[0][0], hbm_budget_bytes=4 << 30, timeout_s=120)
    results = {}
    ids = {}
    t0 = time.time()
    for i, (p, pr, s) in enumerate(reqs):
        ids[i] = srv.submit(p, pr, s)
        time.sleep(0.005)
        for j, rid in list(ids.items()):
            if j not in results:
                done, t = srv.poll(rid)
                if done:
                    results[j] = t
    while len(results) < len(reqs):
        assert time.time() - t0 < 120
        for j, rid in ids.items():
            if j not in results:
                done, t = srv.poll(rid)
                if done:
                    results[j] = t
        time.sleep(0.001)
    assert srv.stats().kernel_launches == 1       # continuous: one launch served them all
    srv.run_all()                                 # close the session
    srv.close()
    for i, (p, pr, s) in enumerate(reqs):
        _same(results[i], _single(karl, p, pr, s, karl.FP64))


def test_empty_request_and_invalid_submit(karl):
    reqs = _requests(2, seed=1)
    p, pr, s = reqs[0]
    srv = karl.Server(p, hbm_budget_bytes=1 << 30, timeout_s=60)
    empty = inputs.Primaries(np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0, np.uint8), 10)
    rid = srv.submit(p, empty, 1)
    bad = pr.slice(0, 10)
    bad.mu[0] = 2.0
    with pytest.raises(karl.KarlError):
        srv.submit(p, bad, 1)
    srv.run_all()
    done, t = srv.poll(rid)
    assert done and t["ledger"].sum() == 0 and not t["density"].any()
    with pytest.raises(karl.KarlError):
        srv.poll(rid)                              # already collected
    srv.close()


@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
def test_many_small_requests_all_finish(karl, prec_name):
    # many short two-pass requests in one launch: many pass transitions race
    # with warps claiming primaries; every request must finish and equal its
    # single run
    prec = karl.FP32 if prec_name == "fp32" else karl.FP64
    rng = np.random.default_rng(21)
    reqs = []
    for i in range(48):
        col = rng.uniform(0.1, 1.0) * 5e21
        length = rng.uniform(2.0, 10.0)
        n0 = inputs.parabolic_n0(col, length)
        prob = inputs._problem(f"s{i}", length, 100, inputs.parabolic_segment_means(n0, length, 100),
                               full=True)
        reqs.append((prob, inputs.decay_primaries(prob, int(rng.integers(5, 60)), 300 + i), 900 + i))
    for rep in range(3):
        srv = karl.Server(reqs[0][0], precision=prec, hbm_budget_bytes=2 << 30, timeout_s=30)
        ids = [srv.submit(p, pr, s) for p, pr, s in reqs]
        srv.run_all()
        for (p, pr, s), rid in zip(reqs, ids):
            done, t = srv.poll(rid)
            assert done
            if rep == 0:
                _same(t, _single(karl, p, pr, s, prec))
        srv.close()


def test_contexts_come_and_go_during_a_served_launch(karl):
    # A served launch holds the device until its session closes.  A context
    # made before it and destroyed while it runs (by a destructor, say), and
    # a context created meanwhile, must not wait for it: a device-wide
    # synchronising free there would stall the host until the launch's
    # deadline while the launch waits for the host.
    reqs = _requests(2, seed=5)
    p, pr, s = reqs[0]
    old = karl.Context(p)
    srv = karl.Server(p, hbm_budget_bytes=1 << 30, timeout_s=30)
    try:
        rid = srv.submit(p, pr, s)              # admitted: the launch starts and stays up
        t0 = time.time()
        old.close()
        new = karl.Context(p)
        new.close()
        dt = time.time() - t0
        srv.run_all()
        done, t = srv.poll(rid)
    finally:
        srv.close()
    assert done and parity.ledger_balances(t["ledger"])
    assert dt < 5.0, dt
