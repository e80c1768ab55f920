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


def _tiny_requests(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        col = rng.uniform(0.1, 1.0) * 5e21
        length = rng.uniform(0.5, 2.0)
        n0 = inputs.parabolic_n0(col, length)
        prob = inputs._problem(f"t{i}", length, 50, inputs.parabolic_segment_means(n0, length, 50),
                               full=True)
        out.append((prob, inputs.decay_primaries(prob, int(rng.integers(1, 12)), 500 + i),
                    4000 + i))
    return out


@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
def test_slots_recycled_quickly_in_a_running_launch(karl, prec_name):
    """Two slots and 96 tiny two-pass requests, all submitted at once and
    collected by polling while the launch keeps running: each slot is reused
    about 48 times, so warps scanning for primaries keep meeting slots whose
    request has just finished and been replaced.  A claim must only ever take
    primaries of the request (generation) whose state it read; every result
    equals its single run bit for bit."""
    prec = karl.FP32 if prec_name == "fp32" else karl.FP64
    reqs = _tiny_requests(96, seed=33)
    srv = karl.Server(reqs[0][0], precision=prec, max_slots=2, hbm_budget_bytes=1 << 30,
                      timeout_s=60)
    ids = [srv.submit(p, pr, s) for p, pr, s in reqs]
    assert srv.stats().waiting == len(reqs) - 2
    results = {}
    t0 = time.time()
    while len(results) < len(reqs):
        assert time.time() - t0 < 60
        for j, rid in enumerate(ids):
            if j not in results:
                done, t = srv.poll(rid)
                if done:
                    results[j] = t
        time.sleep(0.0005)
    st = srv.stats()
    srv.run_all()
    srv.close()
    assert st.completed == len(reqs)
    for i, (p, pr, s) in enumerate(reqs):
        assert parity.ledger_balances(results[i]["ledger"])
        _same(results[i], _single(karl, p, pr, s, prec))


def test_served_request_matches_oracle(karl):
    """A request served in a mix follows the FP64 oracle's histories: same
    tallies in law and the same recombination target field (within 1e-3
    relative L2) -- not only the single-run CUDA path's."""
    import oracle
    reqs = _requests(5, seed=13)
    p, pr, s = reqs[1]
    srv = karl.Server(p, hbm_budget_bytes=2 << 30, timeout_s=120)
    ids = [srv.submit(q, qr, qs) for q, qr, qs in reqs]
    srv.run_all()
    _, t = srv.poll(ids[1])
    srv.close()
    o = oracle.run(p, pr, seed=s, n_threads=8)
    assert parity.ledger_balances(t["ledger"])
    assert parity.rel_l2(t["field"], o["field"]) < 1e-3
    nc_g, nc_o = int(t["ledger"][karl.N_COLLISIONS_ALL]), int(o["ledger"][oracle.N_COLLISIONS_ALL])
    assert abs(nc_g - nc_o) <= 2e-3 * nc_o, (nc_g, nc_o)
    for k in ("spectrum", "cross_pos", "cross_neg"):
        z, pv = parity.poisson_two_sample(t[k], o[k])
        assert parity.excursions_ok(z) and pv > 0.01, k
    # matched streams: the channel counts of the last pass agree closely
    cg, co = t["chan_count"].astype(np.float64), o["chan_count"].astype(np.float64)
    assert np.all(np.abs(cg - co) <= 4 * np.sqrt(np.maximum(cg + co, 1.0)) + 0.002 * co)


def test_autotune_times_every_candidate_shape(karl, tmp_path, monkeypatch):
    """The autotuner launches the multi-request kernel with each candidate
    shape and caches a valid one."""
    from paper_2503_10263_gb300 import autotune
    monkeypatch.setenv("KARL_CACHE_DIR", str(tmp_path))
    batch = inputs.config4_batch(n_configs=3, meta_seed=5, np_lo=200, np_hi=400)
    for prec in (karl.FP64, karl.FP32):
        shape = autotune.tune(prec, force=True, batch=batch)
        assert shape in autotune.CANDIDATES
        assert autotune.tune(prec) == shape                  # served from the cache
