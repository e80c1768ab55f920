"""Parity of the CUDA transport path (through the C ABI) with the FP64 oracle.

Matched-stream runs (same seed) follow the same random numbers on both sides,
so histories coincide except where a last-bit difference between the GPU and
host libm flips a decision; unmatched runs are compared statistically with the
3-sigma / chi^2 acceptance of tests/parity.py.  Integer tallies of the GPU
are bit-reproducible (integer atomics commute), which the shard test checks.
"""
import math
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2503_10263_gb300 import inputs
from tests import closed_forms as cf
from tests import parity

pytestmark = pytest.mark.gpu

RAW = ("spectrum", "time_fx", "cross_pos", "cross_neg", "recomb", "ledger", "chan_count")


@pytest.fixture(scope="module")
def karl():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_10263_gb300 import karl as k
    return k


def _same_histories(g, o):
    return float(np.mean(g["per_primary"] == o["per_primary"]))


# ---------------------------------------------------------------------------
# config 1 (plain method, FP64): 1e4 beta electrons, 1000 segments, 4 channels

def test_config1_matched_streams(karl):
    prob, prims = inputs.config1()
    ctx = karl.Context(prob)
    g = ctx.run(prims, seed=1)
    o = oracle.run(prob, prims, seed=1, n_threads=8)
    assert parity.ledger_balances(g["ledger"])
    assert _same_histories(g, o) >= 0.995
    for k in ("spectrum", "cross_pos", "cross_neg"):
        z, p = parity.poisson_two_sample(g[k], o[k])
        assert parity.excursions_ok(z), k
        assert p > 0.01, k
    tg = g["time_fx"].astype(np.float64)
    to = o["time_fx"].astype(np.float64)
    assert np.abs(tg - to).sum() / to.sum() < 5e-3
    nc_g, nc_o = int(g["ledger"][karl.N_COLLISIONS]), int(o["ledger"][karl.N_COLLISIONS])
    assert abs(nc_g - nc_o) <= 0.005 * nc_o
    np.testing.assert_allclose(g["density"], o["density"], rtol=0.02, atol=1e-3 * o["density"].max())


def _batched(run_pass_fn, prims, k, seed, n_decays):
    edges = np.linspace(0, prims.n, k + 1).astype(int)
    out = {key: [] for key in ("spectrum", "time_fx", "cross_pos")}
    for a, b in zip(edges[:-1], edges[1:]):
        t = run_pass_fn(prims.slice(a, b - a), seed, a, n_decays)
        for key in out:
            out[key].append(t[key].astype(np.float64))
    return {key: np.stack(v) for key, v in out.items()}


def test_config1_independent_streams_statistical(karl):
    prob, prims = inputs.config1()
    ctx = karl.Context(prob)
    kb = 32
    gb = _batched(lambda p, s, off, nd: ctx.run_pass(p, s, 1, pid_offset=off, n_decays=nd),
                  prims, kb, 11, prims.n_decays)
    ob = _batched(lambda p, s, off, nd: oracle.run_pass(prob, p, s, 1, pid_offset=off,
                                                        n_decays=nd, n_threads=8),
                  prims, kb, 12, prims.n_decays)
    # spectra: Poisson on the summed counts
    z, p = parity.poisson_two_sample(gb["spectrum"].sum(0), ob["spectrum"].sum(0))
    assert parity.excursions_ok(z) and p > 0.01
    # time/density and crossings: one long random walk spans many adjacent
    # bins, so the bins are correlated; compare 10 z-groups of the 32
    # primary-id batches with Hotelling's T^2 (covariance from the batches)
    for key in ("time_fx", "cross_pos"):
        a = parity.coarse_groups(gb[key][:, 0].reshape(kb, -1), 10)
        b = parity.coarse_groups(ob[key][:, 0].reshape(kb, -1), 10)
        assert parity.hotelling_two_sample(a, b) > 0.01, key


# ---------------------------------------------------------------------------
# config 2 shape (two passes, ions, clustering, recombination), reduced decays

def test_config2_small_two_pass_matched(karl):
    prob, prims = inputs.config2(n_decays=3000, seed=2)
    ctx = karl.Context(prob)
    g = ctx.run(prims, seed=5)
    o = oracle.run(prob, prims, seed=5, n_threads=8)
    assert parity.ledger_balances(g["ledger"])
    assert _same_histories(g, o) >= 0.99
    # recombination target field (pass-1 densities) within 1e-3 relative L2
    assert parity.rel_l2(g["field"], o["field"]) < 1e-3
    for k in ("spectrum", "cross_pos"):
        z, p = parity.poisson_two_sample(g[k], o[k])
        assert parity.excursions_ok(z) and p > 0.01, k
    L = g["ledger"]
    assert L[karl.BIRTHS + inputs.T3P] > 0


def test_fp32_form_against_fp64_oracle(karl):
    prob, prims = inputs.config3()
    ctx = karl.Context(prob)
    kb = 32
    gb = _batched(lambda p, s, off, nd: ctx.run_pass(p, s, 1, pid_offset=off, n_decays=nd,
                                                     precision=karl.FP32),
                  prims, kb, 1, prims.n_decays)
    ob = _batched(lambda p, s, off, nd: oracle.run_pass(prob, p, s, 1, pid_offset=off,
                                                        n_decays=nd, n_threads=8),
                  prims, kb, 1, prims.n_decays)
    z, p = parity.poisson_two_sample(gb["spectrum"].sum(0), ob["spectrum"].sum(0))
    assert parity.excursions_ok(z) and p > 0.01
    a = parity.coarse_groups(gb["time_fx"][:, 0].reshape(kb, -1), 10)
    b = parity.coarse_groups(ob["time_fx"][:, 0].reshape(kb, -1), 10)
    assert parity.hotelling_two_sample(a, b) > 0.01
    # every bin of each tally: deviation of the FP32 form from the FP64 oracle
    # in standard errors of the 32 primary-id batches, 3-sigma excursions no
    # more than chance allows and chi^2 over the bins
    for key in ("time_fx", "cross_pos", "spectrum"):
        z, _ = parity.batch_two_sample(gb[key].reshape(kb, -1), ob[key].reshape(kb, -1))
        s = parity.deviation_summary(z, 2 * (kb - 1))
        print(f"PARITY config 3 FP32 {key}: bins {s['bins']}, median |z| {s['median_abs_z']:.3f}, "
              f"max |z| {s['max_abs_z']:.2f}, beyond 3 sigma {s['beyond_3']} "
              f"(chance allows {s['allowed_beyond_3']:.1f}), chi2 p {s['chi2_p']:.3g}")
        assert s["beyond_3"] <= s["allowed_beyond_3"] and s["chi2_p"] > 1e-3, key


# ---------------------------------------------------------------------------
# closed forms reproduced on the GPU

def test_gpu_beam_survival_closed_form(karl):
    rng = np.random.default_rng(7)
    nz, length, sigma = 40, 1.0, 1e-20
    n_seg = rng.uniform(0.0, 2.0, nz) * 1.5e20
    n_seg[5:8] = 0.0
    nodes = inputs.energy_nodes(64, 1.0, 2e4)
    ch = inputs.Channel("absorb", inputs.EXCITATION, 0, -1, 99.5, np.full_like(nodes, sigma))
    prob = inputs.uniform_problem(1.0, length, nz, [ch], n_energy=64)
    prob.n_seg_m3 = n_seg
    n = 400_000
    for prec in (karl.FP64, karl.FP32):
        g = karl.Context(prob).run(inputs.beam(n, 0.0, 100.0, 1.0), seed=3, precision=prec)
        emp = g["cross_pos"][0].astype(np.float64) / n
        surv = cf.survival_at_faces(n_seg, length / nz, sigma)
        assert np.max(np.abs(emp[1:] - surv[1:])) < 1.95 / math.sqrt(n)


@pytest.mark.parametrize("e_kev", [1.0, 5.0, 18.6])
def test_gpu_speed_is_relativistic_at_beta_energies(karl, e_kev):
    """Vacuum flights of beta-energy electrons: the time tally per segment is
    L / (|mu| v) with v = c sqrt(1 - 1/gamma^2) (Sec. 3.1's Lorentz factor),
    to one 2^-50 s unit per flight in FP64 and to FP32 rounding in the
    precision form."""
    from tests.test_oracle_pins import _absorber_problem, vacuum_time_units
    nz, length, n = 10, 1.0, 64
    prob = _absorber_problem(np.zeros(nz), length, 1e-20)
    for mu in (1.0, -0.37):
        z0 = 0.0 if mu > 0 else length
        q = vacuum_time_units(e_kev * 1e3, mu, length / nz)
        for prec, rel in ((karl.FP64, 1e-12), (karl.FP32, 2e-6)):
            g = karl.Context(prob).run(inputs.beam(n, z0, e_kev * 1e3, mu), seed=1, precision=prec)
            t = g["time_fx"][0, 1:-1, 0].astype(np.float64)
            tol = 0.5 * n + rel * n * q
            assert np.all(np.abs(t - n * q) <= tol), (prec, mu, t / n, q)


def test_gpu_channel_frequencies(karl):
    nodes = inputs.energy_nodes(2048, 1.0, 2e4)
    prob = inputs.uniform_problem(1e19, 1.0, 10, inputs.electron_channels(nodes, False),
                                  e_cut=100.0)
    n = 1_000_000
    e = np.array([100.0])
    sig = np.array([inputs.elastic_sigma(e)[0], inputs.born_bethe(e, 15.4, 4.2)[0],
                    inputs.born_bethe(e, 12.6, 1.6)[0], inputs.born_bethe(e, 0.5, 0.05)[0]])
    p = sig / sig.sum()
    for prec in (karl.FP64, karl.FP32):
        g = karl.Context(prob).run(inputs.beam(n, 0.5, 100.0, 0.0), seed=9, precision=prec)
        cnt = g["chan_count"].astype(np.float64)
        # an elastic recoil that rounds to zero leaves a particle at the cut:
        # rare second collisions, at the same energy and channel law
        tot = cnt.sum()
        assert n <= tot <= n + 10
        assert np.all(np.abs(cnt - tot * p) <= 4 * np.sqrt(tot * p * (1 - p)))
        assert parity.ledger_balances(g["ledger"])


# ---------------------------------------------------------------------------
# edge cases: exact agreement on deterministic outcomes

def test_edge_cases_exact(karl):
    nodes = inputs.energy_nodes(2048, 1.0, 2e4)
    n_seg = np.full(20, 1e19)
    n_seg[:5] = 0.0                           # vacuum at the left end
    prob = inputs.uniform_problem(1.0, 2.0, 20, inputs.electron_channels(nodes, False))
    prob.n_seg_m3 = n_seg
    z = np.array([0.0, 2.0, 0.3, 1.0, 0.0, 2.0, 0.05, 1.5])
    e = np.array([100.0, 100.0, 50.0, 0.5, 18000.0, 10.0, 20.0, 1.0])
    mu = np.array([-1.0, 1.0, 0.0, 0.3, 1.0, -1.0, 0.0, 1.0])
    prims = inputs.Primaries(z, e, mu, np.zeros(8, np.uint8), 8)
    ctx = karl.Context(prob)
    g = ctx.run(prims, seed=4)
    o = oracle.run(prob, prims, seed=4)
    for k in ("spectrum", "cross_pos", "cross_neg", "ledger", "chan_count", "per_primary"):
        np.testing.assert_array_equal(g[k], o[k], err_msg=k)
    L = g["ledger"]
    assert L[karl.DEATHS + 7] == 2             # two primaries with mu = 0 in vacuum: stalled
    assert L[karl.DEATHS + 2] >= 1             # 0.5 eV primary: cut at birth
    # empty run
    empty = inputs.Primaries(np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0, np.uint8), 1)
    t = ctx.run(empty, seed=1)
    assert t["ledger"].sum() == 0 and t["spectrum"].sum() == 0


def test_caps_match_oracle(karl):
    prob, prims = inputs.config2(n_decays=400, seed=3)
    prob.max_collisions = 25
    prob.max_lifetime_s = 2e-6
    g = karl.Context(prob).run(prims, seed=2)
    o = oracle.run(prob, prims, seed=2, n_threads=8)
    assert parity.ledger_balances(g["ledger"])
    assert _same_histories(g, o) >= 0.99
    for r in (3, 4):                           # collision cap, lifetime cap
        gs = g["ledger"][karl.DEATHS + r::8][:karl.N_SPECIES].sum()
        os_ = o["ledger"][karl.DEATHS + r::8][:karl.N_SPECIES].sum()
        assert gs > 0 and abs(int(gs) - int(os_)) <= max(3, 0.01 * os_)


# ---------------------------------------------------------------------------
# ABI behaviour

def test_invalid_primaries_rejected_and_context_survives(karl):
    prob, prims = inputs.config1(n_primaries=100)
    ctx = karl.Context(prob)
    bad = prims.slice(0, 100)
    bad.z_m[3] = prob.length_m + 1.0
    with pytest.raises(karl.KarlError) as ei:
        ctx.run(bad, seed=1)
    assert ei.value.status == karl.EINVAL
    bad.z_m[3] = 1.0
    bad.mu[7] = 1.5
    with pytest.raises(karl.KarlError):
        ctx.run(bad, seed=1)
    t = ctx.run(prims, seed=1)
    assert parity.ledger_balances(t["ledger"])


def test_timeout_returns_status_and_context_survives(karl):
    prob, prims = inputs.config2(n_decays=20000, seed=1)
    ctx = karl.Context(prob)
    with pytest.raises(karl.KarlError) as ei:
        ctx.run(prims, seed=1, timeout_s=1e-6)
    assert ei.value.status == karl.ETIMEOUT
    small = prims.slice(0, 200)
    t = ctx.run(small, seed=1)
    assert parity.ledger_balances(t["ledger"])


def test_cancel_from_another_thread(karl):
    prob, prims = inputs.config2(n_decays=300_000, seed=1)
    ctx = karl.Context(prob)
    err = {}

    def work():
        try:
            ctx.run(prims, seed=1)
        except karl.KarlError as e:
            err["status"] = e.status

    th = threading.Thread(target=work)
    th.start()
    time.sleep(0.3)
    ctx.cancel()
    th.join(timeout=120)
    assert not th.is_alive()
    assert err.get("status") == karl.ECANCELLED
    t = ctx.run(prims.slice(0, 100), seed=1)
    assert parity.ledger_balances(t["ledger"])


def test_shards_sum_to_single_run_bit_exact(karl):
    prob, prims = inputs.config2(n_decays=2000, seed=4)
    ctx = karl.Context(prob)
    full = ctx.run(prims, seed=3)
    cuts = [0, 1111, 2500, prims.n]
    p1 = [ctx.run_pass(prims.slice(a, b - a), 3, 1, pid_offset=a, n_decays=prims.n_decays)
          for a, b in zip(cuts[:-1], cuts[1:])]
    time1 = sum(t["time_fx"] for t in p1)
    p2 = [ctx.run_pass(prims.slice(a, b - a), 3, 2, field_time_in=time1, pid_offset=a,
                       n_decays=prims.n_decays) for a, b in zip(cuts[:-1], cuts[1:])]
    p2[0]["ledger"][karl.N_COLLISIONS_ALL:karl.N_FLIGHTS_ALL + 1] += \
        sum(t["ledger"][karl.N_COLLISIONS_ALL:karl.N_FLIGHTS_ALL + 1] for t in p1)
    for k in RAW:
        np.testing.assert_array_equal(sum(t[k] for t in p2), full[k], err_msg=k)
    again = ctx.run(prims, seed=3)
    for k in RAW + ("per_primary",):
        np.testing.assert_array_equal(again[k], full[k], err_msg=k)


def test_device_buffers_match_host_buffers(karl):
    import torch
    prob, prims = inputs.config1(n_primaries=2000)
    ctx = karl.Context(prob)
    host = ctx.run(prims, seed=7)
    dev = torch.device("cuda:0")
    pt = {"z_m": torch.tensor(prims.z_m, device=dev), "e_ev": torch.tensor(prims.e_ev, device=dev),
          "mu": torch.tensor(prims.mu, device=dev),
          "species": torch.tensor(prims.species, device=dev)}
    t = ctx.empty_tallies(prims.n)
    dt = {k: torch.zeros(v.shape, dtype=torch.float64 if v.dtype == np.float64 else torch.int64,
                         device=dev) for k, v in t.items()}
    ctx.run_device({k: v.data_ptr() for k, v in pt.items()}, prims.n, prims.n_decays,
                   {k: v.data_ptr() for k, v in dt.items()}, seed=7)
    torch.cuda.synchronize()
    for k in RAW + ("per_primary",):
        got = dt[k].cpu().numpy().view(host[k].dtype if host[k].dtype != np.float64 else np.float64)
        np.testing.assert_array_equal(got.reshape(-1)[:host[k].size], host[k].reshape(-1), err_msg=k)
