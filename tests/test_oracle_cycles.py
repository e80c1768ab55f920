"""Pins of the oracle's continuous field update (Sec. 3.6: cycles, each with
the density fields of the cycles before it; Eq. target_field_density with
its deletion term and Eq. simulated_time).  Closed forms: beam survival
through a field given by its time and deletion tallies -- the ion density
minus deletions for an electron beam, the electron field's per-bin densities
(deletions shared by time) weighted by sigma v for an ion beam, negative
densities counting as zero -- and exact invariance of the cycle split."""
import math

import numpy as np
import pytest

import oracle
from paper_2503_10263_gb300 import inputs
from tests import closed_forms as cf

THREADS = 8
Q_T = 2.0**50


def _field_problem(ntb=1, e_min=1.0, e_max=2e4):
    nodes = inputs.energy_nodes(64, e_min, e_max)
    sig = 1e-18
    chans = [inputs.Channel("e+T3", inputs.RECOMBINATION, inputs.E, inputs.T3P, 0.0,
                            np.full_like(nodes, sig)),
             inputs.Channel("T3+e", inputs.RECOMBINATION, inputs.T3P, inputs.E, 0.0,
                            np.full_like(nodes, sig))]
    prob = inputs.uniform_problem(0.0, 2.0, 20, chans, n_energy=64, e_min=e_min, e_max=e_max,
                                  e_cut=0.0, n_tebins=ntb)
    prob.activity_bq = 1e18
    return prob, sig


def test_electron_beam_through_ion_field_with_deletions():
    # ion (T3+) time and deletions per segment chosen so that the density
    # sum t / (t_sim V) - N / V is known, and negative in two segments
    prob, sig = _field_problem()
    nz, dz = prob.n_zbins, prob.length_m / prob.n_zbins
    vol = dz * prob.area_m2
    decays = 1000.0
    tsim = decays / prob.activity_bq
    rng = np.random.default_rng(4)
    n_time = rng.uniform(2e17, 8e17, nz)                   # sum t / (t_sim V)
    dels = np.zeros(nz, np.uint64)
    dels[5] = np.uint64(round(0.4e17 * vol))                # partly cancelled
    dels[11] = np.uint64(round(2e18 * vol))                 # below zero: no field
    dels[12] = np.uint64(round(9e17 * vol))
    t_in = np.zeros((inputs.N_SPECIES, nz + 2, 1), np.uint64)
    t_in[inputs.T3P, 1:nz + 1, 0] = np.round(n_time * tsim * vol * Q_T).astype(np.uint64)
    r_in = np.zeros((inputs.N_SPECIES, nz), np.uint64)
    r_in[inputs.T3P] = dels
    n_exact = t_in[inputs.T3P, 1:nz + 1, 0].astype(np.float64) / Q_T / (tsim * vol)
    field = np.maximum(n_exact - dels.astype(np.float64) / vol, 0.0)
    n = 100_000
    r = oracle.run_cycle(prob, inputs.beam(n, 0.0, 1000.0, 1.0), 31, t_in, r_in, decays,
                         n_threads=THREADS)
    surv = r["cross_pos"][inputs.E].astype(np.float64) / n
    expect = cf.survival_at_faces(field, dz, sig)
    assert np.max(np.abs(surv[1:] - expect[1:])) < 1.95 / math.sqrt(n)
    assert r["recomb"][inputs.T3P][11] == 0 and r["recomb"][inputs.T3P][12] == 0


def test_ion_beam_through_electron_field_shares_deletions_by_time():
    # electron time in two energy bins; the segment's deletions are shared in
    # proportion to time; the ion rate is sum_b n_b sigma v(E_b) / v_ion
    ntb = 4
    prob, sig = _field_problem(ntb=ntb, e_min=1.0, e_max=1e4)
    nz, dz = prob.n_zbins, prob.length_m / prob.n_zbins
    vol = dz * prob.area_m2
    decays = 500.0
    tsim = decays / prob.activity_bq
    eb = prob.e_min_ev * (prob.e_max_ev / prob.e_min_ev) ** ((np.arange(ntb) + 0.5) / ntb)
    vb = np.array([cf.speed(e, inputs.ME_EV) for e in eb])
    dens = np.zeros((nz, ntb))
    dens[:, 1] = 3e13
    dens[:, 3] = 1e13
    dels = np.zeros(nz)
    dels[3:8] = 2e13 * vol                                  # shared 3 : 1 between the bins
    dels[15] = 9e13 * vol                                   # more than there is
    t_in = np.zeros((inputs.N_SPECIES, nz + 2, ntb), np.uint64)
    t_in[inputs.E, 1:nz + 1, :] = np.round(dens * tsim * vol * Q_T).astype(np.uint64)
    r_in = np.zeros((inputs.N_SPECIES, nz), np.uint64)
    r_in[inputs.E] = np.round(dels).astype(np.uint64)
    tt = t_in[inputs.E, 1:nz + 1, :].astype(np.float64)
    share = tt / tt.sum(axis=1, keepdims=True)
    nb = np.maximum(tt / Q_T / (tsim * vol) - (r_in[inputs.E].astype(np.float64) / vol)[:, None]
                    * share, 0.0)
    e_ion = 0.05
    v_ion = cf.speed(math.floor(e_ion * 2**24) / 2**24, inputs.M_T3P_EV)
    rate = (nb * sig * vb[None, :]).sum(axis=1) / v_ion      # per unit path
    n = 100_000
    r = oracle.run_cycle(prob, inputs.beam(n, 0.0, e_ion, 1.0, inputs.T3P), 32, t_in, r_in,
                         decays, n_threads=THREADS)
    surv = r["cross_pos"][inputs.T3P].astype(np.float64) / n
    expect = np.exp(-np.concatenate([[0.0], np.cumsum(rate) * dz]))
    assert np.max(np.abs(surv[1:] - expect[1:])) < 1.95 / math.sqrt(n)
    assert expect[-1] < 0.8                                 # the field matters


def test_cycle_split_is_exact_without_recombination():
    # no recombination channel: the fields do nothing, so any split into
    # cycles gives the tallies of one cycle over all primaries, bit for bit
    prob, prims = inputs.config1(n_primaries=3000, density_m3=3e19)
    one = oracle.run_cycle(prob, prims, 41, None, None, 0.0, n_threads=THREADS)
    for c in (1, 3, 7):
        many = oracle.run_cycles(prob, prims, 41, c, n_threads=THREADS)
        for k in oracle.RAW_KEYS:
            np.testing.assert_array_equal(many[k], one[k], err_msg=f"{c} {k}")
        np.testing.assert_array_equal(many["per_primary"], one["per_primary"])


def test_cycles_conserve_and_feed_back():
    # config-2 physics in cycles: exact ledgers, finite non-negative fields,
    # and the later cycles recombine (the fields come from earlier cycles)
    prob, prims = inputs.config2(n_decays=2000, seed=4, column_m2=2e21, length=4.0, nz=100)
    prob.activity_bq *= 1e9                                  # dense fields: recombination matters
    r = oracle.run_cycles(prob, prims, 43, 4, n_threads=THREADS)
    L = r["ledger"]
    ns = oracle.N_SPECIES
    assert L[oracle.E_IN_PRIMARY] + L[oracle.E_IN_THERMAL] == L[oracle.E_EXIT0:oracle.E_STALLED + 1].sum()
    births = L[oracle.BIRTHS:oracle.BIRTHS + ns]
    deaths = L[oracle.DEATHS:oracle.DEATHS + 8 * ns].reshape(ns, 8).sum(axis=1)
    np.testing.assert_array_equal(births, deaths)
    assert np.all(np.isfinite(r["field"])) and np.all(r["field"] >= 0)
    assert int(np.sum(r["recomb"])) > 0
    # the first cycle alone (fields of zero) does not recombine
    first = oracle.run_cycle(prob, prims.slice(0, prims.n // 4), 43, None, None, 0.0,
                             n_threads=THREADS)
    assert int(np.sum(first["recomb"])) == 0
