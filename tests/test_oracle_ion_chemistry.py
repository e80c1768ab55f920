"""Pins of the oracle's ion chemistry (Sec. 3.3 Clustering, Charge exchange,
Ionization; Sec. 4 Clustering and Charge Exchange test cases): three-body and
rate-coefficient clustering of T+ against the exponential attenuation of the
paper's test (inferred rate coefficients within 1 %), the n(z)^2 column of
three-body clustering through a density gradient, the energy after one and
after many charge exchanges against quadrature of the relative-speed-weighted
Maxwellian, and the T+ product of dissociative ionization."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2503_10263_gb300 import inputs
from tests import closed_forms as cf

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_test_cases.json")))
THREADS = min(8, os.cpu_count() or 1)
KB = 8.617333262e-5


def _quant(e):
    return math.floor(e * 2**24) / 2**24


_ion_problem = inputs.ion_beam_problem
_cx_problem = inputs.charge_exchange_problem


def _attenuation(prob, r, n, lam, length, sp):
    nz = prob.n_zbins
    z = np.linspace(0.0, length, nz + 1)
    emp = r["cross_pos"][sp].astype(np.float64) / n
    assert np.max(np.abs(emp[1:] - np.exp(-z[1:] / lam))) < 1.95 / math.sqrt(n)


# ---------------------------------------------------------------------------
# Sec. 4 clustering of T+: lambda = v / (k_ter n^2) (Eq.
# clustering_test_tertiary_mfp) and lambda = v / (k_rad n) (Eq.
# clustering_test_radiative_rateCoefficient)

@pytest.mark.parametrize("case", ["clustering_tp_tertiary", "clustering_tp_radiative"])
def test_tp_clustering_attenuation_and_inferred_rate(case):
    g = GOLD[case]
    e0 = g["e_ion_ev"]
    nodes = inputs.energy_nodes(64, e0, 10.0)                 # e0 is node 0
    three = case.endswith("tertiary")
    k = g["k_m6ps"] if three else g["k_m3ps"]
    kind = inputs.CLUSTERING3 if three else inputs.CLUSTERING
    ch = inputs.Channel("clust", kind, inputs.TP, inputs.T3P, 0.0,
                        inputs.rate_sigma(nodes, k, inputs.M_TP_EV))
    nm = g["n_m3"]
    v_table = cf.speed(e0, inputs.M_TP_EV)
    lam = v_table / (k * nm ** (2 if three else 1))
    length, nz = 8.0 * lam, 40
    prob = _ion_problem([ch], np.full(nz, nm), length, e0, 10.0)
    n = g["n_events"]
    r = oracle.run(prob, inputs.beam(n, 0.0, e0, 1.0, inputs.TP), seed=13, n_threads=THREADS)
    _attenuation(prob, r, n, lam, length, inputs.TP)
    # maximum-likelihood rate coefficient: clusterings / (T+ time x n^order)
    time = r["time_fx"][inputs.TP].astype(np.float64).sum() / 2**50
    count = int(r["chan_count"][0])
    k_hat = count / time / nm ** (2 if three else 1)
    assert k_hat * cf.speed(_quant(e0), inputs.M_TP_EV) / v_table == \
        pytest.approx(k, rel=g["rel_err"], abs=0)
    L = r["ledger"]
    assert L[oracle.DEATHS + inputs.TP * 8 + 6] == count          # T+ consumed
    assert L[oracle.BIRTHS + inputs.T3P] == count                 # one T3+ each


def test_three_body_rate_follows_density_squared():
    # beam survival through a density ramp: exp(-s3 sum_j n_j^2 dz) at every face
    nz, length = 40, 1.0
    n_seg = np.linspace(2e21, 2e22, nz)
    dz = length / nz
    s3 = 1.0 / float(np.sum(n_seg ** 2) * dz)                   # optical depth 1 in total
    nodes = inputs.energy_nodes(64, 1e-3, 10.0)
    ch = inputs.Channel("clust3", inputs.CLUSTERING3, inputs.TP, inputs.T3P, 0.0,
                        np.full_like(nodes, s3))
    prob = _ion_problem([ch], n_seg, length, 1e-3, 10.0)
    n = 100_000
    r = oracle.run(prob, inputs.beam(n, 0.0, 0.05, 1.0, inputs.TP), seed=14, n_threads=THREADS)
    col2 = np.concatenate([[0.0], np.cumsum(n_seg ** 2) * dz])
    emp = r["cross_pos"][inputs.TP].astype(np.float64) / n
    assert np.max(np.abs(emp[1:] - np.exp(-s3 * col2[1:]))) < 1.95 / math.sqrt(n)
    # the first power of n would give a visibly different profile
    col1 = np.concatenate([[0.0], np.cumsum(n_seg) * dz])
    wrong = np.exp(-col1 / col1[-1])
    assert np.max(np.abs(emp[1:] - wrong[1:])) > 10 / math.sqrt(n)


# ---------------------------------------------------------------------------
# charge exchange (Sec. 3.3; Sec. 4 Charge Exchange: one exchange thermalises)

def test_charge_exchange_takes_the_target_velocity():
    prob = _cx_problem(1e20, 1.0, 10, 80.0)
    m1 = inputs.M_T2P_EV
    for i in range(20):
        e1, mu1, v2 = oracle.charge_exchange(prob, m1, 10.0, 0.3, [i, 7, 4], [5, 11])
        s2 = float(np.dot(v2, v2))
        assert e1 == pytest.approx(0.5 * m1 * s2, rel=1e-12, abs=0)
        assert mu1 == pytest.approx(v2[2] / math.sqrt(s2), abs=1e-12)


def test_charge_exchange_one_collision_energy():
    g = GOLD["charge_exchange"]
    # sigma N = 20: every ion exchanges once and is stopped by the collision cap
    prob = _cx_problem(2e20, 1.0, 10, g["t_k"], max_collisions=1)
    n = 200_000
    e0 = g["e_ion_ev"]
    r = oracle.run(prob, inputs.beam(n, 0.0, e0, 1.0, inputs.T2P), seed=15, n_threads=THREADS)
    L = r["ledger"]
    assert L[oracle.N_COLLISIONS] == n and L[oracle.DEATHS + inputs.T2P * 8 + 3] == n
    assert L[oracle.E_IN_PRIMARY] + L[oracle.E_IN_THERMAL] == L[oracle.E_EXIT0:oracle.E_STALLED + 1].sum()
    m1, mt = inputs.M_T2P_EV, inputs.M_T2_EV
    a2 = KB * g["t_k"] / mt                                        # (thermal speed / c)^2
    x0 = math.sqrt(2.0 * _quant(e0) / m1 / a2)
    m2, m4 = cf.cx_one_collision_speed_moments(x0)
    scale = 0.5 * m1 * a2
    mean_e = L[oracle.E_CAP] / 2**24 / n
    sd = scale * math.sqrt(m4 - m2 * m2)
    assert abs(mean_e - scale * m2) < 5 * sd / math.sqrt(n)


def test_charge_exchange_stationary_energy():
    # 64 exchanges deep inside a thick slab: the energy at the cap follows the
    # stationary density f(u) g(u) of the exchange chain
    g = GOLD["charge_exchange"]
    prob = _cx_problem(1e21, 2.0, 20, g["t_k"], max_collisions=64)
    n = 40_000
    rng = np.random.default_rng(2)
    prims = inputs.Primaries(np.full(n, 1.0), np.full(n, g["e_ion_ev"]), rng.uniform(-1, 1, n),
                             np.full(n, inputs.T2P, np.uint8), n)
    r = oracle.run(prob, prims, seed=16, n_threads=THREADS)
    L = r["ledger"]
    assert L[oracle.DEATHS + inputs.T2P * 8 + 3] == n              # none left the slab
    m1, mt = inputs.M_T2P_EV, inputs.M_T2_EV
    a2 = KB * g["t_k"] / mt
    m2, m4 = cf.cx_stationary_speed_moments()
    scale = 0.5 * m1 * a2
    mean_e = L[oracle.E_CAP] / 2**24 / n
    sd = scale * math.sqrt(m4 - m2 * m2)
    assert abs(mean_e - scale * m2) < 5 * sd / math.sqrt(n)
    # and it is not the gas Maxwellian's 3/2 kT (the relative-speed weight shows)
    assert scale * m2 > 1.05 * 1.5 * KB * g["t_k"] * m1 / mt


# ---------------------------------------------------------------------------
# dissociative ionization (Eq. ionization_diss) makes T+

def test_dissociative_ionization_makes_tp():
    nodes = inputs.energy_nodes(2048, 1.0, 2e4)
    chans = [inputs.Channel("ion", inputs.IONIZATION, inputs.E, inputs.T2P, 15.4,
                            inputs.born_bethe(nodes, 15.4, 4.2)),
             inputs.dissociative_ionization(nodes)]
    prob = inputs.uniform_problem(1e20, 1.0, 10, chans, e_cut=1.0)
    n = 50_000
    r = oracle.run(prob, inputs.beam(n, 0.5, 200.0, 1.0), seed=17, n_threads=THREADS)
    L = r["ledger"]
    c = r["chan_count"]
    assert c[1] > 0
    assert L[oracle.BIRTHS + inputs.TP] == c[1]
    assert L[oracle.BIRTHS + inputs.T2P] == c[0]
    assert L[oracle.N_SPAWN_ION] == c[0] + c[1]
    assert L[oracle.E_LOSS_IONIZ] == c[0] * math.floor(15.4 * 2**24) + c[1] * math.floor(18.1 * 2**24)
    ns = oracle.N_SPECIES
    births = L[oracle.BIRTHS:oracle.BIRTHS + ns]
    deaths = L[oracle.DEATHS:oracle.DEATHS + 8 * ns].reshape(ns, 8).sum(axis=1)
    np.testing.assert_array_equal(births, deaths)


def test_charge_exchange_direction_favours_head_on_targets():
    # an ion at twice the thermal speed scale along +z: the mean z velocity it
    # takes is negative, as the relative-speed weight of the target draw fixes
    prob = _cx_problem(1e20, 1.0, 10, 80.0)
    m1, mt = inputs.M_T2P_EV, inputs.M_T2_EV
    a = math.sqrt(KB * 80.0 / mt)
    x0 = 2.0
    e0 = 0.5 * m1 * (x0 * a) ** 2
    n = 20_000
    wz = np.array([oracle.charge_exchange(prob, m1, e0, 1.0, [i, 3, 4], [9, 1])[2][2] / a
                   for i in range(n)])
    expect = cf.cx_one_collision_mean_wz(x0)
    assert expect < -0.1
    assert abs(wz.mean() - expect) < 5 * wz.std() / math.sqrt(n)


def test_segment_stop_and_optical_depth_agree_for_three_body():
    # Sec. 3.1's segment stop-and-redraw and one optical-depth draw per flight
    # are equal in law; with the n^2 rate of three-body clustering on a ramp
    # both give the survival exp(-s3 sum n_j^2 dz) at the far end
    nz, length = 20, 1.0
    n_seg = np.linspace(2e21, 2e22, nz)
    dz = length / nz
    s3 = 1.0 / float(np.sum(n_seg ** 2) * dz)
    nodes = inputs.energy_nodes(64, 1e-3, 10.0)
    ch = inputs.Channel("clust3", inputs.CLUSTERING3, inputs.TP, inputs.T3P, 0.0,
                        np.full_like(nodes, s3))
    prob = _ion_problem([ch], n_seg, length, 1e-3, 10.0)
    n = 60_000
    beam = inputs.beam(n, 0.0, 0.05, 1.0, inputs.TP)
    a = oracle.run(prob, beam, seed=18, mode=0, n_threads=THREADS)
    b = oracle.run(prob, beam, seed=19, mode=1, n_threads=THREADS)
    p = math.exp(-1.0)
    for r in (a, b):
        k = int(r["cross_pos"][inputs.TP][-1])
        assert abs(k - n * p) < 4 * math.sqrt(n * p * (1 - p)), k
