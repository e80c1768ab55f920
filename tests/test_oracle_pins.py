"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test states the passage it follows.  None of them re-types the oracle's
own formulas: they use closed forms (beam attenuation, the excitation density
pair, truncated-Lorentzian CDF), conservation laws, library routines (numpy's
Philox, scipy's gamma CDF) and exact invariants.
"""
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
M_E = inputs.ME_EV


# ---------------------------------------------------------------------------
# random numbers: Philox4x64-10 against numpy's implementation

def _numpy_block(ctr, key):
    c = sum(int(x) << (64 * i) for i, x in enumerate(ctr))
    bg = np.random.Philox(key=np.array(key, np.uint64), counter=(c - 1) % (1 << 256))
    return bg.random_raw(4)


@pytest.mark.parametrize("ctr,key", [
    ([0, 0, 0, 0], [0, 0]),
    ([1, 2, 3, 4], [5, 6]),
    ([2**64 - 1, 2**64 - 1, 7, 0], [2**63 + 11, 12345]),
    ([123456789, 0xDEADBEEFCAFEBABE, (2 << 8) | 1, 0], [1, 9999]),
])
def test_philox_matches_numpy(ctr, key):
    np.testing.assert_array_equal(oracle.philox4x64(ctr, key), _numpy_block(ctr, key))


# ---------------------------------------------------------------------------
# cross-section lookup (Sec. 3.3 one-dimensional functional; log-node tables)

def test_sigma_exact_for_log_linear_table():
    nodes = inputs.energy_nodes(2048, 1.0, 2e4)
    a, b = 3e-21, 1e-21
    ch = inputs.Channel("t", inputs.EXCITATION, 0, -1, 0.0, a + b * np.log(nodes))
    thr = inputs.Channel("thr", inputs.EXCITATION, 0, -1, 50.0, np.full_like(nodes, 7e-21))
    prob = inputs.uniform_problem(1e19, 1.0, 10, [ch, thr])
    rng = np.random.default_rng(3)
    for e in rng.uniform(1.0, 2e4, 200):
        assert oracle.sigma(prob, 0, e) == pytest.approx(a + b * math.log(e), rel=1e-11, abs=0)
    assert oracle.sigma(prob, 0, 5e4) == pytest.approx(a + b * math.log(2e4), rel=1e-12, abs=0)
    assert oracle.sigma(prob, 1, 50.0) == 0.0
    assert oracle.sigma(prob, 1, 50.000001) == pytest.approx(7e-21, abs=0)


# ---------------------------------------------------------------------------
# free flight: unscattered fraction exp(-sigma int n dz) (Eqs. mean_free_path,
# distance_from_mfp, density_injected) for both flight forms

def _absorber_problem(n_seg, length, sigma):
    nodes = inputs.energy_nodes(64, 1.0, 2e4)
    # any collision leaves E = 0.5 eV < e_cut: the particle stops there
    ch = inputs.Channel("absorb", inputs.EXCITATION, 0, -1, 99.5, np.full_like(nodes, sigma))
    prob = inputs.uniform_problem(1.0, length, len(n_seg), [ch], n_energy=64)
    prob.n_seg_m3 = np.asarray(n_seg, np.float64)
    return prob


@pytest.mark.parametrize("mode", [0, 1])
def test_beam_survival_through_gradient(mode):
    rng = np.random.default_rng(7)
    nz, length, sigma = 40, 1.0, 1e-20
    n_seg = rng.uniform(0.0, 2.0, nz) * 1.5e20
    n_seg[5:8] = 0.0                       # vacuum segments are flown through
    prob = _absorber_problem(n_seg, length, sigma)
    n = 200_000
    prims = inputs.beam(n, 0.0, 100.0, 1.0)
    r = oracle.run(prob, prims, seed=11, mode=mode, n_threads=THREADS)
    dz = length / nz
    surv = cf.survival_at_faces(n_seg, dz, sigma)
    emp = r["cross_pos"][0].astype(np.float64) / n
    # empirical survival function vs exact exponential law (KS 99.9 % bound);
    # face 0 is where the beam starts and is not crossed
    assert emp[0] == 0
    assert np.max(np.abs(emp[1:] - surv[1:])) < 1.95 / math.sqrt(n)
    # every particle either left through z = L or stopped at its collision
    L = r["ledger"]
    assert L[oracle.DEATHS + 1] == r["cross_pos"][0][-1]
    assert L[oracle.DEATHS + 1] + L[oracle.DEATHS + 2] == n
    # mean path length from the time tally = int S(z) dz (Eq. target_field_density's t_i)
    v = cf.speed(100.0, M_E)
    path = r["time_fx"][0, 1:-1, 0].astype(np.float64) / 2**50 * v
    expect = cf.survival_segment_integrals(n_seg, dz, sigma)
    tot, etot = path.sum(), expect.sum() * n
    assert abs(tot - etot) < 4 * cf.bound_sigma(etot, length, n)


def test_mean_free_path_moments_uniform():
    """Mean and variance of the free path in a long uniform column: both
    lambda = 1/(n sigma) (exponential law)."""
    nz, length, sigma, dens = 200, 20.0, 1e-20, 1e20   # lambda = 1 m
    prob = _absorber_problem(np.full(nz, dens), length, sigma)
    n = 100_000
    r = oracle.run(prob, inputs.beam(n, 0.0, 100.0, 1.0), seed=5, n_threads=THREADS)
    surv = r["cross_pos"][0].astype(np.float64) / n        # S at faces
    surv[0] = 1.0                                          # born on face 0
    z = np.linspace(0.0, length, nz + 1)
    # E[d] = int S, E[d^2] = 2 int z S (trapezoid on a 10 cm grid of a 1 m scale)
    m1 = np.trapezoid(surv, z)
    m2 = 2 * np.trapezoid(z * surv, z)
    lam = 1.0 / (dens * sigma)
    assert m1 == pytest.approx(lam, rel=0.02, abs=0)
    assert m2 - m1 ** 2 == pytest.approx(lam ** 2, rel=0.04, abs=0)


# ---------------------------------------------------------------------------
# speed at the beta energies (Sec. 3.1: the particle speed carries the Lorentz
# factor).  Every other speed-dependent pin runs at <= 500 eV, where
# relativity moves v by < 0.1 %; here the time tally of a vacuum flight is held
# to L / (|mu| v) with v = c sqrt(1 - 1/gamma^2), gamma = 1 + E / m c^2, at the
# energies of the beta electrons (1 - 7 % from the Newtonian speed).

ELECTRON_REST_EV = 510998.95            # CODATA 2018 m_e c^2
C_SI = 299792458.0


def vacuum_time_units(e_ev: float, mu: float, seg_len: float) -> float:
    """Time a flight spends in one segment of length seg_len, in 2^-50 s."""
    gamma = 1.0 + e_ev / ELECTRON_REST_EV
    v = C_SI * math.sqrt(1.0 - 1.0 / (gamma * gamma))
    return seg_len / (abs(mu) * v) * 2.0 ** 50


@pytest.mark.parametrize("e_kev", [1.0, 5.0, 18.6])
@pytest.mark.parametrize("mu", [1.0, -0.37])
def test_speed_is_relativistic_at_beta_energies(e_kev, mu):
    nz, length, n = 10, 1.0, 16
    prob = _absorber_problem(np.zeros(nz), length, 1e-20)     # vacuum: straight to the end
    z0 = 0.0 if mu > 0 else length
    r = oracle.run(prob, inputs.beam(n, z0, e_kev * 1e3, mu), seed=1)
    q = vacuum_time_units(e_kev * 1e3, mu, length / nz)
    t = r["time_fx"][0, 1:-1, 0].astype(np.float64)
    # each flight's time in a segment is rounded to one 2^-50 s unit
    tol = 0.5 * n + 1e-6 * q
    assert np.all(np.abs(t - n * q) <= tol), (t / n, q)
    assert r["ledger"][oracle.DEATHS + (1 if mu > 0 else 0)] == n
    # a Newtonian speed, sqrt(2E/m) c, is far outside that bound
    v_newton = C_SI * math.sqrt(2.0 * e_kev * 1e3 / ELECTRON_REST_EV)
    q_newton = length / nz / (abs(mu) * v_newton) * 2.0 ** 50
    assert n * abs(q_newton - q) > 100 * tol


# ---------------------------------------------------------------------------
# channel choice with probability sigma_i n_i / sum (Sec. 2.1)

def test_channel_frequencies_binomial():
    nodes = inputs.energy_nodes(2048, 1.0, 2e4)
    chans = inputs.electron_channels(nodes, full=False)
    prob = inputs.uniform_problem(1e19, 1.0, 10, chans, e_cut=100.0)
    n = 400_000
    # mu = 0: collide in place; e_cut = E: every particle collides exactly once
    r = oracle.run(prob, inputs.beam(n, 0.5, 100.0, 0.0), seed=3, n_threads=THREADS)
    e = np.array([100.0])
    sig = np.array([inputs.elastic_sigma(e)[0], inputs.born_bethe(e, 15.4, 4.2)[0],
                    inputs.born_bethe(e, 12.6, 1.6)[0], inputs.born_bethe(e, 0.5, 0.05)[0]])
    p = sig / sig.sum()
    cnt = r["chan_count"].astype(np.float64)
    # an elastic recoil that rounds to zero leaves a particle at the cut: rare
    # second collisions, at the same energy and with the same channel law
    tot = cnt.sum()
    assert n <= tot <= n + 10
    assert np.all(np.abs(cnt - tot * p) <= 4 * np.sqrt(tot * p * (1 - p)))


# ---------------------------------------------------------------------------
# excitation test of Sec. 4 (Eqs. density_injected, density_single_scattering,
# and the n_s / n_s,2 pair for at most two excitations)

def _excitation_setup():
    g = GOLD["excitation"]
    nodes = inputs.energy_nodes(2048, 1.0, 2e4)
    m_k = 0.5
    ch = inputs.Channel("exc", inputs.EXCITATION, 0, -1, g["e_th_ev"],
                        inputs.born_bethe(nodes, g["e_th_ev"], m_k))
    nz, length, z_n = 30, 1.5, 0.5
    n_seg = np.where((np.arange(nz) + 0.5) * length / nz > z_n, g["n_m3"], 0.0)
    prob = inputs.uniform_problem(1.0, length, nz, [ch], n_tebins=64)
    prob.n_seg_m3 = n_seg
    def lam(e):
        s = inputs.born_bethe(np.array([e]), g["e_th_ev"], m_k)[0] * g["n_m3"]
        return 1.0 / s if s > 0 else math.inf
    return prob, g, lam, z_n


def _tebin(e):
    return int(math.floor(math.log(e) / math.log(2e4) * 64))


def test_excitation_below_threshold_density_is_n0():
    prob, g, lam, z_n = _excitation_setup()
    n = 20_000
    r = oracle.run(prob, inputs.beam(n, 0.0, 12.0, 1.0), seed=2, n_threads=THREADS)
    v = cf.speed(12.0, M_E)
    tsim = n / prob.activity_bq
    n0 = n / (tsim * prob.area_m2 * v)          # Eq. target_field_density, no collisions
    # each segment time is rounded to the 2^-50 s tally unit (dz/v ~ 2.7e7 units)
    np.testing.assert_allclose(r["density"][0], n0, rtol=1e-7)
    # current through every face the beam crosses (it starts on face 0)
    np.testing.assert_allclose(r["current"][0][1:], n / (prob.area_m2 * tsim), rtol=1e-12)
    assert r["ledger"][oracle.N_COLLISIONS] == 0


@pytest.mark.parametrize("e_inj", [20.0, 33.0])
def test_excitation_density_closed_forms(e_inj):
    prob, g, lam, z_n = _excitation_setup()
    e_th = g["e_th_ev"]
    n = 200_000
    r = oracle.run(prob, inputs.beam(n, 0.0, e_inj, 1.0), seed=4, n_threads=THREADS)
    dz = prob.length_m / prob.n_zbins
    energies = [e_inj, e_inj - e_th] + ([e_inj - 2 * e_th] if e_inj > 2 * e_th else [])
    lam1, lam2 = lam(e_inj), lam(e_inj - e_th)
    for order, e in enumerate(energies):
        v = cf.speed(e, M_E)
        t = r["time_fx"][0, 1:-1, _tebin(e)].astype(np.float64) / 2**50
        for j in range(prob.n_zbins):
            lo, hi = j * dz, (j + 1) * dz

            def prob_order(z):
                x = max(z - z_n, 0.0)
                if e_inj > 2 * e_th:
                    return cf.excitation_probabilities(x, lam1, lam2)[order]
                s = math.exp(-x / lam1)
                return s if order == 0 else 1.0 - s
            expect = n / v * cf.segment_average(prob_order, lo, hi, 64)
            # Monte Carlo spread plus half a 2^-50 s tally unit per particle
            tol = 5 * cf.bound_sigma(expect, dz / v, n) + 0.5 * n * 2.0**-50
            assert abs(t[j] - expect) <= tol, (order, j, t[j], expect)


# ---------------------------------------------------------------------------
# clustering test of Sec. 4 (Eq. clustering_test_radiative_cross): T2+ beam
# attenuates with lambda = 1/(sigma n); inferred sigma within 1 %

def test_clustering_attenuation_and_inferred_sigma():
    g = GOLD["clustering_t2p"]
    nodes = inputs.energy_nodes(64, 1.0, 2e4)
    ch = inputs.Channel("clust", inputs.CLUSTERING, inputs.T2P, inputs.T3P, 0.0,
                        np.full_like(nodes, g["sigma_m2"]))
    nz, length = 40, 2.0
    prob = inputs.uniform_problem(g["n_m3"], length, nz, [ch], n_energy=64)
    n = g["n_events"]
    r = oracle.run(prob, inputs.beam(n, 0.0, g["e_ion_ev"], 1.0, inputs.T2P), seed=9,
                   n_threads=THREADS)
    lam = 1.0 / (g["sigma_m2"] * g["n_m3"])
    z = np.linspace(0.0, length, nz + 1)
    emp = r["cross_pos"][inputs.T2P].astype(np.float64) / n
    assert np.max(np.abs(emp[1:] - np.exp(-z[1:] / lam))) < 1.95 / math.sqrt(n)
    # maximum-likelihood mean free path: total T2+ path / number of clusterings
    v = cf.speed(g["e_ion_ev"], inputs.M_T2P_EV)
    path = r["time_fx"][inputs.T2P].astype(np.float64).sum() / 2**50 * v
    k = r["chan_count"][0]
    sigma_hat = k / path / g["n_m3"]
    assert sigma_hat == pytest.approx(g["sigma_m2"], rel=g["rel_err"], abs=0)
    L = r["ledger"]
    assert L[oracle.DEATHS + inputs.T2P * 8 + 6] == k          # T2+ deleted by clustering
    assert L[oracle.BIRTHS + inputs.T3P] == k                  # one T3+ each


# ---------------------------------------------------------------------------
# ionization test of Sec. 4: 30 eV electrons ionize at most once; the slow
# electron follows pdf ~ 1/(1+(W/eps)^2) on [0, (E-I)/2]

def test_ionization_energy_sharing_spectrum():
    from scipy import stats
    g = GOLD["ionization"]
    nodes = inputs.energy_nodes(2048, 1.0, 2e4)
    ch = inputs.Channel("ion", inputs.IONIZATION, 0, -1, 15.4, inputs.born_bethe(nodes, 15.4, 4.2))
    prob = inputs.uniform_problem(g["n_m3"], 1.0, 10, [ch], e_cut=0.0)
    n = 300_000
    rng = np.random.default_rng(1)
    prims = inputs.Primaries(np.full(n, 0.5), np.full(n, g["e_inj_ev"]),
                             rng.uniform(-1, 1, n), np.zeros(n, np.uint8), n)
    r = oracle.run(prob, prims, seed=6, n_threads=THREADS)
    k = int(r["chan_count"][0])
    assert 0 < k <= n
    spec = r["spectrum"][:, 0, :].sum(axis=0).astype(np.float64)
    wmax, eps = (30.0 - 15.4) / 2, 8.0
    # slow electrons alone fill bins 0..6; fast ones (E' = 14.6 - W) fill 8..14
    exp_slow = k * np.diff(cf.lorentz_cdf(np.arange(0, 8.0), eps, wmax))
    hi = 14.6 - np.arange(8, 15, dtype=np.float64)
    exp_fast = k * (cf.lorentz_cdf(hi, eps, wmax) - cf.lorentz_cdf(hi - 1.0, eps, wmax))
    obs = np.concatenate([spec[0:7], spec[8:15]])
    exp = np.concatenate([exp_slow, exp_fast])
    chi2 = float(np.sum((obs - exp) ** 2 / exp))
    assert stats.chi2.sf(chi2, len(obs)) > 0.01
    assert spec[30] == n - k                                   # unscattered primaries
    assert spec.sum() == n + k


# ---------------------------------------------------------------------------
# recombination against a fixed background (Sec. 4, Recombination): both
# partners attenuate exponentially with the frozen pass-1 field

def _recomb_problem():
    nodes = inputs.energy_nodes(2048, 1.0, 2e4)
    rec = inputs.recomb_sigma(nodes, 1e-20)
    chans = [inputs.Channel("e+T3", inputs.RECOMBINATION, inputs.E, inputs.T3P, 0.0, rec.copy()),
             inputs.Channel("T3+e", inputs.RECOMBINATION, inputs.T3P, inputs.E, 0.0, rec.copy())]
    prob = inputs.uniform_problem(0.0, 2.0, 40, chans, n_tebins=64, n_passes=2)
    return prob


def test_recombination_fixed_background_exponential():
    prob = _recomb_problem()
    ne, ni = 40_000, 40_000
    e_e, e_i = 5.0, 0.1
    # energies are carried in units of 2^-24 eV (0.1 eV is not representable)
    e_iq = math.floor(e_i * 2**24) / 2**24
    v_e, v_i = cf.speed(e_e, M_E), cf.speed(e_iq, inputs.M_T3P_EV)
    prims = inputs.Primaries(np.zeros(ne + ni), np.r_[np.full(ne, e_e), np.full(ni, e_i)],
                             np.ones(ne + ni),
                             np.r_[np.zeros(ne, np.uint8), np.full(ni, inputs.T3P, np.uint8)],
                             ne + ni)
    # activity chosen so the pass-1 ion density is 1e21 m^-3
    tsim = ni / (1e21 * prob.area_m2 * v_i)
    prob.activity_bq = (ne + ni) / tsim
    r = oracle.run(prob, prims, seed=8, n_threads=THREADS)
    n_i = ni / (tsim * prob.area_m2 * v_i)
    n_e = ne / (tsim * prob.area_m2 * v_e)
    np.testing.assert_allclose(r["field"][inputs.T3P].sum(axis=1), n_i, rtol=1e-9)
    b = _tebin(e_e)
    e_b = 2e4 ** ((b + 0.5) / 64)
    lam_e = 1.0 / (1e-20 / e_e * n_i)
    lam_i = v_i / (n_e * (1e-20 / e_b) * cf.speed(e_b, M_E))
    z = np.linspace(0.0, prob.length_m, prob.n_zbins + 1)
    for s, n, lam in ((inputs.E, ne, lam_e), (inputs.T3P, ni, lam_i)):
        emp = r["cross_pos"][s].astype(np.float64) / n
        assert np.max(np.abs(emp[1:] - np.exp(-z[1:] / lam))) < 1.95 / math.sqrt(n)
    # each recombination logs one deletion in the partner's field
    assert r["recomb"][inputs.T3P].sum() == r["chan_count"][0]
    assert r["recomb"][inputs.E].sum() == r["chan_count"][1]
    # inferred cross section from the electron attenuation (paper: within 2 %)
    path_e = r["time_fx"][inputs.E].astype(np.float64).sum() / 2**50 * v_e
    sig_hat = r["chan_count"][0] / path_e / n_i
    assert sig_hat == pytest.approx(1e-20 / e_e, rel=GOLD["recombination"]["rel_err"], abs=0)


# ---------------------------------------------------------------------------
# single-collision kinematics by enumeration over the uniforms (Sec. 3.3)

def _words_grid(nu2, nu3, u0=0.5, u1=0.5):
    """Raw words whose top 53 bits put u2, u3 at midpoints of an nu2 x nu3 grid."""
    out = []
    for i in range(nu2):
        for k in range(nu3):
            w = [int(u * 2**53) << 11 for u in (u0, u1, (i + 0.5) / nu2, (k + 0.5) / nu3)]
            out.append(w)
    return out


def test_elastic_kinematics_conservation_and_mean_loss():
    nodes = inputs.energy_nodes(64, 1.0, 2e4)
    prob = inputs.uniform_problem(1e19, 1.0, 10, [inputs.Channel(
        "el", inputs.ELASTIC, 0, -1, 0.0, inputs.elastic_sigma(nodes))], n_energy=64)
    m, mt = M_E, prob.target_mass_ev
    e = 1000.0
    losses = []
    for w in _words_grid(512, 1):
        (e1, mu1, sp), = oracle.collide(prob, 0, 0, e, 1.0, w)
        # mu = 1 incidence: mu1 is the lab polar cosine. Momentum and energy
        # conservation with the target at rest: |p - p'|^2 = 2 M (E - E').
        p2, q2 = 2 * m * e, 2 * m * e1
        pt2 = p2 + q2 - 2 * math.sqrt(p2 * q2) * mu1
        assert pt2 == pytest.approx(2 * mt * (e - e1), rel=2e-4, abs=2 * mt * 1e-7)
        losses.append((e - e1) / e)
    gam = m / mt
    assert np.mean(losses) == pytest.approx(2 * gam / (1 + gam) ** 2, rel=1e-4, abs=0)
    # uniform azimuth: E_phi[mu'] = mu cos(theta), E_phi[mu'^2] = mu^2 c^2 + (1-mu^2) s^2/2
    mu = 0.3
    for i in (3, 100, 400):
        wref = _words_grid(512, 1)[i]
        (_, ct, _), = oracle.collide(prob, 0, 0, e, 1.0, wref)
        outs = [oracle.collide(prob, 0, 0, e, mu, [wref[0], wref[1], wref[2], w[3]])[0][1]
                for w in _words_grid(1, 256)]
        assert np.mean(outs) == pytest.approx(mu * ct, abs=1e-9)
        assert np.mean(np.square(outs)) == pytest.approx(
            mu * mu * ct * ct + (1 - mu * mu) * (1 - ct * ct) / 2, abs=1e-9)


def test_ionization_kinematics_invariants():
    nodes = inputs.energy_nodes(2048, 1.0, 2e4)
    ch = inputs.Channel("ion", inputs.IONIZATION, 0, -1, 15.4, inputs.born_bethe(nodes, 15.4, 4.2))
    prob = inputs.uniform_problem(1e19, 1.0, 10, [ch])
    e, i_ev, eps = 500.0, 15.4, 8.0
    wmax = (e - i_ev) / 2
    for mu in (1.0, 0.37, -0.8, 0.0):
        for w in _words_grid(48, 8):
            (ep, mup, _), (ws, mus, sps) = oracle.collide(prob, 0, 0, e, mu, w)
            assert sps == 0
            assert ep >= ws
            assert ep + ws + i_ev == pytest.approx(e, abs=3e-7)         # energy
            # z-momentum conservation of the binary encounter (no recoil)
            lhs = math.sqrt(ep) * mup + math.sqrt(ws) * mus
            assert lhs == pytest.approx(math.sqrt(e - i_ev) * mu, abs=1e-6)
            # inverse-CDF: the secondary energy sits at its quantile u2
            u2 = (w[2] >> 11) / 2**53
            assert cf.lorentz_cdf(ws, eps, wmax) == pytest.approx(u2, abs=1e-6)


def test_excitation_kinematics():
    nodes = inputs.energy_nodes(64, 1.0, 2e4)
    ch = inputs.Channel("x", inputs.EXCITATION, 0, -1, 12.6, inputs.born_bethe(nodes, 12.6, 1.6))
    prob = inputs.uniform_problem(1e19, 1.0, 10, [ch], n_energy=64)
    (e1, mu1, _), = oracle.collide(prob, 0, 0, 100.0, -0.25, [0, 0, 123 << 20, 456 << 20])
    assert e1 == pytest.approx(100.0 - 12.6, abs=1e-7)
    assert mu1 == -0.25


def test_thermal_product_is_maxwell_boltzmann():
    from scipy import stats
    nodes = inputs.energy_nodes(64, 1.0, 2e4)
    ch = inputs.Channel("cl", inputs.CLUSTERING, inputs.T2P, inputs.T3P, 0.0,
                        np.full_like(nodes, 1e-18))
    prob = inputs.uniform_problem(1e19, 1.0, 10, [ch], n_energy=64)
    rng = np.random.default_rng(12)
    words = rng.integers(0, 2**64, size=(20000, 4), dtype=np.uint64)
    es, mus = [], []
    for w in words:
        (e1, mu1, sp), = oracle.collide(prob, 0, inputs.T2P, 0.01, 1.0, [int(x) for x in w])
        assert sp == inputs.T3P
        es.append(e1)
        mus.append(mu1)
    kt = inputs.KB_EV_PER_K * prob.gas_temperature_k
    assert stats.kstest(es, stats.gamma(1.5, scale=kt).cdf).pvalue > 0.001
    assert stats.kstest(mus, stats.uniform(-1, 2).cdf).pvalue > 0.001


# ---------------------------------------------------------------------------
# conservation (per history and in total) and shard additivity

def _ledger_balances(L):
    e_in = L[oracle.E_IN_PRIMARY] + L[oracle.E_IN_THERMAL]
    e_out = L[oracle.E_EXIT0:oracle.E_STALLED + 1].sum()
    ns = oracle.N_SPECIES
    births = L[oracle.BIRTHS:oracle.BIRTHS + ns]
    deaths = L[oracle.DEATHS:oracle.DEATHS + 8 * ns].reshape(ns, 8).sum(axis=1)
    return e_in == e_out and np.array_equal(births, deaths)


def _small_config2(n_decays=150, seed=3):
    prob, prims = inputs.config2(n_decays=n_decays, seed=seed, column_m2=2e21, length=4.0, nz=100)
    return prob, prims


def test_conservation_total_and_per_history():
    prob, prims = _small_config2()
    r = oracle.run(prob, prims, seed=21, n_threads=THREADS)
    assert _ledger_balances(r["ledger"])
    assert r["ledger"][oracle.N_COLLISIONS] > 1000
    # charge: every ion came from a decay or an ionization, or is a cluster product
    L = r["ledger"]
    assert L[oracle.BIRTHS + inputs.E] == prims.n // 2 + L[oracle.N_SPAWN_E]
    for i in range(0, 40, 3):
        one = prims.slice(i, 1)
        t = oracle.run_pass(prob, one, 21, 1, pid_offset=i, n_decays=prims.n_decays)
        assert _ledger_balances(t["ledger"]), i


def test_shards_sum_to_single_run_bit_exact():
    prob, prims = _small_config2(n_decays=120)
    full = oracle.run(prob, prims, seed=5, n_threads=THREADS)
    cuts = [0, 77, 160, prims.n]
    p1 = [oracle.run_pass(prob, prims.slice(a, b - a), 5, 1, pid_offset=a, n_decays=prims.n_decays)
          for a, b in zip(cuts[:-1], cuts[1:])]
    time1 = sum(t["time_fx"] for t in p1)
    p2 = [oracle.run_pass(prob, prims.slice(a, b - a), 5, 2, field_time_in=time1, pid_offset=a,
                          n_decays=prims.n_decays) for a, b in zip(cuts[:-1], cuts[1:])]
    # a whole run's ledger counts the collisions and flights of both passes
    every = slice(oracle.N_COLLISIONS_ALL, oracle.N_FLIGHTS_ALL + 1)
    p2[0]["ledger"][every] += sum(t["ledger"][every] for t in p1)
    for k in ("spectrum", "time_fx", "cross_pos", "cross_neg", "recomb", "ledger", "chan_count"):
        np.testing.assert_array_equal(sum(t[k] for t in p2), full[k], err_msg=k)
    np.testing.assert_array_equal(np.concatenate([t["per_primary"] for t in p2]),
                                  full["per_primary"])


def test_thread_count_does_not_change_results():
    prob, prims = inputs.config1(n_primaries=2000)
    a = oracle.run(prob, prims, seed=1, n_threads=1)
    b = oracle.run(prob, prims, seed=1, n_threads=THREADS)
    for k in ("spectrum", "time_fx", "cross_pos", "ledger", "per_primary"):
        np.testing.assert_array_equal(a[k], b[k])


def test_segment_stop_and_optical_depth_agree_on_config1():
    """The two flight forms are equal in distribution (memoryless exponential,
    piecewise-constant density): compare total collisions by primary batches."""
    prob, prims = inputs.config1(n_primaries=4000)
    a = oracle.run(prob, prims, seed=1, mode=0, n_threads=THREADS)
    b = oracle.run(prob, prims, seed=2, mode=1, n_threads=THREADS)
    ba = a["per_primary"].reshape(40, -1).sum(axis=1).astype(float)
    bb = b["per_primary"].reshape(40, -1).sum(axis=1).astype(float)
    se = math.sqrt(ba.var(ddof=1) / 40 + bb.var(ddof=1) / 40)
    assert abs(ba.mean() - bb.mean()) < 4 * se
    for s in (0, 1):
        assert abs(int(a["spectrum"][s].sum()) - int(b["spectrum"][s].sum())) < 4 * math.sqrt(4000)


# ---------------------------------------------------------------------------
# inputs: beta spectrum moments against quadrature of its pdf

def test_beta_generator_moments():
    from scipy import integrate
    rng = np.random.default_rng(0)
    e = inputs.sample_beta(rng, 400_000)
    z, _ = integrate.quad(lambda x: inputs.beta_pdf(np.array([x]))[0], 0, 18600, limit=200)
    m1, _ = integrate.quad(lambda x: x * inputs.beta_pdf(np.array([x]))[0], 0, 18600, limit=200)
    m2, _ = integrate.quad(lambda x: x * x * inputs.beta_pdf(np.array([x]))[0], 0, 18600, limit=200)
    mean, var = m1 / z, m2 / z - (m1 / z) ** 2
    assert abs(e.mean() - mean) < 4 * math.sqrt(var / e.size)
    assert e.var() == pytest.approx(var, rel=0.01, abs=0)
    assert 5000 < mean < 6500
