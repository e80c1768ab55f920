"""Pins of the oracle's elastic collision with a moving target (Sec. 3.3
Elastic: the target moves with the gas drift plus a Maxwell-Boltzmann
velocity) and of the thermalisation it produces (Sec. 4, elastic
thermalisation test).  Each pin is fixed by something other than the code
under test: the textbook lab-frame formulas of a target at rest, the
conservation laws of an elastic collision, quadrature of the relative-speed
weighted Maxwellian, and the Maxwell-Boltzmann equilibrium of a test particle.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2503_10263_gb300 import inputs

KB = 8.617333262e-5
C = 299792458.0


def _prob(temperature_k=80.0, drift=0.0):
    prob, _ = inputs.thermalization(temperature_k=temperature_k, drift_mps=drift)
    return prob


def _words(rng, n=4):
    return rng.integers(0, 2**63, size=n, dtype=np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=n, dtype=np.uint64)


def test_target_at_rest_reduces_to_lab_formulas():
    # T = 0 and no drift: the centre-of-mass rotation must give the lab-frame
    # energy and polar angle of the target-at-rest routine (orc_collide)
    prob = _prob(temperature_k=0.0)
    cold, _ = inputs.thermalization(temperature_k=0.0)
    cold.channels[0].target = 0
    rng = np.random.default_rng(5)
    me = float(prob.species_mass_ev[0])
    for _ in range(300):
        # an energy on the 2^-24 eV grid, which the at-rest routine works on
        e = math.floor(float(10 ** rng.uniform(-3, 3)) * 2**24) / 2**24
        mu = float(rng.uniform(-1, 1))
        w = _words(rng)
        e1, mu1, _ = oracle.elastic_moving_target(prob, me, e, mu, w, [0, 0, 0], [1, 2])
        ((ec, muc, _),) = oracle.collide(cold, 0, 0, e, mu, w)
        # the at-rest routine rounds its energy transfer to the nearest 2^-24 eV
        assert abs(e1 - ec) <= 0.5 / 2**24 + 1e-12 * e
        assert abs(mu1 - muc) <= 1e-10


@pytest.mark.parametrize("species", [0, 1])
def test_momentum_and_energy_are_conserved(species):
    prob = _prob(temperature_k=300.0, drift=500.0)
    rng = np.random.default_rng(11 + species)
    m1 = float(prob.species_mass_ev[species])
    m2 = prob.target_mass_ev
    for _ in range(300):
        e = float(10 ** rng.uniform(-3, 2))
        mu = float(rng.uniform(-1, 1))
        e1, mu1, v = oracle.elastic_moving_target(prob, m1, e, mu, _words(rng),
                                                  _words(rng, 3), _words(rng, 2))
        v1, v2, v1n, v2n = v[0:3], v[3:6], v[6:9], v[9:12]
        p0 = m1 * v1 + m2 * v2
        p1 = m1 * v1n + m2 * v2n
        assert np.allclose(p0, p1, rtol=0, atol=1e-12 * np.linalg.norm(p0) + 1e-30)
        k0 = 0.5 * m1 * v1 @ v1 + 0.5 * m2 * v2 @ v2
        k1 = 0.5 * m1 * v1n @ v1n + 0.5 * m2 * v2n @ v2n
        assert abs(k1 - k0) <= 1e-11 * k0
        assert e1 == pytest.approx(0.5 * m1 * v1n @ v1n, rel=1e-12, abs=0)
        assert mu1 == pytest.approx(v1n[2] / np.linalg.norm(v1n), abs=1e-12)
        # the impactor before the collision is the one given
        assert 0.5 * m1 * v1 @ v1 == pytest.approx(e, rel=1e-12, abs=0)
        assert v1[2] / np.linalg.norm(v1) == pytest.approx(mu, abs=1e-12)


def _target_draws(prob, m1, e, mu, n, seed):
    rng = np.random.default_rng(seed)
    out = np.empty((n, 3))
    for i in range(n):
        _, _, v = oracle.elastic_moving_target(prob, m1, e, mu, _words(rng), [i, 7, 9],
                                               [seed, 3])
        out[i] = v[3:6]
    return out


def _weighted_moments(u, a):
    """<|w|^2> and <w . u_hat> of w ~ |u - w| f(w), f a Maxwellian with
    per-component variance a^2, by quadrature over speed and angle."""
    def f(s, c, g):
        rel = math.sqrt(max(u * u + s * s - 2 * u * s * c, 0.0))
        return rel * s * s * math.exp(-s * s / (2 * a * a)) * g(s, c)
    lim = 10 * a
    z = integrate.dblquad(lambda c, s: f(s, c, lambda s, c: 1.0), 0, lim, -1, 1)[0]
    m2 = integrate.dblquad(lambda c, s: f(s, c, lambda s, c: s * s), 0, lim, -1, 1)[0]
    m1 = integrate.dblquad(lambda c, s: f(s, c, lambda s, c: s * c), 0, lim, -1, 1)[0]
    return m2 / z, m1 / z


@pytest.mark.parametrize("ratio", [0.0, 1.0, 30.0])
def test_target_velocity_follows_relative_speed_weight(ratio):
    # impactor speed |u| = ratio * a in the gas frame (no drift): the sampled
    # thermal velocity must have the moments of |u - w| f(w)
    prob = _prob(temperature_k=80.0)
    m2 = prob.target_mass_ev
    a = math.sqrt(KB * 80.0 / m2)
    m1 = float(prob.species_mass_ev[1])          # an ion, so u is comparable to a
    u = ratio * a
    e = 0.5 * m1 * u * u
    n = 20000
    w = _target_draws(prob, m1, max(e, 0.0), 1.0, n, seed=int(ratio * 10) + 1)
    s2 = (w * w).sum(1) / (a * a)
    proj = w[:, 2] / a                             # u points along +z (mu = 1)
    m2_exact, m1_exact = _weighted_moments(u, a)
    se2 = s2.std() / math.sqrt(n)
    se1 = proj.std() / math.sqrt(n)
    assert abs(s2.mean() - m2_exact / a**2) < 4 * se2
    assert abs(proj.mean() - m1_exact / a) < 4 * se1
    assert abs(w[:, 0].mean() / a) < 4 / math.sqrt(n) and abs(w[:, 1].mean() / a) < 4 / math.sqrt(n)


def test_drift_moves_the_targets():
    prob = _prob(temperature_k=80.0, drift=800.0)
    me = float(prob.species_mass_ev[0])
    w = _target_draws(prob, me, 1.0, 0.3, 4000, seed=21)
    a = math.sqrt(KB * 80.0 / prob.target_mass_ev)
    # a fast electron weights targets by |v1 - v2| ~ |v1|: plain Maxwellian + drift
    assert abs(w[:, 2].mean() - 800.0 / C) < 4 * a / math.sqrt(4000)
    assert abs(w[:, 2].std() / a - 1.0) < 0.05


def test_elastic_thermalisation_gives_the_gas_temperature():
    # Sec. 4: 8 meV electrons injected along +z into 1e22 m^-3 of T2 at 80 K,
    # constant elastic cross section.  In equilibrium a test particle follows
    # the gas Maxwellian; exits happen after a number of collisions that does
    # not depend on the energy (constant mean free path), so the exit spectrum
    # is the collision-weighted Maxwellian, E exp(-E/kT) (Gamma(2, kT)):
    # mean 2kT, variance 2(kT)^2.
    prob, prims = inputs.thermalization(n_primaries=2000, length=0.4)
    o = oracle.run(prob, prims, seed=3, n_threads=8)
    spec = o["spectrum"].reshape(2, inputs.N_SPECIES, -1)[:, 0, :].sum(0).astype(float)
    assert spec[-1] == 0
    w = prob.spec_bin_ev
    e = (np.arange(spec.size - 1) + 0.5) * w
    n = spec[:-1].sum()
    assert n == prims.n
    mean = (spec[:-1] * e).sum() / n
    var = (spec[:-1] * e * e).sum() / n - mean**2
    t_fit = mean / (2 * KB)
    sigma_t = t_fit / math.sqrt(2 * n)
    assert abs(t_fit - 80.0) < 4 * sigma_t, t_fit
    assert abs(var / mean**2 - 0.5) < 0.1
    L = o["ledger"]
    assert int(L[0]) + int(L[1]) == int(L[2:12].sum())
    assert int(L[10]) < 0                      # the gas heated the electrons on the whole
