"""Pins of the oracle's ionization with a moving target (Sec. 3.3
Ionization: the target velocity is drawn as for elastic scattering and
redrawn while the impact energy is below the ionization energy; the energy is
shared in the target's frame and the ion leaves with the target velocity).

Fixed by things other than the code under test: the binary-encounter
ionization of a target at rest (the oracle's own at-rest routine, pinned in
test_oracle_pins.py) for a gas at 0 K; quadrature of the impact-energy
distribution of the relative-speed weighted Maxwellian, truncated at the
ionization energy, for an electron just above threshold; and the exact
energy and particle ledger of a run.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2503_10263_gb300 import inputs
from tests import parity

KEY = [12345, 678]


def _problem(temperature_k, moving=True):
    nodes = inputs.energy_nodes(2048, 1.0, 2e4)
    prob = inputs.uniform_problem(1e19, 1.0, 10, inputs.electron_channels(nodes, True),
                                  e_cut=1.0)
    prob.gas_temperature_k = temperature_k
    prob.channels[1].target = 1 if moving else 0            # the ionization channel
    return prob


def _words(rng):
    return rng.integers(0, 2**63, size=4, dtype=np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=4, dtype=np.uint64)


def test_gas_at_zero_kelvin_gives_the_target_at_rest_kinematics():
    prob = _problem(0.0)
    rest = _problem(0.0, moving=False)
    m = oracle.marshal_problem(prob)
    me = float(prob.species_mass_ev[inputs.E])
    mion = float(prob.species_mass_ev[inputs.T2P])
    rng = np.random.default_rng(3)
    for i in range(400):
        e = float(rng.uniform(16.0, 5000.0))
        mu = float(rng.uniform(-1.0, 1.0))
        w = _words(rng)
        got = oracle.ionization_moving_target(prob, 1, me, e, mu, mion, w, [i, 0, 4], KEY,
                                              marshal=m)
        ref = oracle.collide(rest, 1, inputs.E, e, mu, w)        # [(E', mu'), (W, mu_s)]
        assert got["ei"] == pytest.approx(e, rel=1e-12)
        q = 2.0 ** -24                                         # one energy unit
        assert abs(got["e1"] - ref[0][0]) <= 2 * q + 1e-12 * e
        assert abs(got["e2"] - ref[1][0]) <= 2 * q + 1e-12 * e
        assert got["mu1"] == pytest.approx(ref[0][1], abs=1e-7)
        assert got["mu2"] == pytest.approx(ref[1][1], abs=1e-7)
        assert got["eion"] == 0.0


def _accepted_mean_excess(e, ion_e, me, mt, kt):
    """Mean of E_i - I over targets w drawn from |u - w| f(w) (f Maxwellian of
    variance kT/M per component) and kept only where E_i = m |u - w|^2 / 2 > I;
    u along z.  Velocities in units of c; w = (w_par, w_perp) about u."""
    a = math.sqrt(kt / mt)
    u = math.sqrt(2.0 * e / me)
    r2 = 2.0 * ion_e / me                 # |u - w|^2 above this: ionization possible

    def dens(wpar, wperp):
        g = math.sqrt((u - wpar) ** 2 + wperp ** 2)
        return g * math.exp(-(wpar * wpar + wperp * wperp) / (2 * a * a)) * wperp

    def ei(wpar, wperp):
        return 0.5 * me * ((u - wpar) ** 2 + wperp ** 2)

    span = 9.0 * a

    def upper(wperp):                     # accepted: w_par below this
        return u - math.sqrt(r2 - wperp * wperp) if wperp * wperp < r2 else span

    num = integrate.dblquad(lambda wpar, wperp: (ei(wpar, wperp) - ion_e) * dens(wpar, wperp),
                            0.0, span, lambda wp: -span, lambda wp: min(upper(wp), span),
                            epsabs=0, epsrel=1e-9)[0]
    den = integrate.dblquad(lambda wpar, wperp: dens(wpar, wperp), 0.0, span,
                            lambda wp: -span, lambda wp: min(upper(wp), span),
                            epsabs=0, epsrel=1e-9)[0]
    return num / den


def test_impact_energy_near_threshold_against_quadrature():
    # an electron 2 meV above the ionization energy in 80 K T2: the target
    # velocities spread the impact energy over a few meV, and only draws
    # above the ionization energy are kept
    t_k = 80.0
    prob = _problem(t_k)
    m = oracle.marshal_problem(prob)
    me = float(prob.species_mass_ev[inputs.E])
    mion = float(prob.species_mass_ev[inputs.T2P])
    ion_e = prob.channels[1].loss_ev
    e = ion_e + 2e-3
    rng = np.random.default_rng(9)
    n = 20000
    ex = np.empty(n)
    for i in range(n):
        r = oracle.ionization_moving_target(prob, 1, me, e, 1.0, mion, _words(rng), [i, 7, 4],
                                            KEY, marshal=m)
        ex[i] = r["ei"] - ion_e
    assert ex.min() > 0.0
    expect = _accepted_mean_excess(e, ion_e, me, prob.target_mass_ev, 8.617333262e-5 * t_k)
    se = ex.std(ddof=1) / math.sqrt(n)
    assert abs(ex.mean() - expect) < 5 * se, (ex.mean(), expect, se)
    # without the redraw the mean excess would stay near the 2 meV offset
    assert expect - 2e-3 > 20 * se


def test_run_with_moving_ionization_balances_its_ledger():
    prob = _problem(3000.0)
    prims = inputs.beam(3000, 0.5, 60.0, 1.0)
    r = oracle.run(prob, prims, seed=11, n_threads=4)
    L = r["ledger"]
    assert parity.ledger_balances(L)
    assert L[oracle.N_SPAWN_ION] > 0
    assert L[oracle.E_IN_THERMAL] > 0          # ions leave with the targets' energies
    # every ion was made by an ionization
    assert L[oracle.BIRTHS + inputs.T2P] == L[oracle.N_SPAWN_ION]
