"""Pins of the oracle's scattering-angle distributions (Sec. 3.3 Elastic:
isotropic, from a table sampled as a piecewise-linear distribution, or a
composition switching at a threshold energy).  Fixed by the closed-form
inverse of a linear pdf, exact integrals of the tabulated (piecewise-linear)
pdf, and the screened Rutherford form the synthetic tables come from."""
import math

import numpy as np
import pytest

import oracle
from paper_2503_10263_gb300 import inputs


def _prob_with(table):
    prob, _ = inputs.config1(n_primaries=10)
    prob.channels[0].angular = table
    return prob


def test_isotropic_without_table_or_below_threshold():
    prob = _prob_with(inputs.screened_rutherford_table(threshold_ev=100.0))
    iso, _ = inputs.config1(n_primaries=10)
    for u in np.linspace(0.0, 0.999, 37):
        assert oracle.sample_angle(iso, 0, 500.0, u) == 2 * u - 1
        assert oracle.sample_angle(prob, 0, 50.0, u) == 2 * u - 1      # below threshold
        assert oracle.sample_angle(prob, 1, 500.0, u) == 2 * u - 1     # ionization: no table


def test_constant_table_is_isotropic():
    t = inputs.AngularTable(1.0, 1e4, np.full((4, 11), 0.5), 0.0)
    prob = _prob_with(t)
    for u in np.linspace(0.0, 0.999, 37):
        assert oracle.sample_angle(prob, 0, 30.0, u) == pytest.approx(2 * u - 1, abs=1e-14)


def test_linear_pdf_inverts_exactly():
    # p(x) = 1 + 0.5 x is linear, so the piecewise-linear table is exact and
    # cos chi is the root of its CDF: (x + 1) + (x^2 - 1) / 4 = 2u
    t = inputs.AngularTable(1.0, 1e4, np.tile(1.0 + 0.5 * np.linspace(-1, 1, 9), (3, 1)), 0.0)
    prob = _prob_with(t)
    for u in np.linspace(0.0, 0.999, 101):
        roots = np.roots([0.25, 1.0, 0.75 - 2.0 * u])
        x = roots[np.argmin(np.abs(roots - 0.0))].real
        x = max(-1.0, min(1.0, x))
        assert oracle.sample_angle(prob, 0, 10.0, u) == pytest.approx(x, abs=1e-12)


def test_energy_bin_is_selected():
    # bin 0 leans backward, bin 1 forward: log-spaced bins over [1, 100] eV
    x = np.linspace(-1, 1, 5)
    t = inputs.AngularTable(1.0, 100.0, np.stack([1.0 - 0.9 * x, 1.0 + 0.9 * x]), 0.0)
    prob = _prob_with(t)
    us = (np.arange(4000) + 0.5) / 4000
    lo = np.mean([oracle.sample_angle(prob, 0, 3.0, u) for u in us])
    hi = np.mean([oracle.sample_angle(prob, 0, 30.0, u) for u in us])
    # mean of the linear pdf (1 + b x)/2 on [-1, 1] is b / 3
    assert lo == pytest.approx(-0.3, abs=1e-3)
    assert hi == pytest.approx(0.3, abs=1e-3)
    # clamped outside the table's range
    assert np.mean([oracle.sample_angle(prob, 0, 0.5, u) for u in us[::10]]) < 0
    assert np.mean([oracle.sample_angle(prob, 0, 1e4, u) for u in us[::10]]) > 0


def _linear_table_mean(p):
    """Exact mean of x under the normalised piecewise-linear pdf through p."""
    n = p.size
    x = np.linspace(-1, 1, n)
    h = x[1] - x[0]
    mass = 0.5 * h * (p[:-1] + p[1:])
    # integral of x p(x) over [x_i, x_i + h] for p linear in x
    first = h * (x[:-1] * (p[:-1] + p[1:]) / 2 + h * (p[:-1] + 2 * p[1:]) / 6)
    return first.sum() / mass.sum()


def test_screened_rutherford_table_moments():
    t = inputs.screened_rutherford_table(n_bins=4, n_mu=401, e_min_ev=100.0, e_max_ev=1e4)
    prob = _prob_with(t)
    edges = np.geomspace(100.0, 1e4, 5)
    us = (np.arange(20000) + 0.5) / 20000
    for b in range(4):
        e = math.sqrt(edges[b] * edges[b + 1])
        got = np.mean([oracle.sample_angle(prob, 0, e, u) for u in us])
        assert got == pytest.approx(_linear_table_mean(t.pdf[b]), abs=2e-4)
        # and the table approximates the analytic screened Rutherford mean
        eta = 3.4 / e
        exact = 1.0 - 2.0 * eta * ((1.0 + eta) * math.log((1.0 + eta) / eta) - 1.0)
        assert got == pytest.approx(exact, abs=0.02)


def test_collision_uses_the_table():
    # one elastic collision of a 5 keV electron: the lab polar angle follows the
    # tabulated centre-of-mass angle (mu = 1, so mu' is cos of the lab angle)
    prob = _prob_with(inputs.screened_rutherford_table())
    rng = np.random.default_rng(3)
    g = prob.species_mass_ev[0] / prob.target_mass_ev
    for _ in range(50):
        w = rng.integers(0, 2**63, size=4, dtype=np.uint64)
        ((e1, mu1, _),) = oracle.collide(prob, 0, 0, 5000.0, 1.0, w)
        u = float(w[2] >> np.uint64(11)) / 2**53
        c = oracle.sample_angle(prob, 0, math.floor(5000.0 * 2**24) / 2**24, u)
        ct = (c + g) / math.sqrt(1 + 2 * g * c + g * g)
        assert mu1 == pytest.approx(ct, abs=1e-12)
