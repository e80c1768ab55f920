"""Elastic collisions with a moving target on the GPU (Sec. 3.3 Elastic: gas
drift plus a Maxwell-Boltzmann velocity) against the FP64 oracle, on the
elastic thermalisation case of Sec. 4: 8 meV electrons in 1e22 m^-3 of T2 at
80 K, constant cross section, about 6e4 collisions per electron."""
import math

import numpy as np
import pytest

import oracle
from paper_2503_10263_gb300 import inputs
from tests import parity

pytestmark = pytest.mark.gpu

KB = 8.617333262e-5


@pytest.fixture(scope="module")
def karl():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_10263_gb300 import karl as k
    return k


@pytest.fixture(scope="module")
def case():
    prob, prims = inputs.thermalization(n_primaries=2000, length=0.4)
    return prob, prims, oracle.run(prob, prims, seed=3, n_threads=16)


def _exit_stats(prob, t):
    spec = np.asarray(t["spectrum"]).reshape(2, inputs.N_SPECIES, -1)[:, 0, :].sum(0).astype(float)
    e = (np.arange(spec.size - 1) + 0.5) * prob.spec_bin_ev
    n = spec[:-1].sum()
    mean = (spec[:-1] * e).sum() / n
    return spec, n, mean / (2 * KB)


def _coarse(spec, k=40):
    body = spec[:-1]
    return body[: body.size // k * k].reshape(-1, k).sum(1)


def test_fp64_matches_oracle(karl, case):
    prob, prims, o = case
    g = karl.Context(prob).run(prims, seed=3)
    assert parity.ledger_balances(g["ledger"])
    # same random streams: the collision count of each electron's history
    assert float(np.mean(g["per_primary"] == o["per_primary"])) >= 0.95
    sg, n, t_g = _exit_stats(prob, g)
    so, _, t_o = _exit_stats(prob, o)
    assert n == prims.n
    z, p = parity.poisson_two_sample(_coarse(sg), _coarse(so))
    assert parity.excursions_ok(z) and p > 0.01
    assert abs(t_g - t_o) < 0.5
    assert abs(t_g - 80.0) < 4 * 80.0 / math.sqrt(2 * n)


def test_fp32_form_thermalises(karl, case):
    prob, prims, o = case
    g = karl.Context(prob).run(prims, seed=4, precision=karl.FP32)
    assert parity.ledger_balances(g["ledger"])
    sg, n, t_g = _exit_stats(prob, g)
    so, _, _ = _exit_stats(prob, o)
    assert n == prims.n
    z, p = parity.poisson_two_sample(_coarse(sg), _coarse(so))
    assert parity.excursions_ok(z) and p > 0.01
    assert abs(t_g - 80.0) < 4 * 80.0 / math.sqrt(2 * n)
