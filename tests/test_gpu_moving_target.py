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


# ---------------------------------------------------------------------------
# ionization with a moving target (Sec. 3.3 Ionization): electrons just above
# the ionization energy in a warm gas, where the target draws and their
# redraw below threshold shape the kinematics

def _ionization_case(n=20000, seed=17, temperature_k=3000.0):
    nodes = inputs.energy_nodes(2048, 1.0, 2e4)
    prob = inputs.uniform_problem(3e20, 0.3, 30, inputs.electron_channels(nodes, True),
                                  e_cut=1.0)
    prob.gas_temperature_k = temperature_k
    prob.channels[1].target = 1                   # ionization
    rng = np.random.default_rng(seed)
    prims = inputs.Primaries(rng.uniform(0.0, 0.3, n), rng.uniform(15.45, 40.0, n),
                             rng.uniform(-1.0, 1.0, n), np.zeros(n, np.uint8), n)
    return prob, prims


def test_moving_ionization_follows_the_oracle(karl):
    prob, prims = _ionization_case()
    o = oracle.run(prob, prims, seed=21, n_threads=16)
    g = karl.Context(prob).run(prims, seed=21)
    assert parity.ledger_balances(g["ledger"])
    assert g["ledger"][karl.N_SPAWN_ION] > 1000
    assert float(np.mean(g["per_primary"] == o["per_primary"])) >= 0.99
    # the ions' energies come from the targets' velocities: their totals agree
    assert abs(int(g["ledger"][karl.E_IN_THERMAL]) - int(o["ledger"][oracle.E_IN_THERMAL])) <= \
        2e-3 * int(o["ledger"][oracle.E_IN_THERMAL])
    for k in ("spectrum", "cross_pos", "cross_neg"):
        z, p = parity.poisson_two_sample(g[k], o[k])
        assert parity.excursions_ok(z) and p > 0.01, k
    f = karl.Context(prob).run(prims, seed=21, precision=karl.FP32)
    assert parity.ledger_balances(f["ledger"])
    for k in ("spectrum", "cross_pos"):
        z, p = parity.poisson_two_sample(f[k], o[k])
        assert parity.excursions_ok(z) and p > 0.01, k


def test_moving_ionization_served_equals_single_run(karl):
    prob, prims = _ionization_case(n=3000, seed=5)
    single = karl.Context(prob).run(prims, seed=8, per_primary=False)
    srv = karl.Server(prob, hbm_budget_bytes=1 << 30, timeout_s=60)
    rid = srv.submit(prob, prims, 8)
    srv.run_all()
    _, t = srv.poll(rid)
    srv.close()
    for k in ("spectrum", "time_fx", "cross_pos", "cross_neg", "recomb", "ledger", "chan_count"):
        np.testing.assert_array_equal(t[k], single[k], err_msg=k)
