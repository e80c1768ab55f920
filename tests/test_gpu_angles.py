"""Tabulated scattering-angle distributions on the GPU (Sec. 3.3 Elastic:
the centre-of-mass polar angle drawn from a piecewise-linear table of the
impact-energy bin, isotropic below a threshold energy) against the FP64
oracle and against the exact moments of the tabulated pdf."""
import math

import numpy as np
import pytest

import oracle
from paper_2503_10263_gb300 import inputs
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def karl():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_10263_gb300 import karl as k
    return k


def _table_mean(p):
    """Exact mean of cos chi under the normalised piecewise-linear pdf through
    the points p (evenly spaced over [-1, 1])."""
    x = np.linspace(-1, 1, p.size)
    h = x[1] - x[0]
    mass = 0.5 * h * (p[:-1] + p[1:])
    first = h * (x[:-1] * (p[:-1] + p[1:]) / 2 + h * (p[:-1] + 2 * p[1:]) / 6)
    return float(first.sum() / mass.sum())


def _dense_config(n=10_000):
    prob, prims = inputs.config1(n_primaries=n, density_m3=2e20, length=2.0, nz=200)
    prob.channels[0].angular = inputs.screened_rutherford_table()
    return prob, prims


def test_fp64_matched_streams(karl):
    prob, prims = _dense_config()
    g = karl.Context(prob).run(prims, seed=5)
    o = oracle.run(prob, prims, seed=5, n_threads=8)
    assert parity.ledger_balances(g["ledger"])
    assert float(np.mean(g["per_primary"] == o["per_primary"])) >= 0.995
    for k in ("spectrum", "cross_pos", "cross_neg"):
        z, p = parity.poisson_two_sample(g[k], o[k])
        assert parity.excursions_ok(z), k
        assert p > 0.01, k
    nc_g, nc_o = int(g["ledger"][karl.N_COLLISIONS]), int(o["ledger"][karl.N_COLLISIONS])
    assert abs(nc_g - nc_o) <= 0.005 * nc_o


def test_fp32_form_statistical(karl):
    prob, prims = _dense_config()
    g = karl.Context(prob).run(prims, seed=6, precision=karl.FP32)
    o = oracle.run(prob, prims, seed=7, n_threads=8)
    assert parity.ledger_balances(g["ledger"])
    # end spectra summed into 100 eV groups (Poisson), per-channel counts
    for end in (0, 1):
        a = g["spectrum"][end, 0, :-1][:20000].reshape(200, 100).sum(1)
        b = o["spectrum"][end, 0, :-1][:20000].reshape(200, 100).sum(1)
        z, p = parity.poisson_two_sample(a, b)
        assert parity.excursions_ok(z) and p > 0.01, end
    cg, co = g["chan_count"].astype(float), o["chan_count"].astype(float)
    assert np.all(np.abs(cg - co) <= 5 * np.sqrt(cg + co) + 0.02 * co)


def _one_collision_problem(table):
    """A mono-energetic beam (mu = 1) into a thick layer of elastic-only gas
    (sigma N = 20, so every electron collides) with a collision cap of one:
    every electron ends its history right after one elastic collision and
    its energy goes to the cap ledger."""
    nodes = inputs.energy_nodes(64, 1.0, 2.0e4)
    ch = inputs.Channel("elastic", inputs.ELASTIC, inputs.E, -1, 0.0,
                        np.full(nodes.shape, 1e-21), angular=table)
    return inputs.uniform_problem(2e22, 1.0, 10, [ch], n_energy=64, e_cut=0.0,
                                  max_collisions=1)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mean_cosine_equals_table_moment(karl, precision):
    # The energy given to the target over n single collisions at e0 is
    # e0 2g/(1+g)^2 sum(1 - cos chi), so the sampler's mean cos chi is read
    # off the ledgers and compared with the exact mean of the tabulated
    # (piecewise-linear) pdf of the bin holding e0; below the threshold the
    # composition is isotropic (mean 0).
    t = inputs.screened_rutherford_table()
    prec = karl.FP64 if precision == "fp64" else karl.FP32
    n = 1_000_000
    g_ratio = inputs.SPECIES_MASS_EV[0] / inputs.M_T2_EV
    c = 2 * g_ratio / (1 + g_ratio) ** 2
    prob = _one_collision_problem(t)
    ctx = karl.Context(prob)
    for e0 in (5000.0, 50.0):
        b = int(math.floor(math.log(e0 / t.e_min_ev) / math.log(t.e_max_ev / t.e_min_ev)
                           * t.pdf.shape[0]))
        b = min(max(b, 0), t.pdf.shape[0] - 1)
        tabulated = e0 >= t.threshold_ev
        expect = _table_mean(t.pdf[b]) if tabulated else 0.0
        g = ctx.run(inputs.beam(n, 0.0, e0, 1.0), seed=11, precision=prec, per_primary=False)
        L = g["ledger"]
        assert parity.ledger_balances(L)
        assert int(L[karl.N_COLLISIONS]) == n
        assert int(L[karl.DEATHS + 3]) == n                        # all ended by the cap
        loss = (n * e0 * 2**24 - int(L[karl.E_CAP])) / 2**24      # sum of e0 c (1 - cos chi)
        mean_cos = 1.0 - loss / (n * e0 * c)
        x = np.linspace(-1, 1, t.pdf.shape[1])
        p = t.pdf[b] if tabulated else np.ones_like(x)
        m2 = float(np.sum(p * x * x) / np.sum(p))
        sd = math.sqrt(max(m2 - expect ** 2, 1e-6))
        assert abs(mean_cos - expect) < 5 * sd / math.sqrt(n) + 2e-6, (e0, mean_cos, expect)


def test_server_request_equals_single_run(karl):
    prob, prims = _dense_config(3000)
    single = karl.Context(prob).run(prims, seed=9, per_primary=False)
    srv = karl.Server(prob)
    try:
        rid = srv.submit(prob, prims, seed=9)
        srv.run_all()
        done, t = srv.poll(rid)
    finally:
        srv.close()
    assert done
    for k in ("spectrum", "time_fx", "cross_pos", "cross_neg", "ledger", "chan_count"):
        np.testing.assert_array_equal(t[k], single[k], err_msg=k)
