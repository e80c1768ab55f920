"""Full-orbit transport (the Boris mover of Sec. 3.1) on the GPU against the
oracle and against the closed forms its pins use.

The push is compiled without multiply-add contraction, like the oracle, so
between collisions both sides compute the same positions; the histories part
only where a library function (log, sin, cos, tan, atan) rounds differently
in the last place and a discrete decision falls on that difference."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2503_10263_gb300 import inputs
from tests import parity
from tests.test_oracle_orbit import C, Q_TIME, _deaths, _msd_closed_form, _orbit, _prims, _vacuum

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def karl():
    import torch
    assert torch.cuda.is_available()
    from paper_2503_10263_gb300 import build, karl as k
    build.build()
    return k


def _gpu(karl, prob, orb, pr, seed=1, **kw):
    ctx = karl.Context(prob)
    try:
        return ctx.run_orbit(orb, pr, seed=seed, **kw)
    finally:
        ctx.close()


def test_tube_section_follows_the_oracle(karl):
    """Tube section with ionization, clustering, ion scattering and a radial
    field: collision counts per primary, the integer ledger and the tallies
    follow the oracle's run of the same primaries."""
    prob, orb, pr = inputs.orbit_config(n_decays=300, seed=3)
    g = _gpu(karl, prob, orb, pr, seed=3)
    o = oracle.orbit_run(prob, orb, pr, seed=3, n_threads=THREADS)
    same = float(np.mean(g["per_primary"] == o["per_primary"]))
    print(f"PARITY orbit tube section: histories identical {same:.4f} of {pr.n}")
    assert same >= 0.99
    lg, lo = g["ledger"].astype(float), o["ledger"].astype(float)
    assert np.all(np.abs(lg - lo) <= 0.01 * lo + 3 * np.sqrt(lo + 1))
    for key in ("time_z", "time_r"):
        a, b = g[key].astype(float), o[key].astype(float)
        assert abs(a.sum() - b.sum()) <= 0.01 * b.sum()
    for key in ("wall", "spectrum", "cross_pos", "cross_neg", "rcross_out", "rcross_in"):
        a, b = g[key].astype(float).sum(), o[key].astype(float).sum()
        assert abs(a - b) <= 0.01 * b + 3 * math.sqrt(b + 1), key
    E = g["energy"]
    e_in = E[karl.OE_IN_PRIMARY] + E[karl.OE_IN_THERMAL] + E[karl.OE_FIELD_WORK]
    assert abs(e_in - E[karl.OE_EXIT0:karl.OE_STALLED + 1].sum()) < 1e-9 * E[karl.OE_IN_PRIMARY]
    assert g["ledger"][karl.OB_DEATHS + 8 * inputs.T2P + 6] > 0
    assert g["wall"].sum() > 0


@pytest.mark.parametrize("species,e_ev", [(inputs.E, 18600.0), (inputs.T2P, 10.0)])
def test_gyration_decides_wall_hits_on_the_gpu(karl, species, e_ev):
    """The gyration-circle geometry of the oracle pin: wall hit at 0.98 of
    the circle's reach, exit at 1.02, for both charge signs."""
    m = inputs.SPECIES_MASS_EV[species]
    b, mu = 0.5, 0.2
    pc = math.sqrt(e_ev * (e_ev + 2 * m))
    r_l = pc * math.sqrt(1 - mu * mu) / (C * b)
    sgn = -1.0 if species == inputs.E else 1.0
    d = 5.0 * r_l
    omega = b * C * C / (m + e_ev)
    length = 8 * 2 * math.pi / omega * C * pc / (e_ev + m) * mu
    prob = _vacuum(length=length)
    for scale, wall in ((0.98, True), (1.02, False)):
        orb = _orbit(b, tube_radius_m=(d + r_l) * scale, n_rbins=4)
        t = _gpu(karl, prob, orb, _prims([d - r_l], [0.0], [0.0], [e_ev], [mu],
                                         [sgn * 0.5 * math.pi], species))
        assert _deaths(t, species, "wall") == (1 if wall else 0)
        assert _deaths(t, species, "exit1") == (0 if wall else 1)


def test_transit_field_work_and_exb_on_the_gpu(karl):
    """Relativistic transit time, axial-field work with hyperbolic motion,
    and the exact E x B slow mode, as in the oracle pins."""
    m = inputs.ME_EV
    # transit at 18.6 keV, mu = 0.7
    prob = _vacuum(length=1.0)
    orb = _orbit(0.5, tube_radius_m=0.05, n_rbins=5)
    t = _gpu(karl, prob, orb, _prims([0.0], [0.0], [0.1], [18600.0], [0.7], [1.0], inputs.E))
    v = C * math.sqrt(18600.0 * (18600.0 + 2 * m)) / (18600.0 + m)
    expect = 0.9 / (0.7 * v) * Q_TIME
    assert abs(float(t["time_z"].sum()) - expect) < 0.5 * (prob.n_zbins + 12) + 1e-12 * expect
    # electrons accelerated by E_z = -1000 V/m from 100 eV over 1 m
    orb = _orbit(0.5, tube_radius_m=0.05, n_rbins=5, e_z_vm=np.full(prob.n_zbins, -1000.0))
    t = _gpu(karl, prob, orb, _prims([0.0] * 4, [0.0] * 4, [0.0] * 4, [100.0] * 4, [1.0] * 4,
                                     [0.0] * 4, inputs.E))
    assert abs(t["energy"][karl.OE_EXIT1] / 4 - 1100.0) < 0.11
    pc0, pc1 = (math.sqrt(e * (e + 2 * m)) for e in (100.0, 1100.0))
    t_exp = (pc1 - pc0) / (C * 1000.0) * Q_TIME
    assert abs(float(t["time_z"].sum()) / 4 - t_exp) < 1e-4 * t_exp
    # E x B slow mode of a T3+ ion
    mi = inputs.M_T3P_EV
    b, e_r, r0, t_cap = 0.5, 1e4, 0.01, 1e-4
    om, kappa = b * C * C / mi, e_r * C * C / mi
    om_s = 0.5 * (-om + math.sqrt(om * om - 4.0 * kappa))
    vi = abs(om_s) * r0
    e_kin = mi * (1.0 / math.sqrt(1.0 - (vi / C) ** 2) - 1.0)
    prob = _vacuum(length=1.0, lifetime=t_cap)
    orb = _orbit(b, tube_radius_m=0.05, n_rbins=5, e_r_vm2=e_r)
    t = _gpu(karl, prob, orb, _prims([r0], [0.0], [0.5], [e_kin], [0.0],
                                     [0.5 * math.pi if om_s > 0 else -0.5 * math.pi], inputs.T3P))
    x, y = t["end_state"][0, 0], t["end_state"][0, 1]
    turned = math.atan2(y, x)
    assert abs(math.remainder(turned - om_s * t_cap, 2 * math.pi)) < 2e-3 * abs(om_s * t_cap)
    assert abs(math.hypot(x, y) - r0) < 1e-3 * r0


def test_cross_field_diffusion_on_the_gpu(karl):
    """Classical cross-field spread of isotropically scattered electrons at
    Omega = 3 nu (the oracle pin's closed form), with 20000 electrons."""
    m = inputs.ME_EV
    e, n_m3, sigma = 100.0, 1e20, 1e-19
    v = C * math.sqrt(e * (e + 2 * m)) / (e + m)
    nu = n_m3 * sigma * v
    om = 3.0 * nu
    b = om * (m + e) / (C * C)
    t_cap = 10.0 / nu
    nodes = inputs.energy_nodes(64, 1.0, 1e3)
    ch = [inputs.Channel("elastic", inputs.ELASTIC, inputs.E, -1, 0.0, np.full_like(nodes, sigma))]
    prob = inputs.uniform_problem(n_m3, 1000.0, 10, ch, n_energy=64, e_min=1.0, e_max=1e3,
                                  e_cut=0.0, max_lifetime_s=t_cap, max_collisions=10**9)
    prob.target_mass_ev = 1e18
    orb = _orbit(b, frac=0.02, tube_radius_m=10.0, n_rbins=4)
    dt = orb.dt_s[inputs.E]
    om_eff = 2.0 * math.atan(0.5 * om * dt) / dt
    n = 20000
    rng = np.random.default_rng(12)
    pr = _prims(np.zeros(n), np.zeros(n), np.full(n, 500.0), np.full(n, e),
                rng.uniform(-1, 1, n), rng.uniform(0, 2 * math.pi, n), inputs.E)
    t = _gpu(karl, prob, orb, pr, seed=4)
    r2 = t["end_state"][:, 0] ** 2 + t["end_state"][:, 1] ** 2
    expect = _msd_closed_form(v, nu, om_eff, t_cap)
    se = r2.std() / math.sqrt(n)
    print(f"PARITY orbit diffusion: <r^2> {r2.mean():.5e} closed form {expect:.5e} "
          f"({(r2.mean() - expect) / se:+.2f} standard errors)")
    assert abs(r2.mean() - expect) < 5 * se


def test_orbit_reproduces_the_guiding_centre_kernel(karl):
    """Uniform B, no electric field, uniform gas: the full-orbit kernel
    follows the guiding-centre kernel's histories (the oracle pin's
    reduction, here between the two CUDA paths)."""
    prob, prims = inputs.config1(n_primaries=3000, seed=4, density_m3=2e20, length=0.5, nz=50)
    prims.e_ev[:] = np.linspace(50.0, 600.0, prims.n)
    orb = _orbit(0.02, frac=0.1, tube_radius_m=5.0, n_rbins=4)
    rng = np.random.default_rng(9)
    pr = inputs.OrbitPrimaries(np.zeros(prims.n), np.zeros(prims.n), prims.z_m.copy(),
                               prims.e_ev.copy(), prims.mu.copy(),
                               rng.uniform(0, 2 * math.pi, prims.n), prims.species.copy())
    a = _gpu(karl, prob, orb, pr, seed=7)
    ctx = karl.Context(prob)
    try:
        gc = ctx.run(prims, seed=7)
    finally:
        ctx.close()
    same = float(np.mean(a["per_primary"] == gc["per_primary"]))
    print(f"PARITY orbit vs guiding-centre kernel: histories identical {same:.4f}")
    assert same > 0.95


def test_orbit_rejects_what_it_does_not_model(karl):
    """FP32, recombination channels and primaries outside the tube are
    refused with KARL_EINVAL; the context stays usable."""
    prob, orb, pr = inputs.orbit_config(n_decays=10, seed=1)
    ctx = karl.Context(prob)
    try:
        with pytest.raises(karl.KarlError) as e:
            ctx.run_orbit(orb, pr, precision=karl.FP32)
        assert e.value.status == karl.EINVAL
        bad = inputs.OrbitPrimaries(pr.x_m.copy(), pr.y_m.copy(), pr.z_m.copy(), pr.e_ev.copy(),
                                    pr.mu.copy(), pr.phi.copy(), pr.species.copy())
        bad.x_m[3] = 2 * orb.tube_radius_m
        with pytest.raises(karl.KarlError) as e:
            ctx.run_orbit(orb, bad)
        assert e.value.status == karl.EINVAL
        t = ctx.run_orbit(orb, pr)
        assert t["ledger"][karl.OB_N_FLIGHTS] > 0
    finally:
        ctx.close()
    prob2, _ = inputs.config2(n_decays=10)
    ctx = karl.Context(prob2)
    try:
        with pytest.raises(karl.KarlError) as e:
            ctx.run_orbit(orb, pr)
        assert e.value.status == karl.EINVAL
    finally:
        ctx.close()


def test_energy_bin_restarts_on_the_gpu(karl):
    """The Sec. 3.1 stop rule: an electron accelerated from 100 eV to 1100 eV
    flies once per energy bin it passes (17 flights over 64 log bins)."""
    nodes = inputs.energy_nodes(64, 1.0, 2e4)
    ch = [inputs.Channel("elastic", inputs.ELASTIC, inputs.E, -1, 0.0, np.full_like(nodes, 1e-20))]
    prob = inputs.uniform_problem(0.0, 1.0, 10, ch, n_energy=64, e_min=1.0, e_max=2e4,
                                  e_cut=0.0, n_tebins=64, n_spec_bins=4000, spec_bin_ev=1.0)
    orb = _orbit(0.5, tube_radius_m=0.05, n_rbins=5, e_z_vm=np.full(prob.n_zbins, -1000.0))
    pr = _prims([0.0], [0.0], [0.0], [100.0], [1.0], [0.0], inputs.E)
    t = _gpu(karl, prob, orb, pr)
    o = oracle.orbit_run(prob, orb, pr)
    assert int(t["ledger"][karl.OB_N_FLIGHTS]) == int(o["ledger"][oracle.OB_N_FLIGHTS]) == 17
    assert np.array_equal(t["time_z"], o["time_z"])


def test_ion_workload_follows_the_oracle(karl):
    """The ion tube workload of the benchmark (B = 2.5 T, radial field,
    clustering and ion scattering, lifetime cap): matched histories and
    equal tallies up to the parting histories."""
    prob, orb, pr = inputs.orbit_ion_config(n_ions=3000, seed=5)
    g = _gpu(karl, prob, orb, pr, seed=5)
    o = oracle.orbit_run(prob, orb, pr, seed=5, n_threads=THREADS)
    same = float(np.mean(g["per_primary"] == o["per_primary"]))
    print(f"PARITY orbit ions: histories identical {same:.4f} of {pr.n}")
    assert same >= 0.99
    end_same = float(np.mean(np.all(np.abs(g["end_state"] - o["end_state"]) <=
                                    1e-9 * (np.abs(o["end_state"]) + 1e-12), axis=1)))
    print(f"PARITY orbit ions: end states equal to 1e-9 {end_same:.4f}")
    assert end_same >= 0.99
    for key in ("time_z", "time_r"):
        a, b = g[key].astype(float), o[key].astype(float)
        assert np.abs(a - b).sum() <= 0.01 * b.sum()


def test_orbit_edge_cases_match_the_oracle(karl):
    """Degenerate starts, identical on both sides: no primaries; a particle
    on z = L moving out and one on z = 0 moving in -z (zero-length exits); a
    particle just inside the wall moving outward; flights along the axis
    (mu = +-1, the turning frame's special case) through gas; a step cap
    that stalls a gyrating ion."""
    nodes = inputs.energy_nodes(64, 1.0, 2e4)
    ch = [inputs.Channel("elastic", inputs.ELASTIC, inputs.E, -1, 0.0, np.full_like(nodes, 1e-19)),
          inputs.Channel("elastic_T2+", inputs.ELASTIC, inputs.T2P, -1, 0.0,
                         np.full_like(nodes, 1e-19))]
    prob = inputs.uniform_problem(1e19, 1.0, 20, ch, n_energy=64, e_min=1.0, e_max=2e4,
                                  e_cut=0.0, n_spec_bins=4000, spec_bin_ev=1.0)
    orb = _orbit(0.1, frac=0.1, tube_radius_m=0.05, n_rbins=5)
    empty = _prims([], [], [], [], [], [], inputs.E)
    g = _gpu(karl, prob, orb, empty)
    o = oracle.orbit_run(prob, orb, empty)
    for k in ("time_z", "ledger", "spectrum"):
        assert not np.any(g[k]) and not np.any(o[k]), k
    r = 0.05 * (1 - 1e-9)
    pr = _prims([0.0, 0.0, r, 0.0, 0.0, 0.01],
                [0.0, 0.0, 0.0, 0.0, 0.0, 0.0],
                [1.0, 0.0, 0.5, 0.3, 0.7, 0.5],
                [500.0, 500.0, 500.0, 300.0, 300.0, 1.0],
                [0.5, -0.5, 0.0, 1.0, -1.0, 0.0],
                [0.0, 0.0, 0.0, 0.0, 0.0, 0.5 * math.pi],
                inputs.E)
    pr.species[5] = inputs.T2P
    for max_steps in (0, 200):
        orb.max_steps = max_steps
        g = _gpu(karl, prob, orb, pr, seed=9)
        o = oracle.orbit_run(prob, orb, pr, seed=9)
        np.testing.assert_array_equal(g["ledger"], o["ledger"])
        np.testing.assert_array_equal(g["per_primary"], o["per_primary"])
        for k in ("time_z", "time_r", "cross_pos", "cross_neg", "rcross_out", "rcross_in",
                  "wall", "spectrum"):
            np.testing.assert_array_equal(g[k], o[k], err_msg=k)
        np.testing.assert_allclose(g["end_state"], o["end_state"], rtol=1e-12, atol=1e-15)
    assert _deaths(g, inputs.E, "exit1") >= 1 and _deaths(g, inputs.E, "exit0") >= 1
    assert _deaths(g, inputs.E, "wall") >= 1
    assert _deaths(g, inputs.T2P, "stalled") == 1


def test_ion_workload_full_size_sampled(karl):
    """The default line's ion workload (131072 ions, the benchmark's launch):
    the GPU runs all of it; the oracle runs 16 sampled ranges of 64 ions with
    the same primary ids, whose collision counts and end states must match."""
    prob, orb, pr = inputs.orbit_ion_config(n_ions=1 << 17, seed=1)
    g = _gpu(karl, prob, orb, pr, seed=200)
    rng = np.random.default_rng(3)
    same = total = 0
    for a in rng.choice(pr.n // 64, 16, replace=False) * 64:
        sub = inputs.OrbitPrimaries(*(getattr(pr, k)[a:a + 64] for k in
                                      ("x_m", "y_m", "z_m", "e_ev", "mu", "phi", "species")),
                                    pid_offset=int(a))
        o = oracle.orbit_run(prob, orb, sub, seed=200, n_threads=THREADS)
        same += int(np.sum(o["per_primary"] == g["per_primary"][a:a + 64]))
        close = np.all(np.abs(o["end_state"] - g["end_state"][a:a + 64]) <=
                       1e-9 * (np.abs(o["end_state"]) + 1e-12), axis=1)
        same += int(np.sum(close))
        total += 128
    print(f"PARITY orbit ions full size: sampled counts and end states equal {same / total:.4f}")
    assert same / total >= 0.99
    E = g["energy"]
    e_in = E[karl.OE_IN_PRIMARY] + E[karl.OE_IN_THERMAL] + E[karl.OE_FIELD_WORK]
    assert abs(e_in - E[karl.OE_EXIT0:karl.OE_STALLED + 1].sum()) < 1e-9 * e_in
    L = g["ledger"]
    assert L[karl.OB_BIRTHS:karl.OB_BIRTHS + 4].sum() == L[karl.OB_DEATHS:karl.OB_DEATHS + 32].sum()
    assert np.all(g["time_z"].sum(axis=1) == g["time_r"].sum(axis=1))


def test_energy_bin_restarts_keep_the_free_path_law_on_the_gpu(karl):
    """The oracle pin's accelerated electrons through constant-cross-section
    gas: every energy-bin restart draws a new optical depth, so the
    uncollided fraction stays exp(-n sigma L); the GPU's flights, restarts
    and collision counts equal the oracle's."""
    n_m3, sigma, length = 2e20, 1e-20, 0.5
    nodes = inputs.energy_nodes(64, 100.0, 2e3)
    ch = [inputs.Channel("elastic", inputs.ELASTIC, inputs.E, -1, 0.0, np.full_like(nodes, sigma))]
    prob = inputs.uniform_problem(n_m3, length, 10, ch, n_energy=64, e_min=100.0, e_max=2e3,
                                  e_cut=0.0, n_tebins=32)
    prob.target_mass_ev = 1e18
    orb = _orbit(0.05, frac=0.1, tube_radius_m=1.0, n_rbins=4,
                 e_z_vm=np.full(prob.n_zbins, -2000.0))
    n = 6000
    pr = _prims(np.zeros(n), np.zeros(n), np.zeros(n), np.full(n, 150.0), np.ones(n),
                np.zeros(n), inputs.E)
    g = _gpu(karl, prob, orb, pr, seed=8)
    o = oracle.orbit_run(prob, orb, pr, seed=8, n_threads=THREADS)
    assert float(np.mean(g["per_primary"] == o["per_primary"])) >= 0.99
    p = math.exp(-n_m3 * sigma * length)
    k = int(np.sum(g["per_primary"] == 0))
    assert abs(k - n * p) < 5 * math.sqrt(n * p * (1 - p))


def test_orbit_shards_add_up_to_the_single_run(karl):
    """Two primary-id ranges run separately (with their id offsets) give
    tallies whose sum is the single run's, bit for bit: the per-rank step of
    shard.run_orbit_sharded on one device."""
    from paper_2503_10263_gb300 import shard
    prob, orb, pr = inputs.orbit_config(n_decays=200, seed=6)
    ctx = karl.Context(prob)
    try:
        full = ctx.run_orbit(orb, pr, seed=31)
        parts = []
        for rank in range(2):
            a, b = shard.shard_range(pr.n, rank, 2)
            sub = inputs.OrbitPrimaries(*(getattr(pr, k)[a:b].copy() for k in
                                          ("x_m", "y_m", "z_m", "e_ev", "mu", "phi", "species")),
                                        pid_offset=a)
            parts.append(ctx.run_orbit(orb, sub, seed=31))
    finally:
        ctx.close()
    for k in shard.ORBIT_RAW_KEYS:
        np.testing.assert_array_equal(parts[0][k] + parts[1][k], full[k], err_msg=k)
