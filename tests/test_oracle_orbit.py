"""Pins of the oracle's full-orbit mode (the Boris mover of Sec. 3.1) against
closed forms of charged-particle motion and transport, and against the
oracle's guiding-centre transport where the two must agree in law.

Each case fixes a different part of the mover: the gyration radius (with its
relativistic gamma) and the sense of rotation for both charge signs, the
relativistic parallel speed, the work of an axial electric field with the
hyperbolic motion of a constant force, the exact slow (E x B) rotation in a
linear radial field, the classical cross-field diffusion coefficient of
isotropic scattering, attenuation along the field, and the ledgers."""
import math

import numpy as np
import pytest

import oracle
from paper_2503_10263_gb300 import inputs

C = 299792458.0
Q_TIME = 2.0 ** 50


def _vacuum(length=1.0, nz=10, lifetime=math.inf):
    nodes = inputs.energy_nodes(64, 1e-4, 1e5)
    ch = [inputs.Channel("elastic", inputs.ELASTIC, inputs.E, -1, 0.0, np.full_like(nodes, 1e-20))]
    prob = inputs.uniform_problem(0.0, length, nz, ch, n_energy=64, e_min=1e-4, e_max=1e5,
                                  e_cut=0.0, max_lifetime_s=lifetime, n_spec_bins=4000,
                                  spec_bin_ev=1.0)
    return prob


def _prims(x, y, z, e, mu, phi, sp):
    n = len(x)
    f = lambda v: np.ascontiguousarray(np.broadcast_to(np.asarray(v, np.float64), (n,)))
    return inputs.OrbitPrimaries(f(x), f(y), f(z), f(e), f(mu), f(phi),
                                 np.ascontiguousarray(np.broadcast_to(np.uint8(sp), (n,))))


def _omega(b_t, e_ev, m_ev):
    """Relativistic gyro frequency e B / (gamma m) (rad/s)."""
    return b_t * C * C / (m_ev + e_ev)


def _orbit(b_t, frac=0.01, **kw):
    return inputs.Orbit(b_t=b_t, dt_s=inputs.boris_dt(b_t, frac), **kw)


def _deaths(t, species, reason):
    return int(t["ledger"][oracle.OB_DEATHS + 8 * species + oracle.ORBIT_REASONS.index(reason)])


@pytest.mark.parametrize("species,e_ev", [(inputs.E, 18600.0), (inputs.T2P, 10.0)])
def test_gyration_radius_and_sense_decide_wall_hits(species, e_ev):
    """A particle whose gyration circle (radius p_perp / (|q| B), centre on the
    side v x z for q > 0) reaches to d + r_L from the axis hits a wall at
    0.98 of that and misses one at 1.02 of it.  With the opposite sense of
    rotation the centre moves by 2 r_L and both outcomes flip; without the
    relativistic gamma the 18.6 keV electron's radius is 3.6 % short."""
    m = inputs.SPECIES_MASS_EV[species]
    b = 0.5
    mu = 0.2
    pc = math.sqrt(e_ev * (e_ev + 2 * m))               # eV
    r_l = pc * math.sqrt(1 - mu * mu) / (C * b)          # p_perp / (e B), m
    sgn = -1.0 if species == inputs.E else 1.0
    d = 5.0 * r_l
    # centre = x0 + sgn r_L (v x z): with v_perp along sgn y, v x z = sgn x, so
    # the particle starts at the point of its circle nearest the axis
    phi = sgn * 0.5 * math.pi
    x0 = d - r_l
    omega = _omega(b, e_ev, m)
    v_par = C * pc / (e_ev + m) * mu
    length = 8 * 2 * math.pi / omega * v_par             # eight gyrations before z = L
    prob = _vacuum(length=length)
    for scale, wall in ((0.98, True), (1.02, False)):
        orb = _orbit(b, tube_radius_m=(d + r_l) * scale, n_rbins=4)
        t = oracle.orbit_run(prob, orb, _prims([x0], [0.0], [0.0], [e_ev], [mu], [phi], species))
        assert _deaths(t, species, "wall") == (1 if wall else 0)
        assert _deaths(t, species, "exit1") == (0 if wall else 1)


@pytest.mark.parametrize("e_ev", [1000.0, 18600.0])
def test_parallel_transit_time_is_relativistic(e_ev):
    """In vacuum the time from z0 to L is (L - z0) / (mu v) with the
    relativistic speed, and the radial time tally holds the same total."""
    m = inputs.ME_EV
    mu, z0, length = 0.7, 0.1, 1.0
    prob = _vacuum(length=length)
    orb = _orbit(0.5, tube_radius_m=0.05, n_rbins=5)
    t = oracle.orbit_run(prob, orb, _prims([0.0], [0.0], [z0], [e_ev], [mu], [1.0], inputs.E))
    v = C * math.sqrt(e_ev * (e_ev + 2 * m)) / (e_ev + m)
    expect = (length - z0) / (mu * v) * Q_TIME
    got = float(t["time_z"].sum())
    assert got == float(t["time_r"].sum())
    # every run of steps in one cell is rounded once to the 2^-50 s unit
    tol = 0.5 * (prob.n_zbins + 2 * orb.n_rbins + 2) + 1e-12 * expect
    assert abs(got - expect) < tol
    newton = (length - z0) / (mu * C * math.sqrt(2 * e_ev / m)) * Q_TIME
    assert abs(newton - expect) > 1e3 * tol
    assert _deaths(t, inputs.E, "exit1") == 1


@pytest.mark.parametrize("e0,ez,e_end", [(100.0, -1000.0, 1100.0), (2000.0, 1000.0, 1000.0)])
def test_axial_field_work_and_hyperbolic_motion(e0, ez, e_end):
    """An electron along B in a uniform axial field E_z gains -e E_z L of
    kinetic energy over the column (field-work ledger and exit spectrum), and
    its transit time is that of a constant force: t = (p_f - p_0) / (e |E_z|),
    momenta from the relativistic energies."""
    m = inputs.ME_EV
    length, n = 1.0, 4
    prob = _vacuum(length=length)
    orb = _orbit(0.5, tube_radius_m=0.05, n_rbins=5, e_z_vm=np.full(prob.n_zbins, ez))
    t = oracle.orbit_run(prob, orb, _prims([0.0] * n, [0.0] * n, [0.0] * n, [e0] * n, [1.0] * n,
                                           [0.0] * n, inputs.E))
    assert _deaths(t, inputs.E, "exit1") == n
    e_exit = t["energy"][oracle.OE_EXIT1] / n
    assert abs(e_exit - e_end) < 1e-4 * e_end
    assert abs(t["energy"][oracle.OE_FIELD_WORK] / n - (e_end - e0)) < 1e-4 * e_end
    assert t["spectrum"][1, inputs.E, int(e_end - 1)] + t["spectrum"][1, inputs.E, int(e_end)] == n
    pc0, pc1 = (math.sqrt(e * (e + 2 * m)) for e in (e0, e_end))
    t_exp = abs(pc1 - pc0) / (C * abs(ez)) * Q_TIME
    assert abs(float(t["time_z"].sum()) / n - t_exp) < 1e-4 * t_exp


def test_exb_rotation_in_a_linear_radial_field():
    """In E = e_r (x, y, 0) and B along z, w = x + i y obeys
    w'' = kappa w - i Omega w' (kappa = q e_r / m, Omega = q B / m); started on
    the slow mode w = r0 exp(i omega_s t), omega_s = (-Omega + sqrt(Omega^2 -
    4 kappa)) / 2 (about -e_r / B, the E x B rotation), an ion keeps its
    radius and turns by omega_s T until the lifetime cap T."""
    m = inputs.M_T3P_EV
    b, e_r, r0, t_cap = 0.5, 1e4, 0.01, 1e-4
    om = b * C * C / m
    kappa = e_r * C * C / m
    om_s = 0.5 * (-om + math.sqrt(om * om - 4.0 * kappa))
    assert abs(om_s + e_r / b) < 0.01 * abs(om_s)        # close to, but not, the drift limit
    v = abs(om_s) * r0
    e_kin = m * (1.0 / math.sqrt(1.0 - (v / C) ** 2) - 1.0)
    prob = _vacuum(length=1.0, lifetime=t_cap)
    orb = _orbit(b, tube_radius_m=0.05, n_rbins=5, e_r_vm2=e_r)
    phi = 0.5 * math.pi if om_s > 0 else -0.5 * math.pi
    t = oracle.orbit_run(prob, orb, _prims([r0], [0.0], [0.5], [e_kin], [0.0], [phi], inputs.T3P))
    assert _deaths(t, inputs.T3P, "cap_time") == 1
    x, y = t["end_state"][0, 0], t["end_state"][0, 1]
    turned = math.atan2(y, x)
    expect = math.remainder(om_s * t_cap, 2 * math.pi)
    assert abs(math.remainder(turned - expect, 2 * math.pi)) < 2e-3 * abs(om_s * t_cap)
    assert abs(math.hypot(x, y) - r0) < 1e-3 * r0
    drift_only = math.remainder(-e_r / b * t_cap, 2 * math.pi)
    assert abs(math.remainder(turned - drift_only, 2 * math.pi)) > 5e-3


def _msd_closed_form(v, nu, omega, t):
    """<x^2 + y^2>(t) for a stationary velocity with correlation
    (v^2/3) exp(-nu s) cos(omega s) per transverse component:
    2 * 2 Re[int_0^t (t - s) exp(-lambda s) ds], lambda = nu - i omega."""
    lam = complex(nu, -omega)
    inner = t / lam - (1.0 - np.exp(-lam * t)) / lam ** 2
    return 4.0 * v * v / 3.0 * inner.real


@pytest.mark.parametrize("ratio", [0.5, 3.0])
def test_cross_field_diffusion(ratio):
    """Electrons scattered isotropically (a heavy target, so the speed stays)
    at the rate nu = n sigma v and gyrating at Omega = ratio nu spread across
    B as the classical result: the velocity correlation (v^2/3) e^(-nu s)
    cos(Omega s) integrated twice (Omega of the discrete rotation,
    2 atan(Omega dt / 2) / dt).  Ratio 3 cuts the spread by about ten against
    the field-free walk."""
    m = inputs.ME_EV
    e, n_m3, sigma = 100.0, 1e20, 1e-19
    v = C * math.sqrt(e * (e + 2 * m)) / (e + m)
    nu = n_m3 * sigma * v
    om = ratio * nu
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
    n = 4000
    rng = np.random.default_rng(11)
    pr = _prims(np.zeros(n), np.zeros(n), np.full(n, 500.0), np.full(n, e),
                rng.uniform(-1, 1, n), rng.uniform(0, 2 * math.pi, n), inputs.E)
    t = oracle.orbit_run(prob, orb, pr, seed=3, n_threads=4)
    assert _deaths(t, inputs.E, "cap_time") == n
    r2 = t["end_state"][:, 0] ** 2 + t["end_state"][:, 1] ** 2
    expect = _msd_closed_form(v, nu, om_eff, t_cap)
    se = r2.std() / math.sqrt(n)
    assert abs(r2.mean() - expect) < 5 * se
    free = _msd_closed_form(v, nu, 0.0, t_cap)
    assert abs(r2.mean() - free) > 5 * se


def test_attenuation_along_b():
    """Gyrating electrons at pitch cosine mu cross a uniform gas column
    without a collision with probability exp(-n sigma L / mu): the path per
    unit length along B is 1 / mu."""
    m = inputs.ME_EV
    e, mu, n_m3, sigma, length = 300.0, 0.6, 1e20, 1e-20, 0.5
    nodes = inputs.energy_nodes(64, 1.0, 1e3)
    ch = [inputs.Channel("elastic", inputs.ELASTIC, inputs.E, -1, 0.0, np.full_like(nodes, sigma))]
    prob = inputs.uniform_problem(n_m3, length, 20, ch, n_energy=64, e_min=1.0, e_max=1e3,
                                  e_cut=0.0)
    orb = _orbit(0.01, frac=0.1, tube_radius_m=1.0, n_rbins=4)
    n = 6000
    pr = _prims(np.zeros(n), np.zeros(n), np.zeros(n), np.full(n, e), np.full(n, mu),
                np.linspace(0, 2 * math.pi, n), inputs.E)
    t = oracle.orbit_run(prob, orb, pr, seed=5, n_threads=4)
    p = math.exp(-n_m3 * sigma * length / mu)
    k = int(np.sum(t["per_primary"] == 0))
    assert abs(k - n * p) < 5 * math.sqrt(n * p * (1 - p))


def test_orbit_ledgers_and_tally_invariants():
    """Tube section with ionization, clustering and ion scattering: the
    energy ledger balances (in + field work = out), every birth ends once,
    spectra and end-face crossings count the z exits, the wall tally and the
    outermost radial crossing count the wall deaths, channel counts sum to
    the collisions, and the z and radial time tallies hold the same time."""
    prob, orb, pr = inputs.orbit_config(n_decays=150, seed=2)
    t = oracle.orbit_run(prob, orb, pr, seed=2, n_threads=4)
    E = t["energy"]
    e_in = E[oracle.OE_IN_PRIMARY] + E[oracle.OE_IN_THERMAL] + E[oracle.OE_FIELD_WORK]
    e_out = E[oracle.OE_EXIT0:oracle.OE_STALLED + 1].sum()
    assert abs(e_in - e_out) < 1e-9 * E[oracle.OE_IN_PRIMARY]
    L = t["ledger"]
    deaths = L[oracle.OB_DEATHS:oracle.OB_DEATHS + 32].reshape(4, 8)
    births = L[oracle.OB_BIRTHS:oracle.OB_BIRTHS + 4]
    assert births.sum() == deaths.sum()
    assert births[inputs.E] == pr.n // 2 + L[oracle.OB_N_SPAWN_E]
    assert L[oracle.OB_N_COLLISIONS] == t["chan_count"].sum() > 0
    for s in range(4):
        assert t["spectrum"][0, s].sum() == deaths[s, 0] == t["cross_neg"][s, 0]
        assert t["spectrum"][1, s].sum() == deaths[s, 1] == t["cross_pos"][s, -1]
        assert t["wall"][s].sum() == deaths[s, 2] == t["rcross_out"][s, -1]
        assert t["time_z"][s].sum() == t["time_r"][s].sum()
    assert deaths[:, 2].sum() > 0 and deaths[inputs.T2P, 6] > 0
    assert L[oracle.OB_N_STEPS] > 100 * L[oracle.OB_N_FLIGHTS]


def test_orbit_reproduces_guiding_centre_histories():
    """In a uniform B without electric field and in uniform gas the full-orbit
    mover moves along z exactly as the guiding centre does (path per unit z
    is 1 / |mu|, the same optical depth per flight, the same random numbers,
    the pitch update of the same form), so the two forms follow the same
    histories: collision counts per primary agree for nearly all primaries
    and the end spectra agree within Poisson noise."""
    prob, prims = inputs.config1(n_primaries=600, seed=4, density_m3=2e20, length=0.5, nz=50)
    prims.e_ev[:] = np.linspace(50.0, 600.0, prims.n)
    orb = _orbit(0.02, frac=0.1, tube_radius_m=5.0, n_rbins=4)
    rng = np.random.default_rng(9)
    pr = inputs.OrbitPrimaries(np.zeros(prims.n), np.zeros(prims.n), prims.z_m.copy(),
                               prims.e_ev.copy(), prims.mu.copy(),
                               rng.uniform(0, 2 * math.pi, prims.n), prims.species.copy())
    a = oracle.orbit_run(prob, orb, pr, seed=7, n_threads=4)
    g = oracle.run(prob, prims, seed=7, n_threads=4)
    same = np.mean(a["per_primary"] == g["per_primary"])
    assert same > 0.95, same
    sa = a["spectrum"].astype(float).sum(axis=(1,))
    sg = g["spectrum"].astype(float).sum(axis=(1,))
    assert abs(sa.sum() - sg.sum()) <= 3 * math.sqrt(sa.sum() + sg.sum())
    ta, tg = a["time_z"][inputs.E].astype(float), g["time_fx"][inputs.E, 1:-1, 0].astype(float)
    assert abs(ta.sum() - tg.sum()) < 0.02 * tg.sum()


def test_flight_restarts_at_each_energy_bin():
    """With an electric field a flight ends when the kinetic energy leaves its
    bin of the time tally's energy grid and a new distance is drawn (Sec. 3.1
    stop rule): an electron accelerated from 100 eV to 1100 eV through
    vacuum over 64 log bins of [1 eV, 20 keV] flies once per bin it passes."""
    m = inputs.ME_EV
    nodes = inputs.energy_nodes(64, 1.0, 2e4)
    ch = [inputs.Channel("elastic", inputs.ELASTIC, inputs.E, -1, 0.0, np.full_like(nodes, 1e-20))]
    prob = inputs.uniform_problem(0.0, 1.0, 10, ch, n_energy=64, e_min=1.0, e_max=2e4,
                                  e_cut=0.0, n_tebins=64, n_spec_bins=4000, spec_bin_ev=1.0)
    orb = _orbit(0.5, tube_radius_m=0.05, n_rbins=5, e_z_vm=np.full(prob.n_zbins, -1000.0))
    t = oracle.orbit_run(prob, orb, _prims([0.0], [0.0], [0.0], [100.0], [1.0], [0.0], inputs.E))
    b = [math.floor(math.log(e) / math.log(2e4) * 64) for e in (100.0, 1100.0)]
    assert int(t["ledger"][oracle.OB_N_FLIGHTS]) == b[1] - b[0] + 1 == 17
    assert abs(t["energy"][oracle.OE_EXIT1] - 1100.0) < 0.11


def test_energy_bin_restarts_keep_the_free_path_law():
    """Electrons accelerated along B through uniform gas of constant cross
    section restart their flight at each energy bin they pass (32 bins over
    [100 eV, 2 keV] here); a new optical depth is drawn each time, so, the
    exponential law being memoryless, the fraction crossing the column
    without a collision is still exp(-n sigma L).  Reusing the first draw
    would let far more through."""
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
    t = oracle.orbit_run(prob, orb, pr, seed=8, n_threads=4)
    assert t["ledger"][oracle.OB_N_FLIGHTS] > 5 * n           # restarts happened
    p = math.exp(-n_m3 * sigma * length)
    k = int(np.sum(t["per_primary"] == 0))
    assert abs(k - n * p) < 5 * math.sqrt(n * p * (1 - p))
