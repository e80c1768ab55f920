"""Seeded synthetic inputs for the KARL transport step.

This module builds the problem descriptions that both the CUDA path and the
CPU oracle consume: geometry and gas profile, cross-section tables, species
masses and the primary particles of each decay.  It holds none of the
transport arithmetic (flights, channel choice, kinematics, tallies); it only
writes down inputs, so both sides can be fed identical data.

Every quantity is synthetic.  The paper's cross-section data (Yoon, Janev,
Rudd, Kim, Elsepa), its gas-flow profile and its KATRIN parameter file are not
available, so analytic Born-Bethe-form tables stand in for the data behind the
cross-section figures of Sec. 3.3, and a parabolic profile stands in for the
measured gas column (Sec. 5 example run: L = 16.57 m, B = 2.5 T).

Configurations (sizes follow the hot-path workloads):

* ``config1``: 1e4 beta electrons, uniform 1e19 m^-3 gas in a 10 m column,
  4 electron channels, FP64.
* ``config2``: 1e7 decays (one beta electron and one thermal T2+ each),
  parabolic profile with 5e21 m^-2 column, 7 electron channels, T2+ -> T3+
  clustering and electron-ion recombination (two passes).
* ``config3``: ``config1`` inputs, run in the FP32 precision form.
* ``config4_batch``: 256 source configurations of uneven size.
* ``config5_requests``: Poisson arrivals of config-4-style requests.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# ---------------------------------------------------------------------------
# physical constants (CODATA 2018) used to describe the inputs
AMU_EV = 931.49410242e6          # atomic mass unit, eV/c^2
ME_EV = 510998.95000             # electron rest energy, eV
M_T_ATOM_U = 3.01604928          # tritium atom mass, u
M_T2_EV = 2.0 * M_T_ATOM_U * AMU_EV          # neutral T2 (binding neglected)
M_T2P_EV = M_T2_EV - ME_EV                   # T2+
M_T3P_EV = 3.0 * M_T_ATOM_U * AMU_EV - ME_EV  # T3+
M_TP_EV = M_T_ATOM_U * AMU_EV - ME_EV         # T+
KB_EV_PER_K = 8.617333262e-5
ALPHA_FS = 7.2973525693e-3
PI_A0_SQ_M2 = math.pi * (5.29177210903e-11) ** 2   # 8.797e-21 m^2
RYDBERG_EV = 13.605693122994
T_HALF_S = 12.32 * 365.25 * 86400.0          # tritium half-life

# species and channel kinds (numeric values are part of the C ABI)
E, T2P, T3P, TP = 0, 1, 2, 3
N_SPECIES = 4
SPECIES_MASS_EV = np.array([ME_EV, M_T2P_EV, M_T3P_EV, M_TP_EV], dtype=np.float64)
SPECIES_NAMES = ("e-", "T2+", "T3+", "T+")

ELASTIC, IONIZATION, EXCITATION, CLUSTERING, RECOMBINATION = 0, 1, 2, 3, 4
CHARGE_EXCHANGE, CLUSTERING3 = 5, 6
KIND_NAMES = ("elastic", "ionization", "excitation", "clustering", "recombination",
              "charge_exchange", "clustering3")


@dataclasses.dataclass
class AngularTable:
    """Scattering-angle distribution of an elastic channel (Sec. 3.3
    Elastic): pdf values of cos(chi) on n_mu points evenly spaced over
    [-1, 1], one row per log-spaced impact-energy bin over [e_min, e_max];
    below threshold_ev the scattering is isotropic (a composition)."""
    e_min_ev: float
    e_max_ev: float
    pdf: np.ndarray                # [n_bins][n_mu]
    threshold_ev: float = 0.0


@dataclasses.dataclass
class Channel:
    name: str
    kind: int
    species_in: int
    species_out: int      # ionization: ion species produced (-1 none);
                          # clustering: product; recombination: partner field
    loss_ev: float
    sigma_m2: np.ndarray  # [n_energy] values at the table nodes
    target: int = 0       # 0 target at rest; 1 moving (thermal + gas drift), elastic only
    angular: Optional[AngularTable] = None   # elastic only; None = isotropic


@dataclasses.dataclass
class Problem:
    """One source configuration: geometry, gas, tables and run options."""
    name: str
    length_m: float
    n_zbins: int
    n_seg_m3: np.ndarray           # [n_zbins] piecewise-constant gas density
    area_m2: float
    activity_bq: float
    e_cut_ev: float
    max_collisions: int
    max_lifetime_s: float          # inf = no lifetime cap
    b_tesla: float
    gas_temperature_k: float
    n_tebins: int                  # energy bins of the time (density) tally
    n_spec_bins: int               # end-spectrum bins (+1 overflow)
    spec_bin_ev: float
    species_mass_ev: np.ndarray    # [4]
    target_mass_ev: float          # background gas molecule (T2)
    n_energy: int
    e_min_ev: float
    e_max_ev: float
    ioniz_eps_ev: float
    channels: List[Channel]
    n_passes: int = 1
    gas_drift_mps: float = 0.0     # drift velocity of the gas along +z

    @property
    def n_channels(self) -> int:
        return len(self.channels)

    def energy_nodes(self) -> np.ndarray:
        return energy_nodes(self.n_energy, self.e_min_ev, self.e_max_ev)

    def sigma_matrix(self) -> np.ndarray:
        return np.ascontiguousarray(
            np.stack([c.sigma_m2 for c in self.channels]).astype(np.float64))

    def column_m2(self) -> float:
        return float(np.sum(self.n_seg_m3) * self.length_m / self.n_zbins)


@dataclasses.dataclass
class Primaries:
    z_m: np.ndarray
    e_ev: np.ndarray
    mu: np.ndarray
    species: np.ndarray            # uint8
    n_decays: int

    @property
    def n(self) -> int:
        return int(self.z_m.shape[0])

    def slice(self, first: int, count: int) -> "Primaries":
        s = slice(first, first + count)
        return Primaries(self.z_m[s].copy(), self.e_ev[s].copy(), self.mu[s].copy(),
                         self.species[s].copy(), self.n_decays)


# ---------------------------------------------------------------------------
# cross-section tables (synthetic Born-Bethe form)

def energy_nodes(n: int, e_min: float, e_max: float) -> np.ndarray:
    i = np.arange(n, dtype=np.float64)
    return e_min * (e_max / e_min) ** (i / (n - 1))


def born_bethe(e: np.ndarray, e_k: float, m_k: float) -> np.ndarray:
    """pi a0^2 M (R/E) ln(E/E_k) above threshold, 0 at and below it."""
    out = np.zeros_like(e)
    on = e > e_k
    out[on] = PI_A0_SQ_M2 * m_k * (RYDBERG_EV / e[on]) * np.log(e[on] / e_k)
    return out


def elastic_sigma(e: np.ndarray, s0: float = 1e-19, e_s: float = 10.0) -> np.ndarray:
    return s0 / (1.0 + e / e_s)


def recomb_sigma(e: np.ndarray, s_r: float = 1e-20) -> np.ndarray:
    return s_r * (1.0 / e)


def rate_sigma(e: np.ndarray, k: float, m_ev: float) -> np.ndarray:
    """Cross section standing in for a rate coefficient (Sec. 3.3 Clustering:
    only rate coefficients are known, so the cross section is approximated):
    k / v(E) for an impactor of rest energy m_ev (relativistic speed).  A
    two-body k (m^3/s) gives m^2; a three-body k (m^6/s) gives the m^5
    coefficient of a CLUSTERING3 channel, whose rate per unit path is
    k n^2 / v."""
    x = e / m_ev
    v = 299792458.0 * np.sqrt(x * (2.0 + x)) / (1.0 + x)
    return k / v


def dissociative_ionization(nodes: np.ndarray, loss_ev: float = 18.1, m_k: float = 0.3) -> Channel:
    """e- + T2 -> e- + e- + T+ + T (Eq. ionization_diss): an ionization whose
    ion product is T+ (synthetic Born-Bethe table, 18.1 eV threshold)."""
    return Channel("dissociative_ionization", IONIZATION, E, TP, loss_ev,
                   born_bethe(nodes, loss_ev, m_k))


def electron_channels(nodes: np.ndarray, full: bool) -> List[Channel]:
    """Electron-T2 channels in table (selection) order."""
    ch = [Channel("elastic", ELASTIC, E, -1, 0.0, elastic_sigma(nodes)),
          Channel("ionization", IONIZATION, E, T2P if full else -1, 15.4,
                  born_bethe(nodes, 15.4, 4.2))]
    if full:
        for ek, m in ((8.9, 0.3), (11.4, 0.9), (12.6, 0.7)):
            ch.append(Channel(f"excitation_{ek}", EXCITATION, E, -1, ek,
                              born_bethe(nodes, ek, m)))
        ch.append(Channel("vibration", EXCITATION, E, -1, 0.5, born_bethe(nodes, 0.5, 0.05)))
        ch.append(Channel("rotation", EXCITATION, E, -1, 0.044, born_bethe(nodes, 0.044, 0.02)))
    else:
        ch.append(Channel("excitation", EXCITATION, E, -1, 12.6, born_bethe(nodes, 12.6, 1.6)))
        ch.append(Channel("vibration", EXCITATION, E, -1, 0.5, born_bethe(nodes, 0.5, 0.05)))
    return ch


def ion_channels(nodes: np.ndarray) -> List[Channel]:
    """Recombination (both directions) and T2+ + T2 -> T3+ clustering."""
    rec = recomb_sigma(nodes)
    return [
        Channel("recomb_e_T2+", RECOMBINATION, E, T2P, 0.0, rec.copy()),
        Channel("recomb_e_T3+", RECOMBINATION, E, T3P, 0.0, rec.copy()),
        Channel("clustering_T2+", CLUSTERING, T2P, T3P, 0.0, np.full_like(nodes, 1.91e-18)),
        Channel("recomb_T2+_e", RECOMBINATION, T2P, E, 0.0, rec.copy()),
        Channel("recomb_T3+_e", RECOMBINATION, T3P, E, 0.0, rec.copy()),
    ]


# ---------------------------------------------------------------------------
# gas profiles

def parabolic_segment_means(n0: float, length: float, nz: int) -> np.ndarray:
    """Exact mean of n0[1-(2z/L-1)^2] + 0.05 n0 over each of nz segments."""
    edges = np.linspace(0.0, length, nz + 1)
    u = 2.0 * edges / length - 1.0
    prim = u - u ** 3 / 3.0                    # antiderivative in u
    mean_par = (prim[1:] - prim[:-1]) / (u[1:] - u[:-1])
    return n0 * (mean_par + 0.05)


def parabolic_n0(column_m2: float, length: float) -> float:
    return column_m2 / ((2.0 / 3.0 + 0.05) * length)


def activity_for(column_m2: float, area_m2: float) -> float:
    """Decays/s of the T2 column: two tritium nuclei per molecule."""
    lam = math.log(2.0) / T_HALF_S
    return 2.0 * lam * column_m2 * area_m2


# ---------------------------------------------------------------------------
# primary generators

def beta_pdf(e_ev: np.ndarray, e0: float = 18600.0, z_daughter: int = 2) -> np.ndarray:
    """Allowed beta spectrum F(Z,E) p W (E0-E)^2 with the nonrelativistic
    Fermi function F = 2 pi eta / (1 - exp(-2 pi eta)), eta = Z alpha / beta."""
    e = np.asarray(e_ev, dtype=np.float64)
    w = e + ME_EV
    p = np.sqrt(np.maximum(w * w - ME_EV * ME_EV, 0.0))
    beta = np.where(w > 0, p / w, 0.0)
    out = np.zeros_like(e)
    ok = (e > 0) & (e < e0)
    eta = z_daughter * ALPHA_FS / beta[ok]
    fermi = 2.0 * math.pi * eta / (-np.expm1(-2.0 * math.pi * eta))
    out[ok] = fermi * p[ok] * w[ok] * (e0 - e[ok]) ** 2
    return out


_BETA_CDF = {}


def _beta_cdf(e0: float):
    """Tabulated CDF of the allowed spectrum on 2^18 + 1 points (trapezoid rule)."""
    if e0 not in _BETA_CDF:
        grid = np.linspace(0.0, e0, (1 << 18) + 1)
        pdf = beta_pdf(grid, e0)
        pdf[0] = beta_pdf(np.array([grid[1] * 1e-6]), e0)[0]   # finite limit at E -> 0
        cdf = np.concatenate([[0.0], np.cumsum(0.5 * (pdf[1:] + pdf[:-1]) * np.diff(grid))])
        _BETA_CDF[e0] = (grid, cdf / cdf[-1])
    return _BETA_CDF[e0]


def sample_beta(rng: np.random.Generator, n: int, e0: float = 18600.0) -> np.ndarray:
    """Allowed beta spectrum by inverse transform of its tabulated CDF."""
    grid, cdf = _beta_cdf(e0)
    e = np.interp(rng.uniform(0.0, 1.0, n), cdf, grid)
    return np.clip(e, grid[1] * 1e-3, e0 * (1.0 - 1e-12))


def sample_thermal_energy(rng: np.random.Generator, n: int, t_k: float) -> np.ndarray:
    """Maxwell-Boltzmann kinetic energies: Gamma(3/2, kT)."""
    return rng.gamma(1.5, KB_EV_PER_K * t_k, n)


def isotropic_mu(rng: np.random.Generator, n: int) -> np.ndarray:
    return rng.uniform(-1.0, 1.0, n)


def positions_by_density(rng: np.random.Generator, n: int, n_seg: np.ndarray,
                         length: float) -> np.ndarray:
    """Birth positions with probability proportional to the gas density:
    segment by inverse transform of the cumulative density, then uniform
    within the segment."""
    nz = n_seg.shape[0]
    cdf = np.cumsum(n_seg, dtype=np.float64)
    cdf /= cdf[-1]
    seg = np.minimum(np.searchsorted(cdf, rng.uniform(0.0, 1.0, n), side="right"), nz - 1)
    dz = length / nz
    return np.minimum((seg + rng.uniform(0.0, 1.0, n)) * dz, length)


# ---------------------------------------------------------------------------
# configurations

def _problem(name: str, length: float, nz: int, n_seg: np.ndarray, full: bool,
             n_energy: int = 2048, n_tebins: Optional[int] = None) -> Problem:
    nodes = energy_nodes(n_energy, 1.0, 2.0e4)
    chans = electron_channels(nodes, full)
    if full:
        chans += ion_channels(nodes)
    area = 1.0
    column = float(np.sum(n_seg) * length / nz)
    return Problem(
        name=name, length_m=length, n_zbins=nz, n_seg_m3=np.ascontiguousarray(n_seg, np.float64),
        area_m2=area, activity_bq=activity_for(column, area), e_cut_ev=1.0,
        max_collisions=1_000_000, max_lifetime_s=math.inf, b_tesla=2.5,
        gas_temperature_k=80.0, n_tebins=(64 if full else 1) if n_tebins is None else n_tebins,
        n_spec_bins=20000, spec_bin_ev=1.0, species_mass_ev=SPECIES_MASS_EV.copy(),
        target_mass_ev=M_T2_EV, n_energy=n_energy, e_min_ev=1.0, e_max_ev=2.0e4,
        ioniz_eps_ev=8.0, channels=chans, n_passes=2 if full else 1)


def screened_rutherford_table(e_min_ev: float = 100.0, e_max_ev: float = 2.0e4,
                              n_bins: int = 48, n_mu: int = 201, eta0_ev: float = 3.4,
                              threshold_ev: float = 100.0) -> AngularTable:
    """Synthetic stand-in for the paper's high-energy tables (its Elsepa data
    is not available): the screened Rutherford (Wentzel) form
    p(cos chi) ~ 1 / (1 + 2 eta - cos chi)^2 with eta = eta0 / E at each bin's
    geometric-mean energy, tabulated on n_mu points; isotropic below
    threshold_ev, as the paper composes them for electrons."""
    edges = np.geomspace(e_min_ev, e_max_ev, n_bins + 1)
    mid = np.sqrt(edges[:-1] * edges[1:])
    mu = np.linspace(-1.0, 1.0, n_mu)
    eta = eta0_ev / mid
    pdf = 1.0 / (1.0 + 2.0 * eta[:, None] - mu[None, :]) ** 2
    return AngularTable(e_min_ev, e_max_ev, np.ascontiguousarray(pdf), threshold_ev)


def angular_config(n_primaries: int = 2000, seed: int = 1):
    """Config-1 geometry and channels with the elastic channel's angles from a
    screened-Rutherford table above 100 eV (isotropic below)."""
    prob, prims = config1(n_primaries, seed)
    prob.name = "config1_angular"
    prob.channels[0].angular = screened_rutherford_table()
    return prob, prims


def thermalization(n_primaries: int = 4000, seed: int = 1, density_m3: float = 1e22,
                   length: float = 0.2, nz: int = 200, e_inj_ev: float = 8e-3,
                   sigma_m2: float = 1e-19, temperature_k: float = 80.0,
                   drift_mps: float = 0.0):
    """Elastic thermalisation (Sec. 4): mono-energetic electrons injected in
    the middle of a uniform T2 reservoir, moving along +z; elastic scattering
    on a moving (Maxwell-Boltzmann, drifting) target is the only channel, with
    a constant cross section; no energy cut, so every electron leaves through
    an end."""
    nodes = energy_nodes(64, 1e-5, 1.0)
    chans = [Channel("elastic_moving_target", ELASTIC, E, -1, 0.0,
                     np.full(nodes.shape, sigma_m2), target=1)]
    prob = Problem(
        name="thermalization", length_m=length, n_zbins=nz,
        n_seg_m3=np.full(nz, density_m3, np.float64), area_m2=1.0,
        activity_bq=activity_for(density_m3 * length, 1.0), e_cut_ev=0.0,
        max_collisions=100_000_000, max_lifetime_s=math.inf, b_tesla=2.5,
        gas_temperature_k=temperature_k, n_tebins=1, n_spec_bins=4000, spec_bin_ev=2.5e-5,
        species_mass_ev=SPECIES_MASS_EV.copy(), target_mass_ev=M_T2_EV, n_energy=64,
        e_min_ev=1e-5, e_max_ev=1.0, ioniz_eps_ev=8.0, channels=chans, n_passes=1,
        gas_drift_mps=drift_mps)
    z = np.full(n_primaries, 0.5 * length)
    e = np.full(n_primaries, e_inj_ev)
    mu = np.ones(n_primaries)
    return prob, Primaries(z, e, mu, np.zeros(n_primaries, np.uint8), n_primaries)


def config1(n_primaries: int = 10_000, seed: int = 1, density_m3: float = 1e19,
            length: float = 10.0, nz: int = 1000):
    """Plain method: uniform gas, four electron channels, beta electrons
    born uniformly along z with isotropic pitch."""
    prob = _problem("config1", length, nz, np.full(nz, density_m3), full=False)
    rng = np.random.default_rng(np.random.SeedSequence([seed, 1]))
    z = rng.uniform(0.0, length, n_primaries)
    e = sample_beta(rng, n_primaries)
    mu = isotropic_mu(rng, n_primaries)
    prims = Primaries(z, e, mu, np.zeros(n_primaries, np.uint8), n_primaries)
    return prob, prims


def config2(n_decays: int = 10_000_000, seed: int = 1, column_m2: float = 5e21,
            length: float = 10.0, nz: int = 1000):
    """Full-size plain method: parabolic profile, full channel set, one beta
    electron and one thermal T2+ per decay, both born where the gas is."""
    n0 = parabolic_n0(column_m2, length)
    prob = _problem("config2", length, nz, parabolic_segment_means(n0, length, nz), full=True)
    return prob, decay_primaries(prob, n_decays, seed)


def decay_primaries(prob: Problem, n_decays: int, seed: int) -> Primaries:
    rng = np.random.default_rng(np.random.SeedSequence([seed, 2]))
    z = positions_by_density(rng, n_decays, prob.n_seg_m3, prob.length_m)
    e_beta = sample_beta(rng, n_decays)
    mu_e = isotropic_mu(rng, n_decays)
    e_ion = sample_thermal_energy(rng, n_decays, prob.gas_temperature_k)
    mu_i = isotropic_mu(rng, n_decays)
    # interleave: decay d -> particle 2d (electron), 2d+1 (T2+)
    zz = np.repeat(z, 2)
    ee = np.empty(2 * n_decays); ee[0::2] = e_beta; ee[1::2] = e_ion
    mm = np.empty(2 * n_decays); mm[0::2] = mu_e; mm[1::2] = mu_i
    sp = np.empty(2 * n_decays, np.uint8); sp[0::2] = E; sp[1::2] = T2P
    return Primaries(zz, ee, mm, sp, n_decays)


def config3(n_primaries: int = 10_000, seed: int = 1):
    """Config 1 inputs; the precision form is a run option."""
    prob, prims = config1(n_primaries, seed)
    prob.name = "config3"
    return prob, prims


def config4_batch(n_configs: int = 256, meta_seed: int = 1, np_lo: float = 1e3,
                  np_hi: float = 1e6, nz: int = 1000):
    """Uneven batch of source configurations: column 0.1-1.0 x 5e21 m^-2,
    length 2-10 m, decays log-uniform in [np_lo, np_hi]."""
    rng = np.random.default_rng(np.random.SeedSequence([meta_seed, 4]))
    out = []
    for i in range(n_configs):
        col = rng.uniform(0.1, 1.0) * 5e21
        length = rng.uniform(2.0, 10.0)
        nd = int(round(math.exp(rng.uniform(math.log(np_lo), math.log(np_hi)))))
        n0 = parabolic_n0(col, length)
        prob = _problem(f"config4_{i}", length, nz, parabolic_segment_means(n0, length, nz),
                        full=True)
        seed = (meta_seed << 32) + i
        out.append((prob, decay_primaries(prob, nd, seed), seed))
    return out


def config5_requests(duration_s: float = 60.0, rate_hz: float = 50.0, arrival_seed: int = 1,
                     np_lo: float = 1e3, np_hi: float = 1e6, nz: int = 1000,
                     max_requests: Optional[int] = None):
    """Poisson arrivals of config-4-style requests: (t_arrival, problem,
    primaries, seed)."""
    rng = np.random.default_rng(np.random.SeedSequence([arrival_seed, 5]))
    t = 0.0
    out = []
    i = 0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > duration_s or (max_requests is not None and i >= max_requests):
            break
        col = rng.uniform(0.1, 1.0) * 5e21
        length = rng.uniform(2.0, 10.0)
        nd = int(round(math.exp(rng.uniform(math.log(np_lo), math.log(np_hi)))))
        n0 = parabolic_n0(col, length)
        prob = _problem(f"req_{i}", length, nz, parabolic_segment_means(n0, length, nz),
                        full=True)
        seed = (arrival_seed << 32) + i
        out.append((t, prob, decay_primaries(prob, nd, seed), seed))
        i += 1
    return out


# ---------------------------------------------------------------------------
# small test problems

def uniform_problem(n_seg_m3: float, length: float, nz: int, channels: List[Channel],
                    n_energy: int = 2048, e_min: float = 1.0, e_max: float = 2.0e4,
                    e_cut: float = 1.0, n_tebins: int = 1, n_passes: int = 1,
                    n_spec_bins: int = 20000, spec_bin_ev: float = 1.0,
                    max_collisions: int = 1_000_000, max_lifetime_s: float = math.inf) -> Problem:
    n_seg = np.full(nz, float(n_seg_m3))
    column = float(np.sum(n_seg) * length / nz)
    return Problem(
        name="test", length_m=length, n_zbins=nz, n_seg_m3=n_seg, area_m2=1.0,
        activity_bq=activity_for(column, 1.0) if column > 0 else 1.0, e_cut_ev=e_cut,
        max_collisions=max_collisions, max_lifetime_s=max_lifetime_s, b_tesla=2.5,
        gas_temperature_k=80.0, n_tebins=n_tebins, n_spec_bins=n_spec_bins,
        spec_bin_ev=spec_bin_ev, species_mass_ev=SPECIES_MASS_EV.copy(),
        target_mass_ev=M_T2_EV, n_energy=n_energy, e_min_ev=e_min, e_max_ev=e_max,
        ioniz_eps_ev=8.0, channels=channels, n_passes=n_passes)


def beam(n: int, z0: float, e_ev: float, mu: float, species: int = E) -> Primaries:
    return Primaries(np.full(n, z0), np.full(n, e_ev), np.full(n, mu),
                     np.full(n, species, np.uint8), n)


# ---------------------------------------------------------------------------
# ion chemistry (Sec. 3.3 Clustering, Charge exchange, Ionization)

def ion_chemistry_channels(nodes: np.ndarray, k_ter: float = 2.6e-41,
                           sigma_cx: float = 1e-18) -> List[Channel]:
    """T+ from dissociative ionization, its three-body clustering to T3+
    (table k_ter / v) and its recombination with the electron field, and
    T2+ charge exchange (constant synthetic cross section)."""
    return [dissociative_ionization(nodes),
            Channel("clustering3_T+", CLUSTERING3, TP, T3P, 0.0, rate_sigma(nodes, k_ter, M_TP_EV)),
            Channel("recomb_T+_e", RECOMBINATION, TP, E, 0.0, recomb_sigma(nodes)),
            Channel("charge_exchange_T2+", CHARGE_EXCHANGE, T2P, -1, 0.0,
                    np.full_like(nodes, sigma_cx))]


def chemistry_config(n_decays: int = 3000, seed: int = 1, column_m2: float = 2e21,
                     length: float = 4.0, nz: int = 100, k_ter: float = 2.6e-39):
    """Config-2 physics plus the further ion chemistry of ion_chemistry_channels,
    with the three-body rate raised (default 100 x the paper's 2.6e-41 m^6/s)
    so that T+ clusters within the column; two passes."""
    n0 = parabolic_n0(column_m2, length)
    prob = _problem("chemistry", length, nz, parabolic_segment_means(n0, length, nz), full=True)
    prob.channels += ion_chemistry_channels(prob.energy_nodes(), k_ter=k_ter)
    return prob, decay_primaries(prob, n_decays, seed)


def ion_beam_problem(chans: List[Channel], n_seg: np.ndarray, length: float, e_min: float,
                     e_max: float, **kw) -> Problem:
    """Ion test geometry: the given gas profile, 64-node tables over
    [e_min, e_max], no energy cut."""
    prob = uniform_problem(1.0, length, len(n_seg), chans, n_energy=64, e_min=e_min, e_max=e_max,
                           e_cut=0.0, **kw)
    prob.n_seg_m3 = np.asarray(n_seg, np.float64)
    return prob


def charge_exchange_problem(n_m3: float, length: float, nz: int, t_k: float,
                            sigma_m2: float = 1e-19, **kw) -> Problem:
    """T2+ charge exchange as the only channel (constant cross section) in a
    uniform T2 gas at temperature t_k."""
    nodes = energy_nodes(64, 1e-5, 100.0)
    ch = Channel("cx", CHARGE_EXCHANGE, T2P, -1, 0.0, np.full_like(nodes, sigma_m2))
    prob = ion_beam_problem([ch], np.full(nz, n_m3), length, 1e-5, 100.0, **kw)
    prob.gas_temperature_k = t_k
    return prob


# ---------------------------------------------------------------------------
# full-orbit transport in a tube (Sec. 3.1 Boris mover; Sec. 5 tube currents)

C_LIGHT_MPS = 299792458.0


@dataclasses.dataclass
class Orbit:
    """Fields and tube of a full-orbit run: uniform B along +z, the electric
    field E = (e_r x, e_r y, e_z[segment]), a beam tube of radius R with
    n_rbins radial bins, and the Boris time step of each species."""
    b_t: float
    tube_radius_m: float
    n_rbins: int
    dt_s: np.ndarray                 # [4]
    e_z_vm: Optional[np.ndarray] = None   # [n_zbins] or None (no axial field)
    e_r_vm2: float = 0.0
    max_steps: int = 0               # steps per flight before "stalled"; 0 = 2^40


@dataclasses.dataclass
class OrbitPrimaries:
    x_m: np.ndarray
    y_m: np.ndarray
    z_m: np.ndarray
    e_ev: np.ndarray
    mu: np.ndarray                   # cosine of the angle to +z
    phi: np.ndarray                  # azimuth of the transverse velocity
    species: np.ndarray              # uint8
    pid_offset: int = 0

    @property
    def n(self) -> int:
        return int(self.z_m.shape[0])


def boris_dt(b_t: float, frac: float = 0.1) -> np.ndarray:
    """Time step per species: frac / Omega_max, Omega_max = e B / m the
    largest gyro frequency of the species (at rest), so that
    dt < 1 / Omega_g,max (Eq. boris_timestep_requirement)."""
    omega = abs(b_t) * C_LIGHT_MPS ** 2 / SPECIES_MASS_EV
    return np.ascontiguousarray(frac / np.maximum(omega, 1e-300), np.float64)


def ion_elastic_channels(nodes: np.ndarray, sigma_t2p: float = 3e-19,
                         sigma_t3p: float = 3e-19) -> List[Channel]:
    """Synthetic elastic scattering of T2+ and T3+ on T2 (constant cross
    sections; the paper notes ion scattering cross sections far above the
    electrons')."""
    return [Channel("elastic_T2+", ELASTIC, T2P, -1, 0.0, np.full_like(nodes, sigma_t2p)),
            Channel("elastic_T3+", ELASTIC, T3P, -1, 0.0, np.full_like(nodes, sigma_t3p))]


def orbit_config(n_decays: int = 100_000, seed: int = 1, length: float = 1.0, nz: int = 100,
                 density_m3: float = 5e19, b_t: float = 0.25, tube_radius_m: float = 0.045,
                 n_rbins: int = 45, e_r_vm2: float = 20.0, lifetime_s: float = 2e-4):
    """Tube section for the full-orbit mover: uniform T2 gas, the seven
    electron channels with T2+ ionization, T2+ -> T3+ clustering and ion
    elastic scattering; a beam tube of 45 mm radius (the WGTS tube), a
    radial field of a weak space-charge potential and B = 0.25 T (a tenth of
    the Sec. 5 example, to keep the number of steps per gyration affordable).
    One beta electron and one thermal T2+ per decay, born uniformly over the
    cross section and along z, isotropic (those born within two gyration
    radii of the wall can reach it); a lifetime cap ends slow ions that
    random-walk for long."""
    nodes = energy_nodes(2048, 1.0, 2.0e4)
    chans = electron_channels(nodes, True)
    chans.append(Channel("clustering_T2+", CLUSTERING, T2P, T3P, 0.0, np.full_like(nodes, 1.91e-18)))
    chans += ion_elastic_channels(nodes)
    prob = uniform_problem(density_m3, length, nz, chans, max_lifetime_s=lifetime_s)
    prob.name = "orbit_tube"
    prob.b_tesla = b_t
    orbit = Orbit(b_t=b_t, tube_radius_m=tube_radius_m, n_rbins=n_rbins, dt_s=boris_dt(b_t),
                  e_r_vm2=e_r_vm2)
    rng = np.random.default_rng(np.random.SeedSequence([seed, 6]))
    n = 2 * n_decays
    r = tube_radius_m * np.sqrt(rng.uniform(0.0, 1.0, n))
    a = rng.uniform(0.0, 2.0 * math.pi, n)
    z = rng.uniform(0.0, length, n)
    e = np.empty(n)
    e[0::2] = sample_beta(rng, n_decays)
    e[1::2] = sample_thermal_energy(rng, n_decays, prob.gas_temperature_k)
    sp = np.empty(n, np.uint8)
    sp[0::2] = E
    sp[1::2] = T2P
    prims = OrbitPrimaries(r * np.cos(a), r * np.sin(a), z, e, isotropic_mu(rng, n),
                           rng.uniform(0.0, 2.0 * math.pi, n), sp)
    return prob, orbit, prims


def orbit_ion_config(n_ions: int = 1 << 20, seed: int = 1, length: float = 1.0, nz: int = 100,
                     density_m3: float = 5e19, b_t: float = 2.5, tube_radius_m: float = 0.045,
                     n_rbins: int = 45, e_r_vm2: float = 2e3, lifetime_s: float = 1e-4):
    """Ions in a tube section for the full-orbit mover at the Sec. 5 field
    (B = 2.5 T): thermal T2+ born uniformly over the cross section and along
    z, isotropic, in uniform T2 gas; T2+ -> T3+ clustering and ion elastic
    scattering; a 45 mm tube with a radial field (E x B rotation of about
    800 rad/s); the lifetime cap of 1e-4 s bounds every history to about
    4e4 Boris steps, so the histories are of similar length."""
    nodes = energy_nodes(64, 1e-5, 100.0)
    chans = [Channel("clustering_T2+", CLUSTERING, T2P, T3P, 0.0, np.full_like(nodes, 1.91e-18))]
    chans += ion_elastic_channels(nodes)
    prob = uniform_problem(density_m3, length, nz, chans, n_energy=64, e_min=1e-5, e_max=100.0,
                           e_cut=0.0, max_lifetime_s=lifetime_s, n_spec_bins=1000,
                           spec_bin_ev=1e-3)
    prob.name = "orbit_ions"
    prob.b_tesla = b_t
    orbit = Orbit(b_t=b_t, tube_radius_m=tube_radius_m, n_rbins=n_rbins, dt_s=boris_dt(b_t),
                  e_r_vm2=e_r_vm2)
    rng = np.random.default_rng(np.random.SeedSequence([seed, 7]))
    r = tube_radius_m * np.sqrt(rng.uniform(0.0, 1.0, n_ions))
    a = rng.uniform(0.0, 2.0 * math.pi, n_ions)
    prims = OrbitPrimaries(r * np.cos(a), r * np.sin(a), rng.uniform(0.0, length, n_ions),
                           sample_thermal_energy(rng, n_ions, prob.gas_temperature_k),
                           isotropic_mu(rng, n_ions), rng.uniform(0.0, 2.0 * math.pi, n_ions),
                           np.full(n_ions, T2P, np.uint8))
    return prob, orbit, prims
