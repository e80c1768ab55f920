"""ctypes loader for the FP64 CPU oracle (``oracle/karl_oracle.cpp``).

TEST INFRASTRUCTURE ONLY.  The oracle is the correctness reference for the
CUDA path: only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline may import this module.  The product package never does.

``build()`` compiles the oracle in-tree with g++ (FP contraction off so the
x86 and Arm builds round the same way).  ``run()`` marshals a problem from
``paper_2503_10263_gb300.inputs`` into the oracle's own C structs and returns
the tallies as numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "karl_oracle.cpp")
_HDR = os.path.join(_HERE, "karl_oracle.h")
_LIB = os.path.join(_HERE, "libkarl_oracle.so")

N_SPECIES = 4
N_REASONS = 8
LEDGER_LEN = 64
# ledger slots (mirrors karl_oracle.h)
E_IN_PRIMARY, E_IN_THERMAL, E_EXIT0, E_EXIT1, E_CUTOFF, E_CAP, E_RECOMB, E_CLUSTER, \
    E_LOSS_IONIZ, E_LOSS_EXCIT, E_LOSS_RECOIL, E_STALLED = range(12)
BIRTHS = 12
DEATHS = 16
N_COLLISIONS, N_FLIGHTS, N_SPAWN_E, N_SPAWN_ION = 48, 49, 50, 51
N_COLLISIONS_ALL, N_FLIGHTS_ALL = 52, 53     # every pass of the run
REASONS = ("exit0", "exit1", "cutoff", "cap_coll", "cap_time", "recomb", "cluster", "stalled")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library next to its source."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-pthread", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("length_m", C.c_double), ("n_zbins", C.c_int32), ("n_seg_m3", C.POINTER(C.c_double)),
        ("area_m2", C.c_double), ("activity_bq", C.c_double), ("e_cut_ev", C.c_double),
        ("max_collisions", C.c_uint32), ("max_lifetime_s", C.c_double),
        ("gas_temperature_k", C.c_double), ("n_tebins", C.c_int32), ("n_spec_bins", C.c_int32),
        ("spec_bin_ev", C.c_double), ("species_mass_ev", C.c_double * N_SPECIES),
        ("target_mass_ev", C.c_double), ("n_energy", C.c_int32), ("e_min_ev", C.c_double),
        ("e_max_ev", C.c_double), ("n_channels", C.c_int32), ("kind", C.POINTER(C.c_int32)),
        ("species_in", C.POINTER(C.c_int32)), ("species_out", C.POINTER(C.c_int32)),
        ("loss_ev", C.POINTER(C.c_double)), ("sigma_m2", C.POINTER(C.c_double)),
        ("ioniz_eps_ev", C.c_double), ("target", C.POINTER(C.c_int32)),
        ("gas_drift_mps", C.c_double), ("ang_set", C.POINTER(C.c_int32)),
        ("ang_n_sets", C.c_int32), ("ang_n_bins", C.c_int32), ("ang_n_mu", C.c_int32),
        ("ang_e_min_ev", C.POINTER(C.c_double)), ("ang_e_max_ev", C.POINTER(C.c_double)),
        ("ang_threshold_ev", C.POINTER(C.c_double)), ("ang_pdf", C.POINTER(C.c_double)),
    ]


class _Prims(C.Structure):
    _fields_ = [("n", C.c_int64), ("z_m", C.POINTER(C.c_double)), ("e_ev", C.POINTER(C.c_double)),
                ("mu", C.POINTER(C.c_double)), ("species", C.POINTER(C.c_uint8)),
                ("n_decays", C.c_int64), ("pid_offset", C.c_int64)]


class _Tallies(C.Structure):
    _fields_ = [("spectrum", C.POINTER(C.c_uint64)), ("time_fx", C.POINTER(C.c_uint64)),
                ("cross_pos", C.POINTER(C.c_uint64)), ("cross_neg", C.POINTER(C.c_uint64)),
                ("recomb", C.POINTER(C.c_uint64)), ("ledger", C.POINTER(C.c_int64)),
                ("chan_count", C.POINTER(C.c_uint64)), ("per_primary", C.POINTER(C.c_uint64)),
                ("density", C.POINTER(C.c_double)), ("current", C.POINTER(C.c_double)),
                ("field", C.POINTER(C.c_double))]


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        lib.orc_run.argtypes = [C.POINTER(_Problem), C.POINTER(_Prims), C.c_uint64, C.c_int,
                                C.c_int, C.c_int, C.POINTER(_Tallies)]
        lib.orc_run.restype = C.c_int
        lib.orc_run_pass.argtypes = [C.POINTER(_Problem), C.POINTER(_Prims), C.c_uint64, C.c_int,
                                     C.POINTER(C.c_uint64), C.c_int, C.c_int, C.POINTER(_Tallies)]
        lib.orc_run_pass.restype = C.c_int
        lib.orc_run_cycle.argtypes = [C.POINTER(_Problem), C.POINTER(_Prims), C.c_uint64,
                                      C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.c_double,
                                      C.c_int, C.c_int, C.POINTER(_Tallies)]
        lib.orc_run_cycle.restype = C.c_int
        lib.orc_philox4x64.argtypes = [C.POINTER(C.c_uint64)] * 3
        lib.orc_philox4x64.restype = None
        lib.orc_sigma.argtypes = [C.POINTER(_Problem), C.c_int, C.c_double]
        lib.orc_sigma.restype = C.c_double
        lib.orc_collide.argtypes = [C.POINTER(_Problem), C.c_int, C.c_int, C.c_double, C.c_double,
                                    C.POINTER(C.c_uint64), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double), C.POINTER(C.c_int)]
        lib.orc_collide.restype = C.c_int
        lib.orc_elastic_moving_target.argtypes = [
            C.POINTER(_Problem), C.c_double, C.c_double, C.c_double, C.POINTER(C.c_uint64),
            C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(C.c_double),
            C.POINTER(C.c_double), C.POINTER(C.c_double)]
        lib.orc_elastic_moving_target.restype = None
        lib.orc_charge_exchange.argtypes = [
            C.POINTER(_Problem), C.c_double, C.c_double, C.c_double, C.POINTER(C.c_uint64),
            C.POINTER(C.c_uint64), C.POINTER(C.c_double), C.POINTER(C.c_double),
            C.POINTER(C.c_double)]
        lib.orc_charge_exchange.restype = None
        lib.orc_ionization_moving_target.argtypes = [
            C.POINTER(_Problem), C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
            C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
            C.POINTER(C.c_double)]
        lib.orc_ionization_moving_target.restype = None
        lib.orc_sample_angle.argtypes = [C.POINTER(_Problem), C.c_int, C.c_double, C.c_double]
        lib.orc_sample_angle.restype = C.c_double
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


class _Marshal:
    """Keeps the numpy buffers behind a _Problem alive."""

    def __init__(self, prob):
        self.n_seg = np.ascontiguousarray(prob.n_seg_m3, np.float64)
        self.kind = np.array([c.kind for c in prob.channels], np.int32)
        self.sin = np.array([c.species_in for c in prob.channels], np.int32)
        self.sout = np.array([c.species_out for c in prob.channels], np.int32)
        self.loss = np.array([c.loss_ev for c in prob.channels], np.float64)
        self.target = np.array([getattr(c, "target", 0) for c in prob.channels], np.int32)
        self.sigma = (prob.sigma_matrix() if prob.channels
                      else np.zeros((0, prob.n_energy))).astype(np.float64)
        self.sigma = np.ascontiguousarray(self.sigma)
        s = _Problem()
        s.length_m = prob.length_m
        s.n_zbins = prob.n_zbins
        s.n_seg_m3 = _ptr(self.n_seg, C.c_double)
        s.area_m2 = prob.area_m2
        s.activity_bq = prob.activity_bq
        s.e_cut_ev = prob.e_cut_ev
        s.max_collisions = min(int(prob.max_collisions), 0xFFFFFFFF)
        s.max_lifetime_s = prob.max_lifetime_s
        s.gas_temperature_k = prob.gas_temperature_k
        s.n_tebins = prob.n_tebins
        s.n_spec_bins = prob.n_spec_bins
        s.spec_bin_ev = prob.spec_bin_ev
        for i in range(N_SPECIES):
            s.species_mass_ev[i] = float(prob.species_mass_ev[i])
        s.target_mass_ev = prob.target_mass_ev
        s.n_energy = prob.n_energy
        s.e_min_ev = prob.e_min_ev
        s.e_max_ev = prob.e_max_ev
        s.n_channels = prob.n_channels
        s.kind = _ptr(self.kind, C.c_int32)
        s.species_in = _ptr(self.sin, C.c_int32)
        s.species_out = _ptr(self.sout, C.c_int32)
        s.loss_ev = _ptr(self.loss, C.c_double)
        s.sigma_m2 = _ptr(self.sigma, C.c_double)
        s.ioniz_eps_ev = prob.ioniz_eps_ev
        s.target = _ptr(self.target, C.c_int32)
        s.gas_drift_mps = float(getattr(prob, "gas_drift_mps", 0.0))
        self.ang = angular_sets(prob)
        if self.ang is not None:
            a = self.ang
            s.ang_set = _ptr(a["set"], C.c_int32)
            s.ang_n_sets, s.ang_n_bins, s.ang_n_mu = a["n_sets"], a["n_bins"], a["n_mu"]
            s.ang_e_min_ev = _ptr(a["e_min"], C.c_double)
            s.ang_e_max_ev = _ptr(a["e_max"], C.c_double)
            s.ang_threshold_ev = _ptr(a["threshold"], C.c_double)
            s.ang_pdf = _ptr(a["pdf"], C.c_double)
        self.s = s


def angular_sets(prob):
    """The problem's angle tables as flat arrays (None when every elastic
    channel is isotropic).  All sets must share their bin and point counts."""
    tabs = [getattr(c, "angular", None) for c in prob.channels]
    used = [t for t in tabs if t is not None]
    if not used:
        return None
    nb, nm = used[0].pdf.shape
    order = {}
    for t in used:
        if t.pdf.shape != (nb, nm):
            raise ValueError("angle tables must share their bins and points")
        order.setdefault(id(t), len(order))
    sets = sorted({id(t): t for t in used}.items(), key=lambda kv: order[kv[0]])
    return {
        "set": np.array([order[id(t)] if t is not None else -1 for t in tabs], np.int32),
        "n_sets": len(sets), "n_bins": nb, "n_mu": nm,
        "e_min": np.array([t.e_min_ev for _, t in sets], np.float64),
        "e_max": np.array([t.e_max_ev for _, t in sets], np.float64),
        "threshold": np.array([t.threshold_ev for _, t in sets], np.float64),
        "pdf": np.ascontiguousarray(np.stack([t.pdf for _, t in sets]), np.float64),
    }


def sample_angle(prob, channel: int, e_ev: float, u: float) -> float:
    lib = _load()
    m = _Marshal(prob)
    return float(lib.orc_sample_angle(C.byref(m.s), channel, e_ev, u))


def _prims(pr, pid_offset: int = 0, n_decays: Optional[int] = None):
    z = np.ascontiguousarray(pr.z_m, np.float64)
    e = np.ascontiguousarray(pr.e_ev, np.float64)
    mu = np.ascontiguousarray(pr.mu, np.float64)
    sp = np.ascontiguousarray(pr.species, np.uint8)
    s = _Prims(pr.n, _ptr(z, C.c_double), _ptr(e, C.c_double), _ptr(mu, C.c_double),
               _ptr(sp, C.c_uint8), int(pr.n_decays if n_decays is None else n_decays),
               int(pid_offset))
    return s, (z, e, mu, sp)


def empty_tallies(prob, n_primaries: int) -> Dict[str, np.ndarray]:
    nz, ntb = prob.n_zbins, prob.n_tebins
    return {
        "spectrum": np.zeros((2, N_SPECIES, prob.n_spec_bins + 1), np.uint64),
        "time_fx": np.zeros((N_SPECIES, nz + 2, ntb), np.uint64),
        "cross_pos": np.zeros((N_SPECIES, nz + 1), np.uint64),
        "cross_neg": np.zeros((N_SPECIES, nz + 1), np.uint64),
        "recomb": np.zeros((N_SPECIES, nz), np.uint64),
        "ledger": np.zeros(LEDGER_LEN, np.int64),
        "chan_count": np.zeros(max(prob.n_channels, 1), np.uint64),
        "per_primary": np.zeros(max(n_primaries, 1), np.uint64),
        "density": np.zeros((N_SPECIES, nz), np.float64),
        "current": np.zeros((N_SPECIES, nz + 1), np.float64),
        "field": np.zeros((N_SPECIES, nz, ntb), np.float64),
    }


def _tallies_struct(t: Dict[str, np.ndarray], with_norm: bool = True) -> _Tallies:
    s = _Tallies()
    s.spectrum = _ptr(t["spectrum"], C.c_uint64)
    s.time_fx = _ptr(t["time_fx"], C.c_uint64)
    s.cross_pos = _ptr(t["cross_pos"], C.c_uint64)
    s.cross_neg = _ptr(t["cross_neg"], C.c_uint64)
    s.recomb = _ptr(t["recomb"], C.c_uint64)
    s.ledger = _ptr(t["ledger"], C.c_int64)
    s.chan_count = _ptr(t["chan_count"], C.c_uint64)
    s.per_primary = _ptr(t["per_primary"], C.c_uint64)
    if with_norm:
        s.density = _ptr(t["density"], C.c_double)
        s.current = _ptr(t["current"], C.c_double)
        s.field = _ptr(t["field"], C.c_double)
    return s


def run(prob, prims, seed: int = 1, n_passes: Optional[int] = None, mode: int = 0,
        n_threads: int = 1) -> Dict[str, np.ndarray]:
    """Whole run (one or two passes).  mode 0: optical-depth flights;
    mode 1: paper-literal segment stop and redraw."""
    lib = _load()
    m = _Marshal(prob)
    ps, keep = _prims(prims)
    t = empty_tallies(prob, prims.n)
    ts = _tallies_struct(t)
    npass = prob.n_passes if n_passes is None else n_passes
    rc = lib.orc_run(C.byref(m.s), C.byref(ps), C.c_uint64(seed), npass, mode, n_threads,
                     C.byref(ts))
    if rc != 0:
        raise RuntimeError(f"oracle run failed: {rc}")
    t["per_primary"] = t["per_primary"][:prims.n]
    t["chan_count"] = t["chan_count"][:prob.n_channels]
    return t


def run_pass(prob, prims, seed: int, pass_index: int, field_time_in: Optional[np.ndarray] = None,
             pid_offset: int = 0, n_decays: Optional[int] = None, mode: int = 0,
             n_threads: int = 1) -> Dict[str, np.ndarray]:
    """One pass over a primary-id range, raw tallies only (for sharding)."""
    lib = _load()
    m = _Marshal(prob)
    ps, keep = _prims(prims, pid_offset, n_decays)
    t = empty_tallies(prob, prims.n)
    ts = _tallies_struct(t, with_norm=False)
    fin = None
    if field_time_in is not None:
        fin = np.ascontiguousarray(field_time_in, np.uint64)
    rc = lib.orc_run_pass(C.byref(m.s), C.byref(ps), C.c_uint64(seed), pass_index,
                          _ptr(fin, C.c_uint64) if fin is not None else None, mode, n_threads,
                          C.byref(ts))
    if rc != 0:
        raise RuntimeError(f"oracle pass failed: {rc}")
    t["per_primary"] = t["per_primary"][:prims.n]
    t["chan_count"] = t["chan_count"][:prob.n_channels]
    return t


def run_cycle(prob, prims, seed: int, field_time_in: Optional[np.ndarray],
              field_recomb_in: Optional[np.ndarray], field_decays: float, pid_offset: int = 0,
              mode: int = 0, n_threads: int = 1) -> Dict[str, np.ndarray]:
    """One cycle of the continuous field update over a primary-id range:
    recombination on, fields from the given summed tallies (None: zero)."""
    lib = _load()
    m = _Marshal(prob)
    ps, keep = _prims(prims, pid_offset, prims.n_decays)
    t = empty_tallies(prob, prims.n)
    ts = _tallies_struct(t, with_norm=False)
    fin = None if field_time_in is None else np.ascontiguousarray(field_time_in, np.uint64)
    rin = None if field_recomb_in is None else np.ascontiguousarray(field_recomb_in, np.uint64)
    rc = lib.orc_run_cycle(C.byref(m.s), C.byref(ps), C.c_uint64(seed),
                           _ptr(fin, C.c_uint64) if fin is not None else None,
                           _ptr(rin, C.c_uint64) if rin is not None else None,
                           float(field_decays), mode, n_threads, C.byref(ts))
    if rc != 0:
        raise RuntimeError(f"oracle cycle failed: {rc}")
    t["per_primary"] = t["per_primary"][:prims.n]
    t["chan_count"] = t["chan_count"][:prob.n_channels]
    return t


RAW_KEYS = ("spectrum", "time_fx", "cross_pos", "cross_neg", "recomb", "ledger", "chan_count")


def run_cycles(prob, prims, seed: int, n_cycles: int, mode: int = 0,
               n_threads: int = 1) -> Dict[str, np.ndarray]:
    """The paper's continuous field update (Sec. 3.6): the primaries in
    n_cycles consecutive cycles of indices [c n / C, (c+1) n / C); cycle c runs
    with the fields of the time and deletion tallies of the cycles before it,
    t_sim from their share of the decays; the first with fields of zero.
    Returns the raw tallies summed over the cycles, the density and current
    of Eq. target_field_density and Sec. 2.3 over the whole run, and as
    `field` the per-bin densities a next cycle would use."""
    n = prims.n
    tot = empty_tallies(prob, n)
    for k in RAW_KEYS:
        tot[k] = tot[k].astype(np.int64 if k == "ledger" else np.uint64)
    tot["chan_count"] = tot["chan_count"][:prob.n_channels]
    tot["per_primary"] = tot["per_primary"][:n]
    for c in range(n_cycles):
        lo, hi = c * n // n_cycles, (c + 1) * n // n_cycles
        if hi <= lo:
            continue
        decays_before = prims.n_decays * lo / n
        if lo == 0:
            t = run_cycle(prob, prims.slice(lo, hi - lo), seed, None, None, 0.0, pid_offset=lo,
                          mode=mode, n_threads=n_threads)
        else:
            t = run_cycle(prob, prims.slice(lo, hi - lo), seed, tot["time_fx"], tot["recomb"],
                          decays_before, pid_offset=lo, mode=mode, n_threads=n_threads)
        for k in RAW_KEYS:
            tot[k] += t[k]
        tot["per_primary"][lo:hi] = t["per_primary"]
    # normalisation over the whole run: Eq. target_field_density, Sec. 2.3
    nz, ntb = prob.n_zbins, prob.n_tebins
    tsim = prims.n_decays / prob.activity_bq
    vol = prob.length_m / nz * prob.area_m2
    tt = tot["time_fx"][:, 1:nz + 1, :].astype(np.float64)           # [4][nz][ntb]
    rec = tot["recomb"].astype(np.float64)                           # [4][nz]
    tot["density"] = tt.sum(axis=2) / 2**50 / (tsim * vol) - rec / vol
    tot["current"] = (tot["cross_pos"].astype(np.float64) -
                      tot["cross_neg"].astype(np.float64)) / (prob.area_m2 * tsim)
    ttot = tt.sum(axis=2, keepdims=True)
    share = np.divide(tt, ttot, out=np.zeros_like(tt), where=ttot > 0)
    tot["field"] = np.maximum(tt / 2**50 / (tsim * vol) - (rec / vol)[:, :, None] * share, 0.0)
    return tot


def philox4x64(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.array(ctr, np.uint64)
    k = np.array(key, np.uint64)
    o = np.zeros(4, np.uint64)
    lib.orc_philox4x64(_ptr(c, C.c_uint64), _ptr(k, C.c_uint64), _ptr(o, C.c_uint64))
    return o


def sigma(prob, channel: int, e_ev: float) -> float:
    lib = _load()
    m = _Marshal(prob)
    return float(lib.orc_sigma(C.byref(m.s), channel, e_ev))


def collide(prob, channel: int, species: int, e_ev: float, mu: float, words):
    """Single collision with given raw Philox words; returns [(E, mu, species)]."""
    lib = _load()
    m = _Marshal(prob)
    w = np.array(words, np.uint64)
    oe = np.zeros(2)
    om = np.zeros(2)
    osp = np.zeros(2, np.int32)
    n = lib.orc_collide(C.byref(m.s), channel, species, e_ev, mu, _ptr(w, C.c_uint64),
                        _ptr(oe, C.c_double), _ptr(om, C.c_double), _ptr(osp, C.c_int))
    return [(float(oe[i]), float(om[i]), int(osp[i])) for i in range(n)]


def elastic_moving_target(prob, m1_ev: float, e_ev: float, mu: float, words, ctr, key):
    """One elastic collision with a moving target: event block `words`, target
    blocks from counter (ctr[0], ctr[1], ctr[2], k) and key; returns
    (E', mu', velocities[12])."""
    lib = _load()
    m = _Marshal(prob)
    w = np.array(words, np.uint64)
    c = np.array(ctr, np.uint64)
    k = np.array(key, np.uint64)
    oe = np.zeros(1)
    om = np.zeros(1)
    v = np.zeros(12)
    lib.orc_elastic_moving_target(C.byref(m.s), m1_ev, e_ev, mu, _ptr(w, C.c_uint64),
                                  _ptr(c, C.c_uint64), _ptr(k, C.c_uint64),
                                  _ptr(oe, C.c_double), _ptr(om, C.c_double),
                                  _ptr(v, C.c_double))
    return float(oe[0]), float(om[0]), v


def charge_exchange(prob, m1_ev: float, e_ev: float, mu: float, ctr, key):
    """One charge exchange: target blocks from counter (ctr[0], ctr[1], ctr[2],
    k) and key; returns (E', mu', target velocity[3] in units of c)."""
    lib = _load()
    m = _Marshal(prob)
    c = np.array(ctr, np.uint64)
    k = np.array(key, np.uint64)
    oe = np.zeros(1)
    om = np.zeros(1)
    v = np.zeros(3)
    lib.orc_charge_exchange(C.byref(m.s), m1_ev, e_ev, mu, _ptr(c, C.c_uint64),
                            _ptr(k, C.c_uint64), _ptr(oe, C.c_double), _ptr(om, C.c_double),
                            _ptr(v, C.c_double))
    return float(oe[0]), float(om[0]), v


def ionization_moving_target(prob, channel: int, m1_ev: float, e_ev: float, mu: float,
                             m_ion_ev: float, words, ctr, key, marshal=None) -> dict:
    """One ionization with a moving target: event block `words` (w[2] shares
    the energy, w[3] the azimuth), target blocks from counter (ctr[0], ctr[1],
    ctr[2], k) and key.  Returns the impactor's, ejected electron's and ion's
    energies and pitch cosines and the impact energy E_i.  Pass the result of
    marshal_problem(prob) as `marshal` to skip re-marshalling in loops."""
    lib = _load()
    m = marshal if marshal is not None else _Marshal(prob)
    w = np.array(words, np.uint64)
    c = np.array(ctr, np.uint64)
    k = np.array(key, np.uint64)
    out = np.zeros(7)
    lib.orc_ionization_moving_target(C.byref(m.s), channel, m1_ev, e_ev, mu, m_ion_ev,
                                     _ptr(w, C.c_uint64), _ptr(c, C.c_uint64),
                                     _ptr(k, C.c_uint64), _ptr(out, C.c_double))
    return {"e1": out[0], "mu1": out[1], "e2": out[2], "mu2": out[3], "eion": out[4],
            "muion": out[5], "ei": out[6]}


def marshal_problem(prob):
    """The oracle's C view of a problem, reusable across single-collision calls."""
    return _Marshal(prob)


# ---- orbit mode: the Boris mover in a tube (mirrors karl_oracle.h) ----
OB_BIRTHS, OB_DEATHS = 0, 4
OB_N_COLLISIONS, OB_N_FLIGHTS, OB_N_STEPS, OB_N_SPAWN_E, OB_N_SPAWN_ION = 36, 37, 38, 39, 40
OB_LEDGER_LEN = 48
ORBIT_REASONS = ("exit0", "exit1", "wall", "cutoff", "cap_coll", "cap_time", "cluster", "stalled")
OE_IN_PRIMARY, OE_IN_THERMAL, OE_EXIT0, OE_EXIT1, OE_WALL, OE_CUTOFF, OE_CAP, OE_CLUSTER, \
    OE_LOSS_IONIZ, OE_LOSS_EXCIT, OE_RECOIL, OE_STALLED, OE_FIELD_WORK = range(13)
OE_LEN = 16


class _Orbit(C.Structure):
    _fields_ = [("b_t", C.c_double), ("tube_radius_m", C.c_double), ("n_rbins", C.c_int32),
                ("e_z_vm", C.POINTER(C.c_double)), ("e_r_vm2", C.c_double),
                ("dt_s", C.c_double * N_SPECIES), ("max_steps", C.c_uint64)]


class _OrbitPrims(C.Structure):
    _fields_ = [("n", C.c_int64), ("x_m", C.POINTER(C.c_double)), ("y_m", C.POINTER(C.c_double)),
                ("z_m", C.POINTER(C.c_double)), ("e_ev", C.POINTER(C.c_double)),
                ("mu", C.POINTER(C.c_double)), ("phi", C.POINTER(C.c_double)),
                ("species", C.POINTER(C.c_uint8)), ("pid_offset", C.c_int64)]


class _OrbitTallies(C.Structure):
    _fields_ = [(k, C.POINTER(C.c_uint64)) for k in
                ("spectrum", "time_z", "time_r", "cross_pos", "cross_neg", "rcross_out",
                 "rcross_in", "wall")] + [
        ("ledger", C.POINTER(C.c_int64)), ("energy", C.POINTER(C.c_double)),
        ("chan_count", C.POINTER(C.c_uint64)), ("per_primary", C.POINTER(C.c_uint64)),
        ("end_state", C.POINTER(C.c_double))]


def empty_orbit_tallies(prob, orbit, n_primaries: int) -> Dict[str, np.ndarray]:
    nz, nr = prob.n_zbins, orbit.n_rbins
    return {
        "spectrum": np.zeros((2, N_SPECIES, prob.n_spec_bins + 1), np.uint64),
        "time_z": np.zeros((N_SPECIES, nz), np.uint64),
        "time_r": np.zeros((N_SPECIES, nr), np.uint64),
        "cross_pos": np.zeros((N_SPECIES, nz + 1), np.uint64),
        "cross_neg": np.zeros((N_SPECIES, nz + 1), np.uint64),
        "rcross_out": np.zeros((N_SPECIES, nr + 1), np.uint64),
        "rcross_in": np.zeros((N_SPECIES, nr + 1), np.uint64),
        "wall": np.zeros((N_SPECIES, nz), np.uint64),
        "ledger": np.zeros(OB_LEDGER_LEN, np.int64),
        "energy": np.zeros(OE_LEN, np.float64),
        "chan_count": np.zeros(max(prob.n_channels, 1), np.uint64),
        "per_primary": np.zeros(max(n_primaries, 1), np.uint64),
        "end_state": np.zeros((max(n_primaries, 1), 8), np.float64),
    }


def orbit_run(prob, orbit, prims, seed: int = 1, n_threads: int = 1) -> Dict[str, np.ndarray]:
    """Full-orbit run (Boris mover, Sec. 3.1) of `prims` (an
    ``inputs.OrbitPrimaries``) in the tube described by `orbit` (an
    ``inputs.Orbit``)."""
    lib = _load()
    if not hasattr(lib, "_orbit_ready"):
        lib.orc_orbit_run.argtypes = [C.POINTER(_Problem), C.POINTER(_Orbit),
                                      C.POINTER(_OrbitPrims), C.c_uint64, C.c_int,
                                      C.POINTER(_OrbitTallies)]
        lib.orc_orbit_run.restype = C.c_int
        lib._orbit_ready = True
    m = _Marshal(prob)
    ez = None if orbit.e_z_vm is None else np.ascontiguousarray(orbit.e_z_vm, np.float64)
    o = _Orbit()
    o.b_t, o.tube_radius_m, o.n_rbins = orbit.b_t, orbit.tube_radius_m, orbit.n_rbins
    o.e_z_vm = _ptr(ez, C.c_double) if ez is not None else None
    o.e_r_vm2 = orbit.e_r_vm2
    for i in range(N_SPECIES):
        o.dt_s[i] = float(orbit.dt_s[i])
    o.max_steps = int(orbit.max_steps)
    arrs = [np.ascontiguousarray(getattr(prims, k), np.float64)
            for k in ("x_m", "y_m", "z_m", "e_ev", "mu", "phi")]
    sp = np.ascontiguousarray(prims.species, np.uint8)
    ps = _OrbitPrims(prims.n, *[_ptr(a, C.c_double) for a in arrs], _ptr(sp, C.c_uint8),
                     int(prims.pid_offset))
    t = empty_orbit_tallies(prob, orbit, prims.n)
    ts = _OrbitTallies()
    for k in ("spectrum", "time_z", "time_r", "cross_pos", "cross_neg", "rcross_out",
              "rcross_in", "wall", "chan_count", "per_primary"):
        setattr(ts, k, _ptr(t[k], C.c_uint64))
    ts.ledger = _ptr(t["ledger"], C.c_int64)
    ts.energy = _ptr(t["energy"], C.c_double)
    ts.end_state = _ptr(t["end_state"], C.c_double)
    rc = lib.orc_orbit_run(C.byref(m.s), C.byref(o), C.byref(ps), C.c_uint64(seed), n_threads,
                           C.byref(ts))
    if rc != 0:
        raise RuntimeError(f"oracle orbit run failed: {rc}")
    t["per_primary"] = t["per_primary"][:prims.n]
    t["end_state"] = t["end_state"][:prims.n]
    t["chan_count"] = t["chan_count"][:prob.n_channels]
    return t
