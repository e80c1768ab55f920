"""Thin ctypes binding of ``libkarl.so`` (C ABI in ``include/karl.h``).

Argument marshalling only: every step of the transport runs in the CUDA
library.  The module raises on import of the library if ``libkarl.so`` has
not been built (``paper_2503_10263_gb300.build.build()``); there is no CPU
fallback.

Module-level functions carry the C names (``karl_create``, ``karl_run``,
``karl_run_pass``, ``karl_destroy``, ...).  ``Context`` wraps them for
problems from ``paper_2503_10263_gb300.inputs``; tallies come back as numpy
arrays (host buffers) or are written to caller-provided device pointers.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkarl.so")

N_SPECIES = 4
N_REASONS = 8
LEDGER_LEN = 64
MAX_CHANNELS = 16
STATIC_SCRATCH_BYTES = 64 << 20     # KARL_STATIC_SCRATCH_BYTES of karl_run_pass_static
FP64, FP32 = 0, 1

# status codes
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EOVERFLOW, ECAPACITY, ECANCELLED, EBUSY, ENOTFOUND = range(10)

# ledger slots
E_IN_PRIMARY, E_IN_THERMAL, E_EXIT0, E_EXIT1, E_CUTOFF, E_CAP, E_RECOMB, E_CLUSTER, \
    E_LOSS_IONIZ, E_LOSS_EXCIT, E_LOSS_RECOIL, E_STALLED = range(12)
BIRTHS, DEATHS = 12, 16
N_COLLISIONS, N_FLIGHTS, N_SPAWN_E, N_SPAWN_ION = 48, 49, 50, 51
N_COLLISIONS_ALL, N_FLIGHTS_ALL = 52, 53     # every pass of the run
# full-orbit runs: integer ledger and energy ledger slots
OB_BIRTHS, OB_DEATHS = 0, 4
OB_N_COLLISIONS, OB_N_FLIGHTS, OB_N_STEPS, OB_N_SPAWN_E, OB_N_SPAWN_ION = 36, 37, 38, 39, 40
ORBIT_LEDGER_LEN, ORBIT_ENERGY_LEN = 48, 16
ORBIT_REASONS = ("exit0", "exit1", "wall", "cutoff", "cap_coll", "cap_time", "cluster", "stalled")
OE_IN_PRIMARY, OE_IN_THERMAL, OE_EXIT0, OE_EXIT1, OE_WALL, OE_CUTOFF, OE_CAP, OE_CLUSTER, \
    OE_LOSS_IONIZ, OE_LOSS_EXCIT, OE_RECOIL, OE_STALLED, OE_FIELD_WORK = range(13)


class KarlError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"karl status {status} ({msg})")
        self.status = status


class Geometry(C.Structure):
    _fields_ = [("length_m", C.c_double), ("n_zbins", C.c_int32),
                ("n_seg_m3", C.POINTER(C.c_double)), ("area_m2", C.c_double),
                ("activity_bq", C.c_double), ("e_cut_ev", C.c_double),
                ("max_collisions", C.c_uint32), ("max_lifetime_s", C.c_double),
                ("gas_temperature_k", C.c_double), ("n_tebins", C.c_int32),
                ("n_spec_bins", C.c_int32), ("spec_bin_ev", C.c_double),
                ("species_mass_ev", C.c_double * N_SPECIES), ("target_mass_ev", C.c_double),
                ("gas_drift_mps", C.c_double)]


class Angular(C.Structure):
    _fields_ = [("n_sets", C.c_int32), ("n_bins", C.c_int32), ("n_mu", C.c_int32),
                ("set", C.POINTER(C.c_int32)), ("e_min_ev", C.POINTER(C.c_double)),
                ("e_max_ev", C.POINTER(C.c_double)), ("threshold_ev", C.POINTER(C.c_double)),
                ("pdf", C.POINTER(C.c_double))]


class XS(C.Structure):
    _fields_ = [("n_energy", C.c_int32), ("e_min_ev", C.c_double), ("e_max_ev", C.c_double),
                ("n_channels", C.c_int32), ("kind", C.POINTER(C.c_int32)),
                ("species_in", C.POINTER(C.c_int32)), ("species_out", C.POINTER(C.c_int32)),
                ("loss_ev", C.POINTER(C.c_double)), ("sigma_m2", C.POINTER(C.c_double)),
                ("ioniz_eps_ev", C.c_double), ("target", C.POINTER(C.c_int32)),
                ("angular", C.POINTER(Angular))]


class Primaries(C.Structure):
    _fields_ = [("n", C.c_int64), ("z_m", C.c_void_p), ("e_ev", C.c_void_p), ("mu", C.c_void_p),
                ("species", C.c_void_p), ("n_decays", C.c_int64), ("pid_offset", C.c_int64),
                ("on_device", C.c_int32)]


class Tallies(C.Structure):
    _fields_ = [("spectrum", C.c_void_p), ("time_fx", C.c_void_p), ("cross_pos", C.c_void_p),
                ("cross_neg", C.c_void_p), ("recomb", C.c_void_p), ("ledger", C.c_void_p),
                ("chan_count", C.c_void_p), ("per_primary", C.c_void_p), ("density", C.c_void_p),
                ("current", C.c_void_p), ("field", C.c_void_p), ("on_device", C.c_int32)]


class RunOpts(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("n_passes", C.c_int32), ("precision", C.c_int32),
                ("block_size", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("timeout_s", C.c_double), ("stream", C.c_void_p)]


class Orbit(C.Structure):
    _fields_ = [("b_t", C.c_double), ("tube_radius_m", C.c_double), ("n_rbins", C.c_int32),
                ("pad", C.c_int32), ("e_z_vm", C.c_void_p), ("e_r_vm2", C.c_double),
                ("dt_s", C.c_double * N_SPECIES), ("max_steps", C.c_uint64)]


class OrbitPrimaries(C.Structure):
    _fields_ = [("n", C.c_int64)] + [(k, C.c_void_p) for k in
                                     ("x_m", "y_m", "z_m", "e_ev", "mu", "phi", "species")] + [
        ("pid_offset", C.c_int64)]


ORBIT_TALLY_KEYS = ("spectrum", "time_z", "time_r", "cross_pos", "cross_neg", "rcross_out",
                    "rcross_in", "wall", "ledger", "energy", "chan_count", "per_primary",
                    "end_state")


class OrbitTallies(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ORBIT_TALLY_KEYS]


class Layout(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("spectrum", "time_fx", "cross", "recomb", "ledger",
                                           "chan_count", "density", "current", "field")]


class RunStats(C.Structure):
    _fields_ = [("kernel_ms", C.c_double * 2), ("collisions", C.c_int64 * 2),
                ("flights", C.c_int64 * 2), ("particles", C.c_int64 * 2),
                ("lane_occupancy", C.c_double * 2),
                ("grid_blocks", C.c_int32), ("block_size", C.c_int32),
                ("queue_capacity", C.c_int32), ("kernel_launches", C.c_int64),
                ("tail_ms", C.c_double * 2), ("spilled", C.c_int64 * 2),
                ("idle_warp_frac", C.c_double * 2)]


_lib = None


def load() -> C.CDLL:
    """Load libkarl.so; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "paper_2503_10263_gb300.build.build() (there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    P = C.POINTER
    lib.karl_create.argtypes = [P(Geometry), P(XS), P(C.c_void_p)]
    lib.karl_run.argtypes = [C.c_void_p, P(Primaries), P(RunOpts), P(Tallies)]
    lib.karl_run_pass.argtypes = [C.c_void_p, P(Primaries), P(RunOpts), C.c_int32,
                                  C.c_void_p, P(Tallies)]
    lib.karl_run_pass_static.argtypes = [C.c_void_p, P(Primaries), P(RunOpts), C.c_int32,
                                         C.c_void_p, P(Tallies)]
    lib.karl_run_cycles.argtypes = [C.c_void_p, P(Primaries), P(RunOpts), C.c_int32, P(Tallies)]
    lib.karl_run_cycle.argtypes = [C.c_void_p, P(Primaries), P(RunOpts), C.c_void_p, C.c_void_p,
                                   C.c_double, P(Tallies)]
    lib.karl_run_orbit.argtypes = [C.c_void_p, P(Orbit), P(OrbitPrimaries), P(RunOpts),
                                   P(OrbitTallies)]
    lib.karl_destroy.argtypes = [C.c_void_p]
    lib.karl_destroy.restype = None
    lib.karl_cancel.argtypes = [C.c_void_p]
    lib.karl_cancel.restype = None
    lib.karl_status_string.argtypes = [C.c_int]
    lib.karl_status_string.restype = C.c_char_p
    lib.karl_last_error.argtypes = [C.c_void_p]
    lib.karl_last_error.restype = C.c_char_p
    lib.karl_tally_layout.argtypes = [C.c_void_p, P(Layout)]
    lib.karl_last_stats.argtypes = [C.c_void_p, P(RunStats)]
    for f in ("karl_create", "karl_run", "karl_run_pass", "karl_run_pass_static",
              "karl_run_cycles", "karl_run_cycle", "karl_tally_layout", "karl_last_stats",
              "karl_run_orbit"):
        getattr(lib, f).restype = C.c_int
    _lib = lib
    return lib


# ---- C-named wrappers -------------------------------------------------------

def karl_status_string(status: int) -> str:
    return load().karl_status_string(status).decode()


def karl_create(geom: Geometry, xs: XS) -> C.c_void_p:
    out = C.c_void_p()
    st = load().karl_create(C.byref(geom), C.byref(xs), C.byref(out))
    if st != OK:
        raise KarlError(st, karl_status_string(st))
    return out


def karl_run(ctx, prim: Primaries, opts: RunOpts, tallies: Tallies) -> int:
    return load().karl_run(ctx, C.byref(prim), C.byref(opts), C.byref(tallies))


def karl_run_pass(ctx, prim: Primaries, opts: RunOpts, pass_index: int, field_time_in,
                  tallies: Tallies) -> int:
    return load().karl_run_pass(ctx, C.byref(prim), C.byref(opts), pass_index, field_time_in,
                                C.byref(tallies))


def karl_run_pass_static(ctx, prim: Primaries, opts: RunOpts, pass_index: int, field_time_in,
                         tallies: Tallies) -> int:
    """karl_run_pass with scratch in the library's static device array: device
    buffers only, tallies overwritten, nothing allocated by the call."""
    return load().karl_run_pass_static(ctx, C.byref(prim), C.byref(opts), pass_index,
                                       field_time_in, C.byref(tallies))


def karl_run_cycles(ctx, prim: Primaries, opts: RunOpts, n_cycles: int, tallies: Tallies) -> int:
    return load().karl_run_cycles(ctx, C.byref(prim), C.byref(opts), n_cycles, C.byref(tallies))


def karl_run_cycle(ctx, prim: Primaries, opts: RunOpts, field_time_in, field_recomb_in,
                   field_decays: float, tallies: Tallies) -> int:
    return load().karl_run_cycle(ctx, C.byref(prim), C.byref(opts), field_time_in,
                                 field_recomb_in, field_decays, C.byref(tallies))


def karl_run_orbit(ctx, orbit: Orbit, prim: OrbitPrimaries, opts: RunOpts,
                   tallies: OrbitTallies) -> int:
    return load().karl_run_orbit(ctx, C.byref(orbit), C.byref(prim), C.byref(opts),
                                 C.byref(tallies))


def karl_destroy(ctx) -> None:
    load().karl_destroy(ctx)


def karl_cancel(ctx) -> None:
    load().karl_cancel(ctx)


def karl_last_error(ctx) -> str:
    return load().karl_last_error(ctx).decode()


def karl_tally_layout(ctx) -> Layout:
    lay = Layout()
    st = load().karl_tally_layout(ctx, C.byref(lay))
    if st != OK:
        raise KarlError(st, karl_status_string(st))
    return lay


def karl_last_stats(ctx) -> RunStats:
    s = RunStats()
    load().karl_last_stats(ctx, C.byref(s))
    return s


# ---- problem marshalling ----------------------------------------------------

def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


class Context:
    """One problem's device context (tables on the GPU) and its runs."""

    def __init__(self, prob):
        self.prob = prob
        self._keep = []
        g = _geometry(prob, self._keep)
        x = _xs(prob, self._keep)
        self.ctx = karl_create(g, x)
        self.layout = karl_tally_layout(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            karl_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != OK:
            raise KarlError(st, f"{karl_status_string(st)}: {karl_last_error(self.ctx)}")

    def empty_tallies(self, n_primaries: int) -> Dict[str, np.ndarray]:
        p = self.prob
        nz, ntb = p.n_zbins, p.n_tebins
        return {
            "spectrum": np.zeros((2, N_SPECIES, p.n_spec_bins + 1), np.uint64),
            "time_fx": np.zeros((N_SPECIES, nz + 2, ntb), np.uint64),
            "cross_pos": np.zeros((N_SPECIES, nz + 1), np.uint64),
            "cross_neg": np.zeros((N_SPECIES, nz + 1), np.uint64),
            "recomb": np.zeros((N_SPECIES, nz), np.uint64),
            "ledger": np.zeros(LEDGER_LEN, np.int64),
            "chan_count": np.zeros(max(p.n_channels, 1), np.uint64),
            "per_primary": np.zeros(max(n_primaries, 1), np.uint64),
            "density": np.zeros((N_SPECIES, nz), np.float64),
            "current": np.zeros((N_SPECIES, nz + 1), np.float64),
            "field": np.zeros((N_SPECIES, nz, ntb), np.float64),
        }

    @staticmethod
    def host_primaries(prims, pid_offset: int = 0, n_decays: Optional[int] = None):
        z = np.ascontiguousarray(prims.z_m, np.float64)
        e = np.ascontiguousarray(prims.e_ev, np.float64)
        mu = np.ascontiguousarray(prims.mu, np.float64)
        sp = np.ascontiguousarray(prims.species, np.uint8)
        s = Primaries(prims.n, z.ctypes.data, e.ctypes.data, mu.ctypes.data, sp.ctypes.data,
                      int(prims.n_decays if n_decays is None else n_decays), int(pid_offset), 0)
        return s, (z, e, mu, sp)

    @staticmethod
    def host_tallies(t: Dict[str, np.ndarray], per_primary: bool = True,
                     with_norm: bool = True) -> Tallies:
        s = Tallies()
        for k in ("spectrum", "time_fx", "cross_pos", "cross_neg", "recomb", "ledger",
                  "chan_count"):
            setattr(s, k, t[k].ctypes.data)
        s.per_primary = t["per_primary"].ctypes.data if per_primary else None
        if with_norm:
            s.density = t["density"].ctypes.data
            s.current = t["current"].ctypes.data
            s.field = t["field"].ctypes.data
        s.on_device = 0
        return s

    def opts(self, seed: int, n_passes: Optional[int] = None, precision: int = FP64,
             block_size: int = 0, blocks_per_sm: int = 0, timeout_s: float = 120.0,
             stream: Optional[int] = None) -> RunOpts:
        npass = self.prob.n_passes if n_passes is None else n_passes
        return RunOpts(seed, npass, precision, block_size, blocks_per_sm, timeout_s, stream)

    def run(self, prims, seed: int = 1, n_passes: Optional[int] = None, precision: int = FP64,
            per_primary: bool = True, **kw) -> Dict[str, np.ndarray]:
        """Whole run with host buffers in and out (karl_run)."""
        ps, keep = self.host_primaries(prims)
        t = self.empty_tallies(prims.n)
        ts = self.host_tallies(t, per_primary)
        o = self.opts(seed, n_passes, precision, **kw)
        self._check(karl_run(self.ctx, ps, o, ts))
        t["per_primary"] = t["per_primary"][:prims.n]
        t["chan_count"] = t["chan_count"][:self.prob.n_channels]
        return t

    def run_pass(self, prims, seed: int, pass_index: int, field_time_in=None,
                 pid_offset: int = 0, n_decays: Optional[int] = None, precision: int = FP64,
                 **kw) -> Dict[str, np.ndarray]:
        """One pass over a primary-id range, raw tallies (karl_run_pass)."""
        ps, keep = self.host_primaries(prims, pid_offset, n_decays)
        t = self.empty_tallies(prims.n)
        ts = self.host_tallies(t, True, with_norm=False)
        o = self.opts(seed, pass_index, precision, **kw)
        fin = None
        if field_time_in is not None:
            fin = np.ascontiguousarray(field_time_in, np.uint64)
        self._check(karl_run_pass(self.ctx, ps, o, pass_index,
                                  fin.ctypes.data if fin is not None else None, ts))
        t["per_primary"] = t["per_primary"][:prims.n]
        t["chan_count"] = t["chan_count"][:self.prob.n_channels]
        return t

    def empty_orbit_tallies(self, orbit, n_primaries: int) -> Dict[str, np.ndarray]:
        p = self.prob
        nz, nr = p.n_zbins, orbit.n_rbins
        return {
            "spectrum": np.zeros((2, N_SPECIES, p.n_spec_bins + 1), np.uint64),
            "time_z": np.zeros((N_SPECIES, nz), np.uint64),
            "time_r": np.zeros((N_SPECIES, nr), np.uint64),
            "cross_pos": np.zeros((N_SPECIES, nz + 1), np.uint64),
            "cross_neg": np.zeros((N_SPECIES, nz + 1), np.uint64),
            "rcross_out": np.zeros((N_SPECIES, nr + 1), np.uint64),
            "rcross_in": np.zeros((N_SPECIES, nr + 1), np.uint64),
            "wall": np.zeros((N_SPECIES, nz), np.uint64),
            "ledger": np.zeros(ORBIT_LEDGER_LEN, np.int64),
            "energy": np.zeros(ORBIT_ENERGY_LEN, np.float64),
            "chan_count": np.zeros(max(p.n_channels, 1), np.uint64),
            "per_primary": np.zeros(max(n_primaries, 1), np.uint64),
            "end_state": np.zeros((max(n_primaries, 1), 8), np.float64),
        }

    def run_orbit(self, orbit, prims, seed: int = 1, per_primary: bool = True,
                  end_state: bool = True, precision: int = FP64, **kw) -> Dict[str, np.ndarray]:
        """Full-orbit run (karl_run_orbit) of ``inputs.OrbitPrimaries`` in the
        tube and fields of ``inputs.Orbit``; host buffers in and out."""
        keep = []
        ez = None
        if orbit.e_z_vm is not None:
            ez = np.ascontiguousarray(orbit.e_z_vm, np.float64)
            keep.append(ez)
        ob = Orbit(orbit.b_t, orbit.tube_radius_m, orbit.n_rbins, 0,
                   ez.ctypes.data if ez is not None else None, orbit.e_r_vm2,
                   (C.c_double * N_SPECIES)(*[float(x) for x in orbit.dt_s]),
                   int(orbit.max_steps))
        arrs = [np.ascontiguousarray(getattr(prims, k), np.float64)
                for k in ("x_m", "y_m", "z_m", "e_ev", "mu", "phi")]
        sp = np.ascontiguousarray(prims.species, np.uint8)
        keep += arrs + [sp]
        ps = OrbitPrimaries(prims.n, *[a.ctypes.data for a in arrs], sp.ctypes.data,
                            int(prims.pid_offset))
        t = self.empty_orbit_tallies(orbit, prims.n)
        ts = OrbitTallies(*[t[k].ctypes.data for k in ORBIT_TALLY_KEYS])
        if not per_primary:
            ts.per_primary = None
        if not end_state:
            ts.end_state = None
        o = self.opts(seed, 1, precision, **kw)
        self._check(karl_run_orbit(self.ctx, ob, ps, o, ts))
        t["per_primary"] = t["per_primary"][:prims.n]
        t["end_state"] = t["end_state"][:prims.n]
        t["chan_count"] = t["chan_count"][:self.prob.n_channels]
        return t

    def run_cycles(self, prims, seed: int, n_cycles: int, precision: int = FP64,
                   per_primary: bool = True, **kw) -> Dict[str, np.ndarray]:
        """The continuous field update over the whole run (karl_run_cycles)."""
        ps, keep = self.host_primaries(prims)
        t = self.empty_tallies(prims.n)
        ts = self.host_tallies(t, per_primary)
        o = self.opts(seed, 2, precision, **kw)
        self._check(karl_run_cycles(self.ctx, ps, o, n_cycles, ts))
        t["per_primary"] = t["per_primary"][:prims.n]
        t["chan_count"] = t["chan_count"][:self.prob.n_channels]
        return t

    def run_cycle(self, prims, seed: int, field_time_in=None, field_recomb_in=None,
                  field_decays: float = 0.0, pid_offset: int = 0, precision: int = FP64,
                  **kw) -> Dict[str, np.ndarray]:
        """One cycle over a primary-id range with the given fields, raw
        tallies (karl_run_cycle)."""
        ps, keep = self.host_primaries(prims, pid_offset)
        t = self.empty_tallies(prims.n)
        ts = self.host_tallies(t, True, with_norm=False)
        o = self.opts(seed, 2, precision, **kw)
        fin = None if field_time_in is None else np.ascontiguousarray(field_time_in, np.uint64)
        rin = None if field_recomb_in is None else np.ascontiguousarray(field_recomb_in, np.uint64)
        self._check(karl_run_cycle(self.ctx, ps, o, fin.ctypes.data if fin is not None else None,
                                   rin.ctypes.data if rin is not None else None,
                                   float(field_decays), ts))
        t["per_primary"] = t["per_primary"][:prims.n]
        t["chan_count"] = t["chan_count"][:self.prob.n_channels]
        return t

    def run_device(self, prim_ptrs: Dict[str, int], n: int, n_decays: int,
                   out_ptrs: Dict[str, int], seed: int = 1, n_passes: Optional[int] = None,
                   precision: int = FP64, stream: Optional[int] = None, pid_offset: int = 0,
                   **kw) -> None:
        """karl_run with device pointers for the primaries and the tallies."""
        ps = Primaries(n, prim_ptrs["z_m"], prim_ptrs["e_ev"], prim_ptrs["mu"],
                       prim_ptrs["species"], n_decays, pid_offset, 1)
        ts = Tallies()
        for k in ("spectrum", "time_fx", "cross_pos", "cross_neg", "recomb", "ledger",
                  "chan_count", "per_primary", "density", "current", "field"):
            setattr(ts, k, out_ptrs.get(k))
        ts.on_device = 1
        o = self.opts(seed, n_passes, precision, stream=stream, **kw)
        self._check(karl_run(self.ctx, ps, o, ts))

    def run_pass_static_device(self, prim_ptrs: Dict[str, int], n: int, n_decays: int,
                               out_ptrs: Dict[str, int], seed: int, pass_index: int,
                               field_time_in: Optional[int] = None, pid_offset: int = 0,
                               precision: int = FP64, stream: Optional[int] = None,
                               **kw) -> None:
        """karl_run_pass_static: device pointers in and out, raw tallies of
        one pass written over out_ptrs, no allocation inside the call."""
        ps = Primaries(n, prim_ptrs["z_m"], prim_ptrs["e_ev"], prim_ptrs["mu"],
                       prim_ptrs["species"], n_decays, pid_offset, 1)
        ts = Tallies()
        for k in ("spectrum", "time_fx", "cross_pos", "cross_neg", "recomb", "ledger",
                  "chan_count", "per_primary"):
            setattr(ts, k, out_ptrs.get(k))
        ts.on_device = 1
        o = self.opts(seed, pass_index, precision, stream=stream, **kw)
        self._check(karl_run_pass_static(self.ctx, ps, o, pass_index, field_time_in, ts))

    def stats(self) -> RunStats:
        return karl_last_stats(self.ctx)

    def cancel(self):
        karl_cancel(self.ctx)


# ---- batched / served form --------------------------------------------------

class ServerOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_slots", C.c_int32),
                ("hbm_budget_bytes", C.c_int64), ("timeout_s", C.c_double),
                ("block_size", C.c_int32), ("blocks_per_sm", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("collected", C.c_int64), ("waiting", C.c_int64), ("collisions", C.c_int64),
                ("kernel_launches", C.c_int64), ("arena_bytes_in_use", C.c_int64),
                ("arena_bytes_peak", C.c_int64), ("lane_occupancy", C.c_double),
                ("kernel_ms", C.c_double)]


_server_bound = False


def _bind_server(lib):
    global _server_bound
    if _server_bound:
        return
    P = C.POINTER
    lib.karl_server_create.argtypes = [P(XS), P(ServerOpts), P(C.c_void_p)]
    lib.karl_server_submit.argtypes = [C.c_void_p, P(Geometry), P(Primaries), C.c_uint64,
                                       C.c_int32, P(Tallies), P(C.c_uint64)]
    lib.karl_server_poll.argtypes = [C.c_void_p, C.c_uint64, P(C.c_int)]
    lib.karl_server_layout.argtypes = [C.c_void_p, P(Geometry), P(Layout)]
    lib.karl_server_run_all.argtypes = [C.c_void_p]
    lib.karl_server_get_stats.argtypes = [C.c_void_p, P(ServerStats)]
    lib.karl_server_destroy.argtypes = [C.c_void_p]
    lib.karl_server_destroy.restype = None
    lib.karl_server_last_error.argtypes = [C.c_void_p]
    lib.karl_server_last_error.restype = C.c_char_p
    for f in ("karl_server_create", "karl_server_submit", "karl_server_poll", "karl_server_layout",
              "karl_server_run_all", "karl_server_get_stats"):
        getattr(lib, f).restype = C.c_int
    _server_bound = True


def _geometry(prob, keep):
    g = Geometry()
    nseg = np.ascontiguousarray(prob.n_seg_m3, np.float64)
    keep.append(nseg)
    g.length_m = prob.length_m
    g.n_zbins = prob.n_zbins
    g.n_seg_m3 = _dptr(nseg)
    g.area_m2 = prob.area_m2
    g.activity_bq = prob.activity_bq
    g.e_cut_ev = prob.e_cut_ev
    g.max_collisions = min(int(prob.max_collisions), 0xFFFFFFFF)
    g.max_lifetime_s = prob.max_lifetime_s if math.isfinite(prob.max_lifetime_s) else math.inf
    g.gas_temperature_k = prob.gas_temperature_k
    g.n_tebins = prob.n_tebins
    g.n_spec_bins = prob.n_spec_bins
    g.spec_bin_ev = prob.spec_bin_ev
    for i in range(N_SPECIES):
        g.species_mass_ev[i] = float(prob.species_mass_ev[i])
    g.target_mass_ev = prob.target_mass_ev
    g.gas_drift_mps = float(getattr(prob, "gas_drift_mps", 0.0))
    return g


def _xs(prob, keep):
    x = XS()
    kind = np.array([c.kind for c in prob.channels], np.int32)
    sin = np.array([c.species_in for c in prob.channels], np.int32)
    sout = np.array([c.species_out for c in prob.channels], np.int32)
    loss = np.array([c.loss_ev for c in prob.channels], np.float64)
    target = np.array([getattr(c, "target", 0) for c in prob.channels], np.int32)
    sig = np.ascontiguousarray(prob.sigma_matrix() if prob.channels
                               else np.zeros((0, prob.n_energy)), np.float64)
    keep += [kind, sin, sout, loss, target, sig]
    x.n_energy = prob.n_energy
    x.e_min_ev = prob.e_min_ev
    x.e_max_ev = prob.e_max_ev
    x.n_channels = prob.n_channels
    x.kind, x.species_in, x.species_out = _iptr(kind), _iptr(sin), _iptr(sout)
    x.loss_ev, x.sigma_m2 = _dptr(loss), _dptr(sig)
    x.ioniz_eps_ev = prob.ioniz_eps_ev
    x.target = _iptr(target)
    ang = _angular(prob, keep)
    if ang is not None:
        x.angular = C.pointer(ang)
    return x


def _angular(prob, keep):
    """karl_angular of the problem's elastic-channel angle tables (one set per
    distinct table object, in channel order), or None when all are isotropic."""
    tabs = [getattr(c, "angular", None) for c in prob.channels]
    sets, index = [], []
    for t in tabs:
        if t is None:
            index.append(-1)
            continue
        for i, u in enumerate(sets):
            if u is t:
                index.append(i)
                break
        else:
            sets.append(t)
            index.append(len(sets) - 1)
    if not sets:
        return None
    nb, nm = np.asarray(sets[0].pdf).shape
    if any(np.asarray(t.pdf).shape != (nb, nm) for t in sets):
        raise ValueError("angle tables of one problem must share their bin and point counts")
    a = Angular()
    idx = np.array(index, np.int32)
    lo = np.array([t.e_min_ev for t in sets], np.float64)
    hi = np.array([t.e_max_ev for t in sets], np.float64)
    thr = np.array([t.threshold_ev for t in sets], np.float64)
    pdf = np.ascontiguousarray(np.stack([np.asarray(t.pdf, np.float64) for t in sets]))
    keep += [idx, lo, hi, thr, pdf, a]
    a.n_sets, a.n_bins, a.n_mu = len(sets), nb, nm
    a.set, a.e_min_ev, a.e_max_ev = _iptr(idx), _dptr(lo), _dptr(hi)
    a.threshold_ev, a.pdf = _dptr(thr), _dptr(pdf)
    return a


class Server:
    """Many requests in one persistent launch (karl_server_*).  The model
    (channels and cross-section tables) is taken from `model_prob`; every
    request brings its own geometry, gas profile, primaries and seed."""

    def __init__(self, model_prob, precision: int = FP64, max_slots: int = 256,
                 hbm_budget_bytes: int = 0, timeout_s: float = 3600.0, block_size: int = 0,
                 blocks_per_sm: int = 0):
        lib = load()
        _bind_server(lib)
        self.lib = lib
        self.model = model_prob
        keep = []
        x = _xs(model_prob, keep)
        o = ServerOpts(precision, max_slots, hbm_budget_bytes, timeout_s, block_size, blocks_per_sm)
        h = C.c_void_p()
        st = lib.karl_server_create(C.byref(x), C.byref(o), C.byref(h))
        if st != OK:
            raise KarlError(st, karl_status_string(st))
        self.h = h
        self._pending = {}             # req id -> (tallies dict, keep-alive objects)

    def _check(self, st):
        if st != OK:
            raise KarlError(st, f"{karl_status_string(st)}: "
                                f"{self.lib.karl_server_last_error(self.h).decode()}")

    def _empty_tallies(self, prob):
        nz, ntb = prob.n_zbins, prob.n_tebins
        return {
            "spectrum": np.zeros((2, N_SPECIES, prob.n_spec_bins + 1), np.uint64),
            "time_fx": np.zeros((N_SPECIES, nz + 2, ntb), np.uint64),
            "cross_pos": np.zeros((N_SPECIES, nz + 1), np.uint64),
            "cross_neg": np.zeros((N_SPECIES, nz + 1), np.uint64),
            "recomb": np.zeros((N_SPECIES, nz), np.uint64),
            "ledger": np.zeros(LEDGER_LEN, np.int64),
            "chan_count": np.zeros(max(self.model.n_channels, 1), np.uint64),
            "density": np.zeros((N_SPECIES, nz), np.float64),
            "current": np.zeros((N_SPECIES, nz + 1), np.float64),
            "field": np.zeros((N_SPECIES, nz, ntb), np.float64),
        }

    def submit(self, prob, prims, seed: int, n_passes: Optional[int] = None,
               pid_offset: int = 0) -> int:
        keep = []
        g = _geometry(prob, keep)
        ps, pk = Context.host_primaries(prims, pid_offset)
        keep.append(pk)
        t = self._empty_tallies(prob)
        ts = Tallies()
        for k in ("spectrum", "time_fx", "cross_pos", "cross_neg", "recomb", "ledger",
                  "chan_count", "density", "current", "field"):
            setattr(ts, k, t[k].ctypes.data)
        ts.per_primary = None
        ts.on_device = 0
        rid = C.c_uint64()
        npass = prob.n_passes if n_passes is None else n_passes
        self._check(self.lib.karl_server_submit(self.h, C.byref(g), C.byref(ps), seed, npass,
                                                C.byref(ts), C.byref(rid)))
        self._pending[rid.value] = (t, keep)
        return rid.value

    def poll(self, req_id: int):
        """(done, tallies or None)."""
        d = C.c_int()
        self._check(self.lib.karl_server_poll(self.h, req_id, C.byref(d)))
        if d.value:
            t, _ = self._pending.pop(req_id)
            t["chan_count"] = t["chan_count"][:self.model.n_channels]
            return True, t
        return False, None

    def run_all(self):
        self._check(self.lib.karl_server_run_all(self.h))

    def stats(self) -> ServerStats:
        s = ServerStats()
        self._check(self.lib.karl_server_get_stats(self.h, C.byref(s)))
        return s

    def close(self):
        if getattr(self, "h", None):
            self.lib.karl_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
