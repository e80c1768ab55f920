"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
exports every entry point include/karl.h declares, and rejects invalid
arguments before any CUDA call."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

from paper_2503_10263_gb300 import build as kbuild
from paper_2503_10263_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def karl():
    kbuild.build()
    from paper_2503_10263_gb300 import karl as k
    k.load()
    return k


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    return sorted(set(re.findall(r"\b(karl_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(karl):
    lib = C.CDLL(karl.LIB_PATH)
    names = _declared("karl.h")
    assert "karl_create" in names and "karl_run" in names
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(karl):
    for s in range(10):
        assert karl.karl_status_string(s)
    assert karl.karl_status_string(0) == "ok"
    assert "unknown" in karl.karl_status_string(99)


def test_create_rejects_invalid_arguments_without_gpu(karl):
    prob, _ = inputs.config1(n_primaries=10)
    bad = [("length_m", -1.0), ("n_zbins", 0), ("area_m2", 0.0), ("activity_bq", 0.0),
           ("n_tebins", 0), ("spec_bin_ev", 0.0)]
    for field, val in bad:
        p, _ = inputs.config1(n_primaries=10)
        setattr(p, field, val)
        with pytest.raises(karl.KarlError) as ei:
            karl.Context(p)
        assert ei.value.status == karl.EINVAL, field
    p, _ = inputs.config1(n_primaries=10)
    p.n_seg_m3 = p.n_seg_m3.copy()
    p.n_seg_m3[3] = -1.0
    with pytest.raises(karl.KarlError):
        karl.Context(p)
    p, _ = inputs.config1(n_primaries=10)
    p.channels[0].sigma_m2 = p.channels[0].sigma_m2.copy()
    p.channels[0].sigma_m2[5] = math.nan
    with pytest.raises(karl.KarlError):
        karl.Context(p)
    p, _ = inputs.config1(n_primaries=10)
    p.channels[1].species_in = 7
    with pytest.raises(karl.KarlError):
        karl.Context(p)
    # a moving target is defined for elastic and ionization channels only
    # (channel 2 of config 1 is an excitation)
    for k, t in ((2, 1), (0, 2)):
        p, _ = inputs.config1(n_primaries=10)
        p.channels[k].target = t
        with pytest.raises(karl.KarlError) as ei:
            karl.Context(p)
        assert ei.value.status == karl.EINVAL
    p, _ = inputs.thermalization(n_primaries=10)
    p.gas_drift_mps = math.inf
    with pytest.raises(karl.KarlError):
        karl.Context(p)


def test_missing_library_fails_loudly(monkeypatch):
    from paper_2503_10263_gb300 import karl as k
    monkeypatch.setattr(k, "_lib", None)
    monkeypatch.setattr(k, "LIB_PATH", "/nonexistent/libkarl.so")
    with pytest.raises(ImportError):
        k.load()


def test_create_rejects_invalid_angle_tables_without_gpu(karl):
    def with_table(k=0, **kw):
        p, _ = inputs.config1(n_primaries=10)
        t = inputs.screened_rutherford_table(n_bins=4, n_mu=9)
        for f, v in kw.items():
            setattr(t, f, v)
        p.channels[k].angular = t
        return p

    x = np.linspace(-1, 1, 9)
    zero_bin = np.stack([1.0 + 0 * x, 0 * x, 1.0 + x, 1.0 - x])
    neg = np.tile(1.0 - 1.5 * x, (4, 1))
    for p in (with_table(k=1),                       # ionization: no angle table
              with_table(e_min_ev=0.0), with_table(e_max_ev=50.0),
              with_table(threshold_ev=-1.0), with_table(threshold_ev=math.nan),
              with_table(pdf=zero_bin), with_table(pdf=neg),
              with_table(pdf=np.ones((4, 1)))):
        with pytest.raises(karl.KarlError) as ei:
            karl.Context(p)
        assert ei.value.status == karl.EINVAL


def test_create_rejects_invalid_ion_chemistry_without_gpu(karl):
    nodes = inputs.energy_nodes(64, 1.0, 2e4)
    bad = [
        # charge exchange of an electron
        [inputs.Channel("cx", inputs.CHARGE_EXCHANGE, inputs.E, -1, 0.0, np.ones(64) * 1e-20)],
        # three-body clustering without a product
        [inputs.Channel("c3", inputs.CLUSTERING3, inputs.TP, -1, 0.0, np.ones(64) * 1e-40)],
        # three field-rate channels on one species
        [inputs.Channel("c3", inputs.CLUSTERING3, inputs.TP, inputs.T3P, 0.0, np.ones(64)),
         inputs.Channel("r1", inputs.RECOMBINATION, inputs.TP, inputs.E, 0.0, np.ones(64)),
         inputs.Channel("c3b", inputs.CLUSTERING3, inputs.TP, inputs.T3P, 0.0, np.ones(64))],
        # unknown kind
        [inputs.Channel("x", 7, inputs.TP, inputs.T3P, 0.0, np.ones(64))],
    ]
    for chans in bad:
        p = inputs.uniform_problem(1e20, 1.0, 10, chans, n_energy=64)
        with pytest.raises(karl.KarlError) as ei:
            karl.Context(p)
        assert ei.value.status == karl.EINVAL


def test_shipped_problems_pass_host_validation():
    # karl_create checks every argument before its first CUDA call: without a
    # GPU a valid problem fails later, with KARL_ECUDA, an invalid one with
    # KARL_EINVAL.  Every problem builder of inputs.py must pass the checks.
    import torch
    if torch.cuda.is_available():
        pytest.skip("with a GPU the problems are created for real by the GPU tests")
    from paper_2503_10263_gb300 import karl as k
    probs = [inputs.config1(n_primaries=10)[0], inputs.config2(n_decays=10)[0],
             inputs.angular_config(n_primaries=10)[0], inputs.thermalization(n_primaries=10)[0],
             inputs.chemistry_config(10)[0],
             inputs.charge_exchange_problem(1e20, 1.0, 10, 80.0)]
    for p in probs:
        with pytest.raises(k.KarlError) as ei:
            k.Context(p)
        assert ei.value.status == k.ECUDA, p.name


def test_autotune_candidates_fit_the_multi_request_kernel():
    """The server accepts blocks of 32..256 threads (multiples of 32)."""
    from paper_2503_10263_gb300 import autotune
    for block, bps in autotune.CANDIDATES:
        assert 32 <= block <= 256 and block % 32 == 0 and bps >= 1
