"""karl_run_pass_static: one pass with all scratch in the library's static
device array.  It runs the same transport kernel as karl_run_pass, and integer
tallies commute, so its raw tallies must equal karl_run_pass's bit for bit, on
two calls in a row (the scratch is reused and must be re-cleared).  Collected
last so that it also runs after every other GPU test in the same process.
"""
import numpy as np
import pytest

from paper_2503_10263_gb300 import inputs

pytestmark = pytest.mark.gpu

RAW = ("spectrum", "time_fx", "cross_pos", "cross_neg", "recomb", "ledger", "chan_count",
       "per_primary")


@pytest.fixture(scope="module")
def karl():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_10263_gb300 import karl as k
    return k


def _device_prims(torch, prims):
    d = {
        "z_m": torch.tensor(np.ascontiguousarray(prims.z_m), dtype=torch.float64, device="cuda"),
        "e_ev": torch.tensor(np.ascontiguousarray(prims.e_ev), dtype=torch.float64, device="cuda"),
        "mu": torch.tensor(np.ascontiguousarray(prims.mu), dtype=torch.float64, device="cuda"),
        "species": torch.tensor(np.ascontiguousarray(prims.species), dtype=torch.uint8,
                                device="cuda"),
    }
    return d, {k: v.data_ptr() for k, v in d.items()}


def _device_tallies(torch, ctx, n):
    host = ctx.empty_tallies(n)
    # 64-bit words; garbage-filled so the test sees any word the call fails to write
    d = {k: torch.full((host[k].size,), -7, dtype=torch.int64, device="cuda") for k in RAW}
    return d, {k: v.data_ptr() for k, v in d.items()}


def _to_host(d, n, nch):
    out = {k: v.cpu().numpy().view(np.uint64) for k, v in d.items()}
    out["ledger"] = out["ledger"].view(np.int64)
    out["per_primary"] = out["per_primary"][:n]
    out["chan_count"] = out["chan_count"][:nch]
    return out


def _same(a, b, prefix):
    for k in RAW:
        np.testing.assert_array_equal(np.asarray(a[k]).ravel(), np.asarray(b[k]).ravel(),
                                      err_msg=f"{prefix}: {k}")


@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
def test_static_pass_equals_run_pass_twice(karl, prec_name):
    import torch
    prec = karl.FP32 if prec_name == "fp32" else karl.FP64
    prob, prims = inputs.config2(n_decays=3000, seed=4)
    ctx = karl.Context(prob)
    seed = 17
    ref1 = ctx.run_pass(prims, seed, 1, n_decays=prims.n_decays, precision=prec)
    ref2 = ctx.run_pass(prims, seed, 2, field_time_in=ref1["time_fx"], n_decays=prims.n_decays,
                        precision=prec)
    dp, pp = _device_prims(torch, prims)
    nch = prob.n_channels
    for call in range(2):                      # two calls in a row on the same scratch
        d1, p1 = _device_tallies(torch, ctx, prims.n)
        ctx.run_pass_static_device(pp, prims.n, prims.n_decays, p1, seed, 1, precision=prec)
        got1 = _to_host(d1, prims.n, nch)
        _same(got1, ref1, f"pass 1, call {call}")
        d2, p2 = _device_tallies(torch, ctx, prims.n)
        ctx.run_pass_static_device(pp, prims.n, prims.n_decays, p2, seed, 2,
                                   field_time_in=d1["time_fx"].data_ptr(), precision=prec)
        got2 = _to_host(d2, prims.n, nch)
        _same(got2, ref2, f"pass 2, call {call}")
    assert int(ref1["ledger"][karl.N_COLLISIONS]) > 0
    st = ctx.stats()
    assert st.queue_capacity >= 1 << 16


def test_static_pass_rejects_what_it_cannot_hold(karl):
    import torch
    # time difference arrays of 2 x 4 x 100002 x 64 x 8 bytes (410 MB) do not
    # fit the 64 MiB array
    nz = 100_000
    big = inputs._problem("big", 10.0, nz, np.full(nz, 1e19), full=False, n_tebins=64)
    _, prims = inputs.config1(n_primaries=10)
    ctx = karl.Context(big)
    dp, pp = _device_prims(torch, prims)
    d, p = _device_tallies(torch, ctx, prims.n)
    with pytest.raises(karl.KarlError) as e:
        ctx.run_pass_static_device(pp, prims.n, prims.n_decays, p, 1, 1)
    assert e.value.status == karl.ECAPACITY
    assert "static scratch" in str(e.value)
    # host buffers are refused: the call copies nothing through staging memory
    small, _ = inputs.config1(n_primaries=10)
    ctx2 = karl.Context(small)
    ps, keep = ctx2.host_primaries(prims)
    t = ctx2.empty_tallies(prims.n)
    ts = ctx2.host_tallies(t, True, with_norm=False)
    st = karl.karl_run_pass_static(ctx2.ctx, ps, ctx2.opts(1, 1), 1, None, ts)
    assert st == karl.EINVAL
    # device primaries and tallies but a host pass-1 time tally for pass 2 (the
    # form karl_run_pass takes): refused before any launch, not read by a kernel
    dp2, pp2 = _device_prims(torch, prims)
    d2, p2 = _device_tallies(torch, ctx2, prims.n)
    host_time = np.zeros(ctx2.empty_tallies(1)["time_fx"].size, np.uint64)
    with pytest.raises(karl.KarlError) as e2:
        ctx2.run_pass_static_device(pp2, prims.n, prims.n_decays, p2, 1, 2,
                                    field_time_in=host_time.ctypes.data)
    assert e2.value.status == karl.EINVAL and "field_time_in" in str(e2.value)
    # a host tally buffer among device ones
    host_ledger = np.zeros(karl.LEDGER_LEN, np.int64)
    p3 = dict(p2, ledger=host_ledger.ctypes.data)
    with pytest.raises(karl.KarlError) as e3:
        ctx2.run_pass_static_device(pp2, prims.n, prims.n_decays, p3, 1, 1)
    assert e3.value.status == karl.EINVAL and "ledger" in str(e3.value)
    # the context still runs
    ctx2.run_pass_static_device(pp2, prims.n, prims.n_decays, p2, 1, 1)


def test_static_pass_leaves_free_device_memory_unchanged(karl):
    """The property the entry point exists for: a call takes no device memory.
    After a first call (which looks up the scratch array's address), free
    device memory is the same before and after each further call."""
    import torch
    prob, prims = inputs.config2(n_decays=2000, seed=6)
    ctx = karl.Context(prob)
    dp, pp = _device_prims(torch, prims)
    d1, p1 = _device_tallies(torch, ctx, prims.n)
    d2, p2 = _device_tallies(torch, ctx, prims.n)
    ctx.run_pass_static_device(pp, prims.n, prims.n_decays, p1, 3, 1)        # set-up call
    torch.cuda.synchronize()
    for call in range(2):
        free0 = torch.cuda.mem_get_info()[0]
        ctx.run_pass_static_device(pp, prims.n, prims.n_decays, p1, 3, 1)
        ctx.run_pass_static_device(pp, prims.n, prims.n_decays, p2, 3, 2,
                                   field_time_in=d1["time_fx"].data_ptr())
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, call
    # control: the same measurement sees a 256 MiB device allocation (torch's
    # cache emptied first, so the block is a new allocation)
    torch.cuda.empty_cache()
    free0 = torch.cuda.mem_get_info()[0]
    block = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    assert free0 - torch.cuda.mem_get_info()[0] >= 256 << 20
    del block
    torch.cuda.empty_cache()
