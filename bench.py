"""Benchmark of the KARL transport hot path on GB300.

One step = one whole run of the full-size plain method (1e7 decays, each a
beta electron and a thermal T2+, parabolic 5e21 m^-2 column over 10 m, 1000
segments, seven electron channels, T2+ -> T3+ clustering and electron-ion
recombination, two passes) through the C ABI.  The metric is collision
events per second (performed interactions of all channels in both passes);
primaries/s and flights/s are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Rank 0 prints one JSON line.  With N > 1 (torchrun) every rank runs its own
replica of the workload with its own primary ids (weak scaling, no
collective on the data path); value = all ranks' collisions / max time.
At N = 1 the default line also carries the FP32 precision form's rate on the
same workload (one timed step), bounded measurements of the batched
form (a batch of config-4 source configurations in one persistent launch)
and of the served form (Poisson arrivals at 0.7x the measured capacity and
at 50 requests/s, p50/p99 latency), both in FP32 as their workloads specify,
and of the full-orbit (Boris mover) transport of a tube section
(--workload orbit gives that workload its own line).
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

BYTES_PER_EVENT_FP64 = 104     # event-based state model: 52 B read + 52 B written per event
BYTES_PER_EVENT_FP32 = 80
# The transport kernel keeps particle state in registers and is bound by the
# FP64 pipe (GB300 runs FP64 at 1/64 of FP32: 2 FP64 thread-instructions per
# SM per cycle).  Work per collision, from ncu captures of the transport
# kernel (both passes, collision-weighted) on the 1e6-decay case of this
# workload (profiles/transport_kernel_config2_1e6_counters.md):
#   FP64_OPS: FP64 add, multiply and fma thread-instructions executed with the
#     predicate on (smsp__sass_thread_inst_executed_op_{dadd,dmul,dfma}_pred_on);
#   FP64_PIPE_CYCLES: SM-cycles the FP64 pipe was busy (sm__pipe_fp64_cycles_active),
#     which also counts the lanes a divergent warp leaves idle;
#   DRAM_BYTES: dram__bytes_read.sum + dram__bytes_write.sum, scaled to a launch
#     by its collisions.
FP64_OPS_PER_COLLISION = {"fp64": 117.7, "fp32": 26.2}
FP64_PIPE_CYCLES_PER_COLLISION = {"fp64": 77.0, "fp32": 27.7}
DRAM_BYTES_PER_COLLISION = {"fp64": 0.157, "fp32": 0.242}
FP64_OPS_PER_SM_CYCLE = 2
THREADS_PER_INSTRUCTION = {"fp64": 24.2, "fp32": 22.6}   # smsp__thread_inst_executed_per_inst_executed
WORKLOAD = ("config2: 1e7 decays (1e7 beta e- + 1e7 thermal T2+), parabolic profile with "
            "5e21 m^-2 column, L = 10 m, 1000 z segments, 7 e- channels + T2+ clustering + "
            "e-/ion recombination, two passes")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_sample(n_decays_total: int, seconds: float, threads: int, mode: int = 0):
    """Time the oracle as it stands on a bounded sample of the same workload:
    the first nd decays, pass 1 and then pass 2 with the fields of that pass 1.
    Returns (collisions of both passes, seconds, nd)."""
    import oracle
    from paper_2503_10263_gb300 import inputs
    oracle.build()

    def run(nd):
        prob, prims = inputs.config2(n_decays=nd, seed=1)
        t0 = time.perf_counter()
        r1 = oracle.run_pass(prob, prims, 1, 1, n_decays=nd, mode=mode, n_threads=threads)
        r2 = oracle.run_pass(prob, prims, 1, 2, field_time_in=r1["time_fx"], n_decays=nd,
                             mode=mode, n_threads=threads)
        dt = time.perf_counter() - t0
        coll = int(r1["ledger"][oracle.N_COLLISIONS]) + int(r2["ledger"][oracle.N_COLLISIONS])
        return coll, dt

    nd0 = max(8, min(500, 64 * threads))
    c0, t0 = run(nd0)
    rate = c0 / max(t0, 1e-6)
    per_decay = c0 / nd0
    nd = int(min(n_decays_total, max(nd0, seconds * rate / max(per_decay, 1))))
    c, dt = run(nd)
    return c, dt, nd


def _cpu_baseline(args, threads):
    """The oracle on the host: all cores (optical-depth flights, the form the
    GPU runs), plus one core and the paper-literal segment-stop form."""
    c, secs, nd = _oracle_sample(args.decays, args.cpu_seconds, threads)
    out = {"value": c / secs, "unit": "collision events/s", "cores": threads, "kind": "oracle",
           "sample": f"first {nd} decays of the workload, pass 1 then pass 2 (collisions of "
                     f"both counted), {secs:.1f} s on {threads} threads, optical-depth flights"}
    c1, s1, n1 = _oracle_sample(args.decays, args.cpu_seconds / 3, 1)
    out["one_core"] = {"value": c1 / s1, "cores": 1,
                       "sample": f"first {n1} decays, both passes, {s1:.1f} s"}
    ca, sa, na = _oracle_sample(args.decays, args.cpu_seconds / 3, threads, mode=1)
    out["segment_stop"] = {"value": ca / sa, "cores": threads,
                           "sample": f"first {na} decays, both passes, {sa:.1f} s, "
                                     "flights stopped and redrawn at every segment face"}
    return out


def run_reference(args):
    """--impl reference: the FP64 CPU oracle on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    coll = secs = 0.0
    nd = 0
    for i in range(args.warmup + args.steps):
        c, dt, nd = _oracle_sample(args.decays, args.ref_step_s, threads)
        if i >= args.warmup:
            coll += c
            secs += dt
    value = coll / secs
    sample = (f"first {nd} decays of the workload (both passes) per step; "
              f"timed steps {args.steps}, warm-up steps {args.warmup}")
    line = {
        "metric": "collision events/s", "value": value, "unit": "collision events/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "sample_decays": nd, "parallelism": "host threads"},
        "cpu_baseline": {"value": value, "unit": "collision events/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "collision events/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2503_10263_gb300 import inputs, karl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2503_10263_gb300 import build as kbuild
    kbuild.build()

    prob, prims = inputs.config2(n_decays=args.decays, seed=1)
    n = prims.n
    pid_offset = rank * n                           # each replica has its own primaries
    ctx = karl.Context(prob)
    prec = karl.FP32 if args.precision == "fp32" else karl.FP64
    stream = torch.cuda.current_stream(dev)
    pt = {"z_m": torch.from_numpy(prims.z_m).to(dev), "e_ev": torch.from_numpy(prims.e_ev).to(dev),
          "mu": torch.from_numpy(prims.mu).to(dev),
          "species": torch.from_numpy(prims.species).to(dev)}
    tmpl = ctx.empty_tallies(0)
    dt = {k: torch.zeros(v.shape, dtype=torch.float64 if v.dtype == np.float64 else torch.int64,
                         device=dev) for k, v in tmpl.items() if k != "per_primary"}
    pptr = {k: v.data_ptr() for k, v in pt.items()}
    optr = {k: v.data_ptr() for k, v in dt.items()}

    def step(i):
        ctx.run_device(pptr, n, prims.n_decays, optr, seed=1000 + i, precision=prec,
                       stream=stream.cuda_stream, pid_offset=pid_offset, timeout_s=args.timeout)
        st = ctx.stats()
        return st

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    coll = flights = parts = launches = 0
    kms = []
    occ = []
    per_pass = []
    ev0.record(stream)
    for i in range(args.steps):
        st = step(args.warmup + i)
        coll += st.collisions[0] + st.collisions[1]
        flights += st.flights[0] + st.flights[1]
        parts += st.particles[0] + st.particles[1]
        launches += st.kernel_launches
        kms += [st.kernel_ms[0], st.kernel_ms[1]]
        occ += [st.lane_occupancy[0], st.lane_occupancy[1]]
        per_pass += [int(st.collisions[0]), int(st.collisions[1])]
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    elapsed = ev0.elapsed_time(ev1) / 1000.0
    led = dt["ledger"].cpu().numpy()
    ok_balance = int(led[0]) + int(led[1]) == int(led[2:12].sum())

    # whole-job aggregation: collisions summed, time = max over ranks
    tot = torch.tensor([float(coll), float(flights), float(prims.n_decays * args.steps)],
                       dtype=torch.float64, device=dev)
    tmax = torch.tensor([elapsed], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    coll_all, flights_all, decays_all = tot.tolist()
    tm = float(tmax.item())
    value = coll_all / tm

    # e2e: the same metric through the public API with host buffers (pinned
    # primaries copied in, tallies read back, every step)
    e2e = None
    if args.e2e_steps > 0:
        hp = {k: torch.from_numpy(getattr(prims, k) if k != "species" else prims.species)
              .pin_memory() for k in ("z_m", "e_ev", "mu")}
        hp["species"] = torch.from_numpy(prims.species).pin_memory()
        hprims = karl.Primaries(n, hp["z_m"].data_ptr(), hp["e_ev"].data_ptr(),
                                hp["mu"].data_ptr(), hp["species"].data_ptr(), prims.n_decays,
                                pid_offset, 0)
        host_t = ctx.empty_tallies(0)
        del host_t["per_primary"]
        ts = karl.Tallies()
        for k, v in host_t.items():
            setattr(ts, k, v.ctypes.data)
        ts.on_device = 0
        h2d = sum(int(v.numel() * v.element_size()) for v in hp.values())
        d2h = sum(int(v.nbytes) for v in host_t.values())
        ecoll = 0
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for i in range(args.e2e_steps):
            o = ctx.opts(seed=5000 + i, precision=prec, stream=stream.cuda_stream,
                         timeout_s=args.timeout)
            stt = karl.karl_run(ctx.ctx, hprims, o, ts)
            if stt != karl.OK:
                raise RuntimeError(karl.karl_last_error(ctx.ctx))
            s2 = ctx.stats()
            ecoll += s2.collisions[0] + s2.collisions[1]
        e_el = time.perf_counter() - t0
        et = torch.tensor([float(ecoll)], dtype=torch.float64, device=dev)
        emax = torch.tensor([e_el], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(et, op=dist.ReduceOp.SUM)
            dist.all_reduce(emax, op=dist.ReduceOp.MAX)
        e2e = {"value": float(et.item()) / float(emax.item()), "unit": "collision events/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": args.e2e_steps}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    hbm, peak_kind = _peaks()
    bpe = BYTES_PER_EVENT_FP32 if prec == karl.FP32 else BYTES_PER_EVENT_FP64
    per_launch_events = coll / max(len(kms), 1)
    avg_ms = sum(kms) / max(len(kms), 1)
    launch_rate = per_launch_events / (avg_ms / 1000.0)          # collisions/s inside the kernel
    hbm_achieved = bpe * launch_rate / 1e9
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_ghz = (clocks["sm_mhz"] if clocks else 2070.0) / 1000.0
    ops = FP64_OPS_PER_COLLISION[args.precision]
    cyc = FP64_PIPE_CYCLES_PER_COLLISION[args.precision]
    dram = DRAM_BYTES_PER_COLLISION[args.precision]
    traffic = dram * per_launch_events if dram else None
    # roofline of the hot-path byte model: an event-based form reads and
    # writes each particle's state once per collision event
    roofline = {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm, "unit": "GB/s",
                "frac": hbm_achieved / hbm, "traffic": traffic,
                "model": f"{bpe} B per collision event (particle state read + written once per "
                         f"event) x collisions of a launch / launch time; {peak_kind} copy "
                         f"bandwidth",
                "kernel": "karl::transport_kernel"}
    # what actually bounds this register-resident kernel: the FP64 pipe
    fp64_issue = None
    if ops:
        peak = FP64_OPS_PER_SM_CYCLE * n_sm * clk_ghz
        fp64_issue = {"achieved": ops * launch_rate / 1e9, "peak": peak,
                      "unit": "G FP64 thread-ops/s", "frac": ops * launch_rate / 1e9 / peak,
                      "ops_per_collision": ops,
                      "threads_per_warp_instruction": THREADS_PER_INSTRUCTION[args.precision],
                      "model": f"FP64 add/mul/fma thread-instructions per collision (ncu) "
                               f"against {FP64_OPS_PER_SM_CYCLE} per SM per cycle x {n_sm} SMs "
                               f"x median SM clock under load"}
    fp64_pipe = None
    if cyc:
        fp64_pipe = {"busy_frac": cyc * launch_rate / 1e9 / (n_sm * clk_ghz),
                     "cycles_per_collision": cyc,
                     "note": "FP64 pipe busy cycles over SM cycles (idle lanes of a divergent "
                             "warp and FP64 compares and conversions included)"}
    line = {
        "metric": "collision events/s", "value": value, "unit": "collision events/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * tm / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec == karl.FP32 else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "decays": args.decays, "primaries_per_decay": 2,
                   "precision": args.precision, "l2": "inputs larger than L2 (primaries 500 MB)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "primaries_per_s": decays_all / tm, "flights_per_s": flights_all / tm,
        "collisions_per_step": coll / args.steps,
        "transport_kernel_ms": kms,
        "collisions_per_launch": per_pass,
        "ns_per_collision_by_pass": [
            round(1e6 * sum(kms[0::2]) / max(sum(per_pass[0::2]), 1), 4),
            round(1e6 * sum(kms[1::2]) / max(sum(per_pass[1::2]), 1), 4)],
        "lane_occupancy": [round(x, 4) for x in occ],
        "ledger_balanced": ok_balance,
        "gpu_launches": launches,
        "roofline": roofline,
        "fp64_issue": fp64_issue,
        "fp64_pipe": fp64_pipe,
        "e2e": e2e,
        "clocks": clocks,
    }
    if args.other_precision and world == 1:
        # the same workload in the other form (FP32 beside the FP64 line), one
        # warm-up step and one timed step, device buffers, CUDA-event kernel time
        other = karl.FP64 if prec == karl.FP32 else karl.FP32
        oname = "fp64" if other == karl.FP64 else "fp32"
        ctx.run_device(pptr, n, prims.n_decays, optr, seed=7000, precision=other,
                       stream=stream.cuda_stream, timeout_s=args.timeout)
        ctx.run_device(pptr, n, prims.n_decays, optr, seed=7001, precision=other,
                       stream=stream.cuda_stream, timeout_s=args.timeout)
        so = ctx.stats()
        oc = [int(so.collisions[0]), int(so.collisions[1])]
        om = [float(so.kernel_ms[0]), float(so.kernel_ms[1])]
        line[oname] = {"value": sum(oc) / (sum(om) / 1000.0), "unit": "collision events/s",
                       "transport_kernel_ms": om, "collisions_per_launch": oc,
                       "ns_per_collision_by_pass": [round(1e6 * om[i] / max(oc[i], 1), 4)
                                                    for i in range(2)],
                       "lane_occupancy": [round(x, 4) for x in so.lane_occupancy],
                       "fp64_ops_per_collision": FP64_OPS_PER_COLLISION[oname],
                       "roofline": {"bound": "hbm", "frac": (BYTES_PER_EVENT_FP32 if oname == "fp32"
                                                             else BYTES_PER_EVENT_FP64)
                                    * sum(oc) / (sum(om) / 1000.0) / 1e9 / hbm,
                                    "unit": "GB/s", "peak": hbm}}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(args, os.cpu_count() or 1)
    if args.forms_configs > 0 and world == 1:
        line["batched"], line["served"] = forms_subline(args)
    if args.orbit_sub_ions > 0 and world == 1:
        line["orbit"] = orbit_measure(args.orbit_sub_ions, 1, 1, args.timeout,
                                      0.0 if args.no_cpu_baseline else 5.0)
        line["orbit"]["workload"] = WORKLOAD_ORBIT
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


WORKLOAD4 = ("config4: 256 source configurations in one persistent launch (column U[0.1,1] x "
             "5e21 m^-2, L U[2,10] m, decays log-U[1e3,1e6], full channel set, two passes)")
WORKLOAD5 = ("config5: Poisson arrivals of config-4-style requests (decays log-U[1e3,1e6]), "
             "admitted by HBM footprint into one running launch (continuous batching)")


def _percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * q / 100.0
    f = int(math.floor(k))
    c = min(f + 1, len(xs) - 1)
    return xs[f] + (xs[c] - xs[f]) * (k - f)


def run_batch(args):
    """config 4: the whole batch of source configurations per step, through
    the server API (inputs copied in and tallies read back every step)."""
    import torch

    from paper_2503_10263_gb300 import autotune, build as kbuild, inputs, karl
    kbuild.build()
    torch.cuda.set_device(0)
    prec = karl.FP32 if args.precision == "fp32" else karl.FP64
    block, bps = autotune.tune(prec)
    batch = inputs.config4_batch(n_configs=args.configs, meta_seed=1)
    n_decays = sum(pr.n_decays for _, pr, _ in batch)
    h2d = sum(pr.n * 25 for _, pr, _ in batch)

    def step():
        srv = karl.Server(batch[0][0], precision=prec, hbm_budget_bytes=args.budget_gb << 30,
                          timeout_s=args.timeout, block_size=block, blocks_per_sm=bps)
        ids = [srv.submit(p, pr, s) for p, pr, s in batch]
        srv.run_all()
        coll = 0
        d2h = 0
        for rid in ids:
            done, t = srv.poll(rid)
            coll += int(t["ledger"][karl.N_COLLISIONS_ALL])
            d2h += sum(v.nbytes for v in t.values())
        st = srv.stats()
        srv.close()
        return coll, st.kernel_ms, st.kernel_launches, d2h, st.lane_occupancy

    for _ in range(args.warmup):
        step()
    sampler = ClockSampler(0)
    sampler.start()
    t0 = time.perf_counter()
    coll = kms = launches = d2h = 0
    occ = []
    for _ in range(args.steps):
        c, k, l, d, o = step()
        coll += c
        kms += k
        launches += l
        d2h = d
        occ.append(o)
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    line = {
        "metric": "collision events/s", "value": coll / (kms / 1000.0), "unit": "collision events/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * wall / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec == karl.FP32 else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD4, "configs": args.configs, "decays": n_decays,
                   "block_size": block, "blocks_per_sm": bps, "launches_per_step": launches / args.steps},
        "primaries_per_s": n_decays * args.steps / (kms / 1000.0),
        "e2e": {"value": coll / wall, "unit": "collision events/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "lane_occupancy": occ, "clocks": clocks,
    }
    if args.compare_plain:
        line["plain_one_at_a_time"] = plain_sequential(batch, prec, args.timeout)
    print(json.dumps(line), flush=True)


def plain_sequential(batch, prec, timeout):
    """The same requests through the plain single-request path (karl_run),
    one after another: the comparison for the batched and served forms."""
    import torch

    from paper_2503_10263_gb300 import karl
    coll = 0
    kms = 0.0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for p, pr, s in batch:
        ctx = karl.Context(p)
        t = ctx.run(pr, seed=s, precision=prec, per_primary=False, timeout_s=timeout)
        st = ctx.stats()
        coll += int(t["ledger"][karl.N_COLLISIONS_ALL])
        kms += float(st.kernel_ms[0]) + float(st.kernel_ms[1])
        ctx.close()
    wall = time.perf_counter() - t0
    return {"value": coll / wall, "kernel_value": coll / (kms / 1000.0),
            "unit": "collision events/s", "requests": len(batch),
            "note": "karl_run per request, host buffers, two passes each; value = wall clock, "
                    "kernel_value = transport kernel time only"}


def serve_arrivals(srv, reqs, karl):
    """Submit each request at its arrival time into the running server and
    collect results as they finish; returns (latencies, collisions, wall s).
    Latency = completion - arrival on the host clock."""
    t0 = time.perf_counter()
    nxt = 0
    open_ids = {}
    lat, coll = [], 0
    while nxt < len(reqs) or open_ids:
        now = time.perf_counter() - t0
        while nxt < len(reqs) and reqs[nxt][0] <= now:
            ta, p, pr, s = reqs[nxt]
            open_ids[srv.submit(p, pr, s)] = ta
            nxt += 1
        for rid in list(open_ids):
            done, t = srv.poll(rid)
            if done:
                lat.append(time.perf_counter() - t0 - open_ids.pop(rid))
                coll += int(t["ledger"][karl.N_COLLISIONS_ALL])
        time.sleep(0.0005)
    return lat, coll, time.perf_counter() - t0


def forms_subline(args):
    """Bounded measurements of the batched and served forms (FP32, as their
    workloads specify) for the default line: one batch of the first
    args.forms_configs source configurations of the config-4 batch (one warm-up
    batch, one timed), then Poisson arrivals of config-5-style requests at 0.7x
    the capacity that batch measured and at 50 requests/s, each for a stated
    window, the latency of every request from arrival to result."""
    from paper_2503_10263_gb300 import autotune, inputs, karl
    prec = karl.FP32
    t_tune = time.perf_counter()
    block, bps = autotune.tune(prec)
    t_tune = time.perf_counter() - t_tune
    batch = inputs.config4_batch(n_configs=args.forms_configs, meta_seed=1)
    n_decays = sum(pr.n_decays for _, pr, _ in batch)

    def one_batch():
        srv = karl.Server(batch[0][0], precision=prec, hbm_budget_bytes=args.budget_gb << 30,
                          timeout_s=args.timeout, block_size=block, blocks_per_sm=bps)
        t0 = time.perf_counter()
        ids = [srv.submit(p, pr, s) for p, pr, s in batch]
        srv.run_all()
        coll = sum(int(srv.poll(rid)[1]["ledger"][karl.N_COLLISIONS_ALL]) for rid in ids)
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        return coll, wall, st

    one_batch()
    coll, wall, st = one_batch()
    batched = {"value": coll / (st.kernel_ms / 1000.0), "unit": "collision events/s",
               "e2e": coll / wall, "collisions": coll, "both_passes": True,
               "configs": len(batch), "decays": n_decays, "kernel_launches": st.kernel_launches,
               "lane_occupancy": st.lane_occupancy, "block_size": block, "blocks_per_sm": bps,
               "autotune_s": round(t_tune, 1), "precision": "fp32",
               "workload": f"first {len(batch)} configurations of the config-4 batch, one "
                           f"persistent launch, inputs copied in and tallies read back"}
    # capacity in requests/s: sustained rate over the mean work of a request
    mean_coll = coll / len(batch)
    capacity = (coll / wall) / mean_coll
    served = {"capacity_req_s": capacity, "precision": "fp32", "loads": []}
    for rate, window in ((0.7 * capacity, args.serve_window_low), (50.0, args.serve_window_high)):
        reqs = inputs.config5_requests(duration_s=window, rate_hz=rate, arrival_seed=1)
        if not reqs:
            continue
        srv = karl.Server(reqs[0][1], precision=prec, hbm_budget_bytes=args.budget_gb << 30,
                          max_slots=1024, timeout_s=args.timeout, block_size=block,
                          blocks_per_sm=bps)
        lat, scoll, swall = serve_arrivals(srv, reqs, karl)
        srv.run_all()
        sst = srv.stats()
        srv.close()
        served["loads"].append({
            "offered_req_s": rate, "arrival_window_s": window, "requests": len(reqs),
            "p50_latency_s": _percentile(lat, 50), "p99_latency_s": _percentile(lat, 99),
            "sustained_collisions_per_s": scoll / swall, "wall_s": swall,
            "kernel_launches": sst.kernel_launches})
    return batched, served


WORKLOAD_ORBIT = ("orbit ions: full-orbit Boris mover at B = 2.5 T with a radial field of "
                  "2e3 V/m^2 in a 45 mm tube (45 radial bins), 1 m of 5e19 m^-3 T2 in 100 "
                  "segments; thermal T2+ born over the cross section, T2+ -> T3+ clustering, "
                  "ion elastic scattering; lifetime cap 1e-4 s (about 3.5e4 steps per ion)")
# Per Boris step of the orbit kernel (ncu, profiles/orbit_kernel_ions_counters.md):
# FP64 add/mul/fma thread-instructions with the predicate on, and SM-cycles
# the FP64 pipe was busy
FP64_OPS_PER_STEP = 118.1
FP64_PIPE_CYCLES_PER_STEP = 91.8


def orbit_measure(n_ions: int, steps: int, warmup: int, timeout: float, cpu_seconds: float,
                  lifetime_s: float = 1e-4):
    """Full-orbit workload: `steps` timed runs of n_ions ions through
    karl_run_orbit (host buffers, so the wall time includes the copies), the
    kernel time from CUDA events; the oracle timed on a bounded sample."""
    from paper_2503_10263_gb300 import inputs, karl
    prob, orb, pr = inputs.orbit_ion_config(n_ions=n_ions, seed=1, lifetime_s=lifetime_s)
    ctx = karl.Context(prob)
    try:
        for i in range(warmup):
            ctx.run_orbit(orb, pr, seed=100 + i, timeout_s=timeout)
        kms = wall = 0.0
        nsteps = coll = launches = d2h = 0
        for i in range(steps):
            t0 = time.perf_counter()
            t = ctx.run_orbit(orb, pr, seed=200 + i, timeout_s=timeout)
            wall += time.perf_counter() - t0
            d2h = sum(v.nbytes for v in t.values())
            st = ctx.stats()
            kms += st.kernel_ms[0]
            launches += st.kernel_launches
            nsteps += int(t["ledger"][karl.OB_N_STEPS])
            coll += int(t["ledger"][karl.OB_N_COLLISIONS])
    finally:
        ctx.close()
    out = {"value": nsteps / (kms / 1000.0), "unit": "Boris steps/s",
           "collisions_per_s": coll / (kms / 1000.0), "steps_per_run": nsteps / steps,
           "collisions_per_run": coll / steps, "kernel_launches_per_run": launches / steps,
           "e2e": {"value": nsteps / wall, "unit": "Boris steps/s",
                   "h2d_bytes_per_step": pr.n * 49, "d2h_bytes_per_step": d2h},
           "ions": pr.n}
    # the orbit kernel is bound by the FP64 pipe: "alu" roofline against the
    # FP64 issue rate of 2 thread-instructions per SM per cycle at 2.07 GHz
    peak = FP64_OPS_PER_SM_CYCLE * 152 * 2.07e9
    out["roofline"] = {"bound": "alu", "achieved": FP64_OPS_PER_STEP * out["value"] / 1e9,
                       "peak": peak / 1e9, "unit": "G FP64 thread-ops/s",
                       "frac": FP64_OPS_PER_STEP * out["value"] / peak,
                       "ops_per_step": FP64_OPS_PER_STEP, "kernel": "karl::orbit_kernel",
                       "traffic": None,
                       "fp64_pipe_busy_frac": FP64_PIPE_CYCLES_PER_STEP * out["value"] /
                       (152 * 2.07e9)}
    if cpu_seconds > 0:
        import oracle
        threads = os.cpu_count() or 1
        m = 64
        while True:
            sub = inputs.OrbitPrimaries(*(getattr(pr, k)[:m] for k in
                                          ("x_m", "y_m", "z_m", "e_ev", "mu", "phi", "species")))
            t0 = time.perf_counter()
            o = oracle.orbit_run(prob, orb, sub, seed=200, n_threads=threads)
            dt = time.perf_counter() - t0
            if dt > 0.25 * cpu_seconds or 2 * m > pr.n:
                break
            m *= 2
        out["cpu_baseline"] = {"value": float(o["ledger"][oracle.OB_N_STEPS]) / dt,
                               "unit": "Boris steps/s", "cores": threads, "kind": "oracle",
                               "sample": f"first {m} primaries of the workload, {dt:.1f} s"}
    return out


def run_orbit_line(args):
    """--workload orbit: the full-orbit workload's own JSON line."""
    import torch
    from paper_2503_10263_gb300 import build as kbuild
    kbuild.build()
    torch.cuda.set_device(0)
    sampler = ClockSampler(0)
    sampler.start()
    t0 = time.perf_counter()
    m = orbit_measure(args.orbit_ions, args.steps, args.warmup, args.timeout,
                      0.0 if args.no_cpu_baseline else args.cpu_seconds, args.orbit_lifetime)
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    line = {"metric": "Boris steps/s", "value": m["value"], "unit": "Boris steps/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * wall / max(args.steps + args.warmup, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_ORBIT, "ions": args.orbit_ions,
                       "lifetime_s": args.orbit_lifetime,
                       "l2": "tallies L2-resident; particle state in registers"},
            "clocks": clocks}
    line.update({k: v for k, v in m.items() if k != "value"})
    print(json.dumps(line), flush=True)


def run_serve(args):
    """config 5: Poisson arrivals submitted on time into one running launch;
    latency = completion - arrival on the host clock."""
    import torch

    from paper_2503_10263_gb300 import autotune, build as kbuild, inputs, karl
    kbuild.build()
    torch.cuda.set_device(0)
    prec = karl.FP32 if args.precision == "fp32" else karl.FP64
    block, bps = autotune.tune(prec)
    reqs = inputs.config5_requests(duration_s=args.serve_seconds, rate_hz=args.rate, arrival_seed=1)
    srv = karl.Server(reqs[0][1], precision=prec, hbm_budget_bytes=args.budget_gb << 30,
                      max_slots=1024, timeout_s=args.timeout, block_size=block, blocks_per_sm=bps)
    sampler = ClockSampler(0)
    sampler.start()
    lat, coll, wall = serve_arrivals(srv, reqs, karl)
    srv.run_all()
    st = srv.stats()
    srv.close()
    clocks = sampler.stop()
    offered = sum(pr.n_decays for _, _, pr, _ in reqs)
    line = {
        "metric": "p99 request latency", "value": _percentile(lat, 99), "unit": "s",
        "higher_is_better": False, "n_gpus": 1, "steps": 1, "warmup": 0,
        "ms_per_step": 1000.0 * wall, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == karl.FP32 else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD5, "rate_hz": args.rate, "arrival_seconds": args.serve_seconds,
                   "requests": len(reqs), "decays": offered, "block_size": block,
                   "blocks_per_sm": bps},
        "p50_latency_s": _percentile(lat, 50), "p99_latency_s": _percentile(lat, 99),
        "sustained_collisions_per_s": coll / wall, "kernel_launches": st.kernel_launches,
        "arena_bytes_peak": st.arena_bytes_peak, "clocks": clocks,
    }
    if args.compare_plain:
        line["plain_one_at_a_time"] = plain_serve(reqs, prec, args.timeout)
    print(json.dumps(line), flush=True)


def plain_serve(reqs, prec, timeout):
    """The same arrivals served first-come first-served by the plain path:
    one karl_run at a time, each request waiting for the one before it."""
    import torch

    from paper_2503_10263_gb300 import karl
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat, coll = [], 0
    for ta, p, pr, s in reqs:
        now = time.perf_counter() - t0
        if now < ta:
            time.sleep(ta - now)
        ctx = karl.Context(p)
        t = ctx.run(pr, seed=s, precision=prec, per_primary=False, timeout_s=timeout)
        ctx.close()
        lat.append(time.perf_counter() - t0 - ta)
        coll += int(t["ledger"][karl.N_COLLISIONS_ALL])
    wall = time.perf_counter() - t0
    return {"p50_latency_s": _percentile(lat, 50), "p99_latency_s": _percentile(lat, 99),
            "sustained_collisions_per_s": coll / wall, "requests": len(reqs),
            "note": "first-come first-served, one karl_run (two passes) per request"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--decays", type=int, default=10_000_000)
    # default: the plain method (config 2) in FP64, the batched and served
    # forms (configs 4 and 5) in FP32, as their workloads specify
    ap.add_argument("--precision", choices=["fp64", "fp32"], default=None)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--timeout", type=float, default=600.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-step-s", type=float, default=10.0)
    ap.add_argument("--workload", choices=["config2", "config4", "config5", "orbit"],
                    default="config2")
    ap.add_argument("--orbit-ions", type=int, default=1 << 20,
                    help="ions of the full-orbit workload (--workload orbit)")
    ap.add_argument("--other-precision", type=int, default=1,
                    help="default line: also time the other form (FP32 beside FP64) once")
    ap.add_argument("--orbit-lifetime", type=float, default=1e-4,
                    help="lifetime cap of the full-orbit workload (shorter: a small profiling case)")
    ap.add_argument("--orbit-sub-ions", type=int, default=1 << 17,
                    help="ions of the default line's full-orbit measurement (0: leave it out)")
    ap.add_argument("--configs", type=int, default=256)
    ap.add_argument("--budget-gb", type=int, default=48)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--forms-configs", type=int, default=48,
                    help="default line: configurations of the bounded batched/served "
                         "measurement (0: leave it out)")
    ap.add_argument("--serve-window-low", type=float, default=8.0)
    ap.add_argument("--serve-window-high", type=float, default=1.5)
    ap.add_argument("--compare-plain", action="store_true",
                    help="config4/config5: also run the requests one at a time through karl_run")
    args = ap.parse_args()
    if args.precision is None:
        args.precision = "fp64" if args.workload in ("config2", "orbit") else "fp32"
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "config4":
        run_batch(args)
    elif args.workload == "config5":
        run_serve(args)
    elif args.workload == "orbit":
        run_orbit_line(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
