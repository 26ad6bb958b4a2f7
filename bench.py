#!/usr/bin/env python3
"""Benchmark of the trapped-ion timestep on GB300.

Workload (one bench step): the two-species precision workload -- 3072 Ca+ and 1024 NH3+
ions, Gaussian cloud sigma = 100 um (seed 1), thermal 10 mK, linear Paul trap
Omega = 2 pi 3.85 MHz, q = 0.3, a = -0.001, f_z = 0.2 MHz, Langevin 1e5 1/s to 1 mK --
advanced by 5000 velocity-Verlet steps at dt = T_RF/20 in the FP32 precision form
(FP32 pair forces with compensated accumulation, FP64 state).  Metric: ion-steps/s
(ions x timesteps / s); pair-interactions/s (ordered pairs N(N-1) per timestep) beside it.

  value      device-timed (CUDA events on the launching stream), state resident in HBM
  e2e        the same metric through the C ABI with host buffers: create (H2D copy of
             x, v, species) + 5000 steps + state read-back (D2H) every bench step
  roofline   the step kernel against the FP32-pipe roof of its instruction mix
  cpu_baseline  the FP64 oracle (C, OpenMP) on this host's cores, bounded sample
  extra      the plain FP64 GPU form on the same workload, the N = 32768 crystal

``--impl reference`` times the FP64 oracle on the host cores instead (the comparison
arm for this method: there is no other implementation of it to run).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

STEPS_PER_BENCH_STEP = 5000
# FP32-pipe instructions per ordered pair in the hi/lo pair term: 9 FADD (differences),
# 3 FMUL/FFMA (r^2), 3 FMUL (z_j r^-3), 3 FFMA (accumulate); plus 1 MUFU rsqrt.  When every
# ion is singly charged the z_j product is skipped (it is exact), leaving 17.
FP32_OPS_PER_PAIR = 18


def ops_per_pair(species):
    return FP32_OPS_PER_PAIR - 1 if all(float(s.charge_e) == 1.0 for s in species) else FP32_OPS_PER_PAIR

FP32_LANES_PER_SM = 128
MUFU_PER_SM = 16
NOMINAL_SM_MHZ = 2070.0
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum, per timestep) of the step
# kernel from one ncu capture, keyed by a fingerprint of the CUDA sources the kernel is
# built from and by its launch shape (threads, ions per thread, packed, jsplit, fused); the
# bench reports it only while both still match, and null otherwise.
KERNEL_DRAM_TRAFFIC = {
    # row-persistent form, 28 ions per CTA: 505 856 B read + 1 792 B written over the second
    # 20-timestep launch of mix_n4096 (ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum)
    ("5161dcdda9021abe", (512, 1, 1, 28, 5)): 25382.4,
}
KERNEL_SOURCES = ("persistent.cu", "iontrap_internal.cuh")


def kernel_fingerprint():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1907_10514_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# timesteps per cooperative launch of the grid-persistent form (include/iontrap.h)
GP_STEPS_PER_LAUNCH = 1000


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def shard(items, rank: int, world: int):
    """The units (ensembles, requests) a rank advances: every world-th one from its
    rank -- independent problems, no collective on the data path."""
    return list(items)[rank::world]


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _gather(ws, obj):
    """Every rank's obj, on every rank (result reporting only; no data-path exchange)."""
    if ws == 1:
        return [obj]
    import torch.distributed as dist
    out = [None] * ws
    dist.all_gather_object(out, obj)
    return out


def _max_over_ranks(ws, x):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def cpu_oracle_rate(w, steps: int):
    """ion-steps/s of the FP64 oracle on this host (OpenMP, all cores)."""
    import oracle
    q, m, qm0 = oracle.ion_arrays(w.species, w.species_of_ion)
    p = oracle.params(w.trap, qm0)
    x, v, a = oracle.run(w.x0, w.v0, q, m, p, 0)
    t0 = time.perf_counter()
    oracle.run(x, v, q, m, p, steps, step0=0, a0=a)
    dt = time.perf_counter() - t0
    return w.n * steps / dt, oracle.threads(), dt


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return
    import iongen
    w = iongen.mix_n4096()
    per_step = args.ref_sample_steps
    for _ in range(args.warmup):
        cpu_oracle_rate(w, max(1, per_step // 4))
    rates, secs = [], []
    for _ in range(args.steps):
        r, cores, dt = cpu_oracle_rate(w, per_step)
        rates.append(r)
        secs.append(dt)
    value = statistics.median(rates)
    line = {
        "impl": "reference", "metric": "ion-steps/s", "value": value, "unit": "ion-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.median(secs), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "mix_n4096: 3072 Ca+ + 1024 NH3+, Gaussian 100 um, RF trap q=0.3 "
                               "a=-0.001, Langevin; FP64 oracle", "n_ions": w.n,
                   "timesteps_per_step": per_step, "l2": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": "ion-steps/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} timesteps of the N=4096 workload per bench step"},
        "e2e": {"value": value, "unit": "ion-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_gpu(args):
    import torch
    ws, rank = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.cuda.current_device()
    import iongen
    import paper_1907_10514_gb300 as it

    if args.only == "serve":  # the serving measurement alone (e.g. at full step budgets)
        with ClockSampler(dev) as clk:
            sv = serve_measurement(it, torch, args, rank, ws)
        if rank == 0:
            print(json.dumps({"leg": "serve", "n_gpus": ws, "serve": sv, "clocks": clk.summary()}))
        return

    w = iongen.mix_n4096()
    n = w.n
    nsteps = STEPS_PER_BENCH_STEP
    stream = torch.cuda.Stream()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.add_(1.0)

    params = it.make_params(w.trap, precision=it.IONTRAP_PREC_FP32)
    # per-rank replica (weak scaling: every rank advances its own copy of the workload)
    sim = it.Simulation(w.species, w.species_of_ion, w.x0, w.v0, params, stream=stream)
    if args.tune_us > 0:
        sim.autotune(trial_us=args.tune_us)  # the library's autotuner (state unchanged)
    cfg = sim.config()
    sim.step(200)
    sim.sync()
    for _ in range(args.warmup):
        flush_l2()
        sim.step(nsteps)
    sim.sync()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    _barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        torch.cuda.nvtx.range_push("timed")
        for k in range(args.steps):
            flush_l2()
            ev[k][0].record(stream)
            sim.step(nsteps)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        _barrier(ws)
    sim.sync()
    force_err = sampled_force_error(it, sim, w) if rank == 0 else None
    ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = _max_over_ranks(ws, sum(ms))
    ms_per_step = total_ms / args.steps
    value = ws * n * nsteps * args.steps / (total_ms / 1e3)
    pairs = n * (n - 1)
    kernel_us = ms_per_step * 1e3 / nsteps
    achieved_gpairs = pairs / (kernel_us * 1e-6) / 1e9
    opp = ops_per_pair(w.species)
    peak_gpairs = sms * NOMINAL_SM_MHZ * 1e6 * min(FP32_LANES_PER_SM / opp, MUFU_PER_SM) / 1e9
    sim.close()

    # e2e: through the C ABI with host buffers, H2D + D2H inside the timed region
    x_out = np.empty((3, n))
    v_out = np.empty((3, n))
    e2e_t = []
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = it.iontrap_create(w.species, w.species_of_ion, w.x0, w.v0, params, 0, stream)
        it.iontrap_step(h, nsteps)
        it.iontrap_state(h, n, x_out, v_out)
        t1 = time.perf_counter()
        it.iontrap_destroy(h)
        if k >= args.warmup:
            e2e_t.append(t1 - t0)
    e2e_s = _max_over_ranks(ws, sum(e2e_t))
    e2e_value = ws * n * nsteps * args.steps / e2e_s
    h2d = w.x0.nbytes + w.v0.nbytes + w.species_of_ion.nbytes + 8
    d2h = x_out.nbytes + v_out.nbytes + 8

    extra = {}
    if rank == 0 and not args.no_extra:
        extra = extra_measurements(it, torch, stream, sms, args)
        extra["plain_n64"] = plain_n64_measurement(it, torch, stream)
    # independent ensembles and requests: every rank advances its own shard, no collective
    # on the data path; rank 0 reports the aggregate over the slowest rank's time
    if not args.no_batched:
        b = _gather(ws, batched_measurement(it, torch, stream, rank, ws, tune_us=args.tune_us))
        if rank == 0:
            extra["batched_512"] = aggregate_batched(b)
    if not args.no_serve:
        sv = serve_measurement(it, torch, args, rank, ws)
        if rank == 0:
            extra["serve"] = sv
    if rank == 0:
        probe = {}
        for kind, name in ((0, "ffma"), (1, "ffma2"), (2, "mufu_rsqrt"), (3, "dfma"), (4, "fadd2"), (5, "cvt_f32_f64")):
            ops, mhz = it.iontrap_alu_probe(kind, 4000 if kind in (3, 5) else 20000)
            probe[name] = round(ops, 2)
        probe["sm_mhz"] = round(mhz)
        extra["alu_probe_lane_ops_per_clk_per_sm"] = probe

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        full = None
        if not args.no_extra:
            extra["oracle_timing"] = oracle_timing(args)
            full = extra["oracle_timing"].get("mix_n4096")
        if full:  # the oracle's full run of the workload, timed in oracle_timing
            cpu = {"value": full["ion_steps_per_s"], "unit": "ion-steps/s", "cores": extra["oracle_timing"]["cores"],
                   "kind": "oracle",
                   "sample": f"the full {full['timesteps']}-timestep run of the same N=4096 workload "
                             f"({full['seconds']:.1f} s, FP64 C/OpenMP)"}
        else:
            rate, cores, dt = cpu_oracle_rate(w, args.cpu_sample_steps)
            cpu = {"value": rate, "unit": "ion-steps/s", "cores": cores, "kind": "oracle",
                   "sample": f"{args.cpu_sample_steps} timesteps of the same N=4096 workload "
                             f"({dt:.1f} s, FP64 C/OpenMP)"}

    fp = kernel_fingerprint()
    traffic = KERNEL_DRAM_TRAFFIC.get((fp, tuple(cfg[:5])))
    # the same roof at the pipe rates the probe measured for this loop's packed mix
    # (opp - 5 FADD2/FMUL2 lane-ops at the FADD2 rate, 5 FFMA2 at the FFMA2 rate per pair)
    measured_roof = None
    pr = extra.get("alu_probe_lane_ops_per_clk_per_sm") if extra else None
    if pr and pr.get("fadd2") and pr.get("ffma2"):
        lanes = opp / ((opp - 5) / pr["fadd2"] + 5 / pr["ffma2"])
        measured_roof = sms * NOMINAL_SM_MHZ * 1e6 * lanes / opp / 1e9
    peaks = _peaks()
    line = {
        "metric": "ion-steps/s", "value": value, "unit": "ion-steps/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "mix_n4096: 3072 Ca+ + 1024 NH3+, Gaussian 100 um, 10 mK, RF trap "
                               "q=0.3 a=-0.001 f_z=0.2 MHz, Langevin 1e5/s 1 mK, dt=T_RF/20, "
                               "FP32 pairs + Kahan, FP64 state",
                   "n_ions": n, "timesteps_per_step": nsteps, "tile": list(cfg),
                   "tile_fields": "threads, ions_per_thread, packed, jsplit, fused, pdl, graph (autotuned)",
                   "l2": "flushed (256 MB write) between timed steps; state is L2-resident within a step"},
        "pair_interactions_per_s": value * (n - 1),
        "unordered_pairs_per_s": value * (n - 1) / 2,
        "pairs_note": "pair_interactions_per_s counts ordered pairs N(N-1) per timestep, as the kernels evaluate "
                      "them; the method itself needs the N(N-1)/2 unordered pairs (unordered_pairs_per_s)",
        "force_rel_rms_vs_oracle": force_err,
        "error_note": "GPU Coulomb accelerations vs the FP64 oracle on 256 sampled ions of the final state "
                      "(bar 1e-5); trajectories: tests/test_gpu_parity.py",
        "e2e": {"value": e2e_value, "unit": "ion-steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps * (-(-nsteps // GP_STEPS_PER_LAUNCH) if cfg[4] >= 4 else nsteps),
        "roofline": {"bound": "alu", "achieved": achieved_gpairs, "peak": peak_gpairs,
                     "unit": "Gpair/s", "frac": achieved_gpairs / peak_gpairs,
                     "traffic": traffic,
                     "traffic_unit": "DRAM bytes per timestep (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                     "traffic_source": (f"ncu capture (20-timestep launch) of kernel sources {fp} at this launch shape"
                                        if traffic is not None
                                        else f"no ncu capture of kernel sources {fp} at launch shape {list(cfg[:5])}"),
                     "basis": f"{sms} SMs x {NOMINAL_SM_MHZ:.0f} MHz x {FP32_LANES_PER_SM} FP32 lanes / "
                              f"{opp} FP32 instr per ordered pair (MUFU roof "
                              f"{MUFU_PER_SM}/clk/SM not binding); achieved = N(N-1) per timestep / "
                              "mean time per timestep over the timed region",
                     "peak_source": "derived from SM count, nominal max SM clock and FP32 lane count",
                     "peak_at_measured_pipe_rates": measured_roof,
                     "frac_of_measured_pipe_rates": (achieved_gpairs / measured_roof) if measured_roof else None,
                     "measured_pipe_rates_basis": "the loop's packed mix (FADD2/FMUL2 and 5 FFMA2 per pair) at the "
                                                  "lane rates iontrap_alu_probe measured in this run",
                     "hbm_peak_gbs_measured": peaks.get("hbm_gbs")},
        "clocks": clk.summary(),
    }
    if cpu:
        line["cpu_baseline"] = cpu
    if extra:
        line["extra"] = extra
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def extra_measurements(it, torch, stream, sms, args):
    """Plain FP64 form on the same workload; the N = 32768 crystal in the FP32 form."""
    import iongen
    out = {}
    w = iongen.mix_n4096()
    n = w.n
    p64 = it.make_params(w.trap, precision=it.IONTRAP_PREC_FP64)
    with it.Simulation(w.species, w.species_of_ion, w.x0, w.v0, p64, stream=stream) as s:
        s.step(5)
        s.sync()
        k = args.fp64_steps
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(k)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        err64 = sampled_force_error(it, s, w)
    out["fp64_form_mix_n4096"] = {"ion_steps_per_s": n * k / (ms / 1e3),
                                  "pair_interactions_per_s": n * (n - 1) * k / (ms / 1e3),
                                  "us_per_timestep": 1e3 * ms / k, "timesteps": k,
                                  "force_rel_rms_vs_oracle": err64,
                                  "error_sample": "256 ions of the final state"}
    # the same workload with species-selective cooling (Sec. 3): Ca+ laser-cooled along x on
    # top of its bath, NH3+ in a bath of its own; forces changed through iontrap_set_params
    pc = it.make_params(w.trap, precision=it.IONTRAP_PREC_FP32)
    cool = [(w.trap.gamma, w.trap.T_bath, (1e5, 0.0, 0.0)), (2e5, 2e-3, (0.0, 0.0, 0.0))]
    with it.Simulation(w.species, w.species_of_ion, w.x0, w.v0, pc, stream=stream) as s:
        s.set_params(pc, cool)
        s.step(100)
        s.sync()
        k = 1000
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(k)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        out["mix_n4096_species_cooling"] = {"ion_steps_per_s": n * k / (ms / 1e3), "us_per_timestep": 1e3 * ms / k,
                                            "timesteps": k, "tile": list(s.config()),
                                            "cooling": "Ca+: bath 1e5/s 1 mK + laser (1e5, 0, 0)/s; NH3+: bath 2e5/s 2 mK",
                                            "force_rel_rms_vs_oracle": sampled_force_error(it, s, w),
                                            "error_sample": "256 ions of the final state"}
    # the same workload recording x and the secular velocity (average over one RF period)
    # every RF period into a device buffer (dump + timeAvg, Sec. 3 "Writing/reading data")
    with it.Simulation(w.species, w.species_of_ion, w.x0, w.v0, pc, stream=stream) as s:
        k = 1000
        fields = it.IONTRAP_REC_X | it.IONTRAP_REC_VAVG
        buf = torch.empty((k // 20) * 2 * 3 * n, dtype=torch.float64, device="cuda")
        s.step(100)
        s.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step_record(k, 20, fields, 20, buf.data_ptr())
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        xs = s.state()[0]
        rec_last = buf.view(k // 20, 2, 3, n)[-1, 0].cpu().numpy()
        out["mix_n4096_record_every_rf_period"] = {"ion_steps_per_s": n * k / (ms / 1e3), "us_per_timestep": 1e3 * ms / k,
                                                   "timesteps": k, "records": k // 20,
                                                   "fields": "x and the velocity averaged over 20 steps",
                                                   "last_record_equals_state": bool(np.array_equal(rec_last, xs)),
                                                   "force_rel_rms_vs_oracle": sampled_force_error(it, s, w),
                                                   "error_sample": "256 ions of the final state"}
    out.update(modes_measurements(it, stream))
    wc = iongen.crystal_n32768()
    nc = wc.n
    pc = it.make_params(wc.trap, precision=it.IONTRAP_PREC_FP32)
    with it.Simulation(wc.species, wc.species_of_ion, wc.x0, wc.v0, pc, stream=stream) as s:
        s.autotune(trial_us=args.tune_us * 4)
        s.step(10)
        s.sync()
        k = 1000
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(k)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        cfg = s.config()
    with it.Simulation(wc.species, wc.species_of_ion, wc.x0, wc.v0, pc, stream=stream) as s:
        errs, done = [], 0
        for mark in (0, 142, 285, 428, 571, 714, 857, 999):
            s.step(mark - done)
            done = mark
            errs.append(sampled_force_error(it, s, wc, k=256, seed=mark))
    us = 1e3 * ms / k
    gp = nc * (nc - 1) / (us * 1e-6) / 1e9
    peak = sms * NOMINAL_SM_MHZ * 1e6 * FP32_LANES_PER_SM / ops_per_pair(wc.species) / 1e9
    out["crystal_n32768"] = {"ion_steps_per_s": nc * k / (ms / 1e3),
                             "pair_interactions_per_s": nc * (nc - 1) * k / (ms / 1e3),
                             "us_per_timestep": us, "timesteps": k, "tile": list(cfg),
                             "roofline_frac": gp / peak, "achieved_gpair_s": gp, "peak_gpair_s": peak,
                             "force_rel_rms_vs_oracle_max": max(errs),
                             "error_sample": "256 ions at steps 0, 142, ..., 999 of a 1000-step run"}
    return out


def modes_measurements(it, stream):
    """The minimiser on a 1024-ion Ca+ crystal in a pseudopotential trap (Sec. 3
    "Minimisation") and the device Hessian of a 2048-ion crystal (Sec. 5 "Normal modes")."""
    import iongen
    out = {}
    n = 1024
    w0 = 2 * math.pi * 0.3e6
    freqs = [(1.2 * w0, 1.3 * w0, w0)]
    trap = iongen.Trap(Omega=iongen.OMEGA_RF, a=0.0, q=0.3, omega_z=2 * math.pi * 0.2e6, gamma=0.0, T_bath=0.0,
                       dt=iongen.rf_period_dt(iongen.OMEGA_RF), seed=5)
    x0 = iongen.gaussian_positions(n, 60e-6, seed=5)
    sp = np.zeros(n, np.uint8)
    e, eps0, amu = 1.602176634e-19, 8.8541878128e-12, 1.66053906660e-27
    m = iongen.CA40.mass_amu * amu
    l = (e * e / (4 * math.pi * eps0 * m * w0 ** 2)) ** (1 / 3)
    fscale = m * w0 ** 2 * l
    p = it.make_params(trap, flags=it.IONTRAP_PSEUDO)
    with it.Simulation([iongen.CA40], sp, x0, None, p, stream=stream) as s:
        s.set_pseudo_frequencies(freqs)
        t0 = time.perf_counter()
        iters, fn = s.minimize(20000, 0.05 * l, 1e-4 * fscale * math.sqrt(n), dt=5 * trap.dt)
        wall = time.perf_counter() - t0
    out["minimize_crystal_n1024"] = {"iterations": iters, "seconds": wall, "us_per_iteration": 1e6 * wall / max(iters, 1),
                                     "force_norm_over_scale": fn / fscale,
                                     "note": "FP32 pair kernel + 3 reduction/update kernels per iteration, "
                                             "host check every 64 iterations"}
    nh = 2048
    xh = iongen.gaussian_positions(nh, 80e-6, seed=6)
    with it.Simulation([iongen.CA40], np.zeros(nh, np.uint8), xh, None, p, stream=stream) as s:
        s.hessian()
        t0 = time.perf_counter()
        H = s.hessian()
        wall = time.perf_counter() - t0
    import oracle
    q, mm, qm0 = oracle.ion_arrays([iongen.CA40], np.zeros(nh, np.uint8))
    Ho = oracle.hessian(xh, q, mm, oracle.params(trap, qm0, oracle.PSEUDO))
    out["hessian_n2048"] = {"seconds": wall, "bytes": 9 * nh * nh * 8,
                            "max_abs_dev_over_max_abs_vs_oracle": float(np.abs(H - Ho).max() / np.abs(Ho).max()),
                            "note": "FP64 device kernels + device-to-host copy of the 3n x 3n matrix"}
    del H, Ho
    return out


def sampled_force_error(it, sim, w, k=256, seed=0):
    """Relative RMS of the GPU Coulomb accelerations at the current state against the FP64
    oracle on k sampled ions (the oracle evaluates those ions' sums exactly)."""
    import oracle
    f = sim.forces()
    x = sim.state()[0]
    q, m, _ = oracle.ion_arrays(w.species, w.species_of_ion)
    idx = np.random.default_rng(seed).choice(w.n, min(k, w.n), replace=False)
    ref = oracle.coulomb_accel(x, q, m, idx=idx)
    return float(np.sqrt(((f[:, idx] - ref) ** 2).sum() / (ref ** 2).sum()))


def batched_measurement(it, torch, stream, rank=0, world=1, steps=2000, tune_us=0.0):
    """This rank's shard of the 512 independent Ca+ ensembles (N log-uniform in [16, 2048])
    advanced together by iontrap_step_many (batched resident kernels), 2000 steps."""
    import iongen
    stable = lambda species, trap: it.iontrap_stable(species, it.make_params(trap))
    every = iongen.batched_512(stable=stable, steps=steps)
    ws = [every[k] for k in shard(range(len(every)), rank, world)]
    sims = [it.Simulation(w.species, w.species_of_ion, w.x0, w.v0, it.make_params(w.trap), stream=stream)
            for w in ws]
    try:
        hs = [s.handle for s in sims]
        tuned = {}
        if tune_us > 0:  # the batched launch's autotuner: group shapes per N bucket (states unchanged)
            it.iontrap_autotune_many(hs, trial_us=tune_us)
            tuned = {e["log2n"]: {"ctas_per_group": e["splits"], "parts": e["ions_per_thread"] or "cost model",
                                  "us_per_step_of_the_batch": round(e["us_per_step"], 2)}
                     for e in it.iontrap_tuning_get() if e["precision"] == it.IONTRAP_TUNE_BATCHED}
        it.iontrap_step_many(hs, [100] * len(hs))  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it.iontrap_step_many(hs, [steps] * len(hs))
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        pick = np.random.default_rng(7 + rank).choice(len(ws), min(8, len(ws)), replace=False)
        errs = [sampled_force_error(it, sims[k], ws[k], k=64, seed=int(k)) for k in pick]
    finally:
        for s in sims:
            s.close()
    return {"ensembles": len(ws), "ions": sum(w.n for w in ws), "pairs": sum(w.n * (w.n - 1) for w in ws),
            "ms": ms, "steps": steps, "errs": errs, "redraws": sum(w.redraws for w in ws), "tuned": tuned}


def aggregate_batched(parts):
    ms = max(p["ms"] for p in parts)
    steps = parts[0]["steps"]
    ions = sum(p["ions"] for p in parts)
    pairs = sum(p["pairs"] for p in parts)
    return {"ensembles": sum(p["ensembles"] for p in parts), "ions": ions, "timesteps": steps, "ms": ms,
            "ranks": len(parts), "ms_per_rank": [p["ms"] for p in parts],
            "force_rel_rms_vs_oracle_max": max(max(p["errs"]) for p in parts if p["errs"]),
            "error_sample": "8 ensembles per rank, 64 ions each, after the run",
            "ion_steps_per_s": ions * steps / (ms / 1e3), "pair_interactions_per_s": pairs * steps / (ms / 1e3),
            "unstable_trap_redraws": sum(p["redraws"] for p in parts),
            "tuned_group_shapes_by_log2n": parts[0]["tuned"],
            "launches_per_rank": 2 * ((steps + 999) // 1000)}


def _serve_run(it, torch, work, arrivals, budget_bytes, keep=(), chunk_steps=100, max_parallel=0):
    """Submit each request at its arrival time (s after the start) to a fresh serving
    loop and poll it; returns (latencies s, wall s, {index: final x} for ``keep``)."""
    srv = it.iontrap_server_create(mem_budget_bytes=budget_bytes, max_resident=4096, chunk_steps=chunk_steps,
                                   max_parallel=max_parallel)
    lat = [None] * len(work)
    kept, index, ns = {}, {}, {}
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k, pending = 0, len(work)
        while pending:
            now = time.perf_counter() - t0
            while k < len(work) and arrivals[k] <= now:
                w = work[k]
                rid = it.iontrap_server_submit(srv, w.species, w.species_of_ion, w.x0, w.v0, it.make_params(w.trap),
                                               w.steps)
                index[rid], ns[rid] = k, w.n
                k += 1
            done = it.iontrap_server_poll(srv)
            for rid in done:
                i = index[rid]
                lat[i] = time.perf_counter() - t0 - arrivals[i]
                x, _, step, status = it.iontrap_server_result(srv, rid, ns[rid])
                if i in keep:
                    kept[i] = (x, step, status)
                pending -= 1
            if not done:
                time.sleep(0.0002)
        wall = time.perf_counter() - t0
    finally:
        it.iontrap_server_destroy(srv)
    return lat, wall, kept


def _fifo_fp64(it, torch, work, arrivals, cap_s, chunk=200):
    """The plain FP64 form, one simulation at a time in arrival order, each started no
    earlier than its arrival and stepped in chunks of 200 steps; the run stops at the
    first chunk boundary after cap_s of wall time (the request in progress is not served).
    Returns the latencies of the served requests (None for the others) and the wall time."""
    lat = [None] * len(work)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k, w in enumerate(work):
        now = time.perf_counter() - t0
        if now > cap_s or arrivals[k] > cap_s:
            break
        if arrivals[k] > now:
            time.sleep(arrivals[k] - now)
        h = it.iontrap_create(w.species, w.species_of_ion, w.x0, w.v0,
                              it.make_params(w.trap, precision=it.IONTRAP_PREC_FP64))
        try:
            done = 0
            while done < w.steps and time.perf_counter() - t0 <= cap_s:
                it.iontrap_step(h, min(chunk, w.steps - done))
                it.iontrap_sync(h)
                done += min(chunk, w.steps - done)
            if done == w.steps:
                it.iontrap_state(h, w.n)
                lat[k] = time.perf_counter() - t0 - arrivals[k]
        finally:
            it.iontrap_destroy(h)
        if lat[k] is None:
            break
    return lat, time.perf_counter() - t0


def _pct(lat_s):
    """p50 and p99 of latencies given in seconds, in ms."""
    v = np.array(lat_s, dtype=np.float64) * 1e3
    return {"p50_ms": float(np.percentile(v, 50)), "p99_ms": float(np.percentile(v, 99))}


def serve_measurement(it, torch, args, rank=0, world=1):
    """The request stream (Poisson 200/s, N log-uniform in [8, 65536], step budgets
    log-uniform in [1e3, 1e5], Ca+ or 80/20 Ca+/NH3+): its first K requests, each step
    budget divided by step_scale, through the continuous-batching server -- at their
    generated arrival times (offered load far above one GPU's capacity), and again with the
    arrivals stretched to 0.7 of the measured capacity -- and the plain FP64 form serving
    the same K one at a time (FIFO).  Latency = completion - arrival.  With several ranks
    each rank serves its shard of the K requests on its own GPU."""
    import iongen
    import oracle
    stable = lambda species, trap: it.iontrap_stable(species, it.make_params(trap))
    full = iongen.serve_stream(stable=stable)
    full_pairs = sum(r.n * r.n * r.steps for r in full)
    K, scale = args.serve_requests, args.serve_step_scale
    reqs = full[:K]
    for r in reqs:
        r.steps = max(1, int(round(r.steps / scale)))
    mine = shard(range(K), rank, world)
    work = [iongen.request_workload(reqs[k]) for k in mine]
    arrivals = [reqs[k].arrival_s for k in mine]
    pairs_of = [w.n * (w.n - 1) * w.steps for w in work]
    budget = args.serve_budget_mb << 20
    # sampled results whose error against the oracle is stated (their final state's forces)
    keep = set(np.random.default_rng(11).choice(len(work), min(6, len(work)), replace=False).tolist())
    lat, wall, kept = _serve_run(it, torch, work, arrivals, budget, keep, args.serve_chunk_steps, args.serve_parallel)
    cap_mine = sum(pairs_of) / wall
    # the companion run: the same requests, arrivals stretched so that the offered load is
    # 0.7 of the capacity the first run sustained
    span = max(arrivals) if arrivals else 0.0
    stretch = (sum(pairs_of) / (0.7 * cap_mine)) / span if span > 0 else 1.0
    arr07 = [a * stretch for a in arrivals]
    lat07, wall07, _ = _serve_run(it, torch, work, arr07, budget, (), args.serve_chunk_steps, args.serve_parallel)
    lat64, wall64 = _fifo_fp64(it, torch, work, arrivals, args.serve_fp64_cap_s)
    errs = []
    for i, (x, step, status) in sorted(kept.items()):
        w = work[i]
        if status != 0 or step != w.steps:
            errs.append({"request": mine[i], "n": w.n, "status": status})
            continue
        q, m, _ = oracle.ion_arrays(w.species, w.species_of_ion)
        with it.Simulation(w.species, w.species_of_ion, x, None, it.make_params(w.trap)) as s:
            f = s.forces()
        idx = np.random.default_rng(i).choice(w.n, min(128, w.n), replace=False)
        ref = oracle.coulomb_accel(x, q, m, idx=idx)
        err = float(np.sqrt(((f[:, idx] - ref) ** 2).sum() / max((ref ** 2).sum(), 1e-300))) if w.n > 1 else 0.0
        errs.append({"request": mine[i], "n": w.n, "steps": w.steps, "force_rel_rms_vs_oracle": err})
    mine_out = {"ns": [w.n for w in work], "lat": lat, "wall": wall, "lat07": lat07, "wall07": wall07, "arr07": arr07,
                "lat64": lat64,
                "wall64": wall64, "arrivals": arrivals, "pairs": sum(pairs_of),
                "ion_steps": sum(w.n * w.steps for w in work), "errs": errs,
                "redraws": sum(reqs[k].redraws for k in mine), "n": len(work)}
    parts = _gather(world, mine_out)
    if rank != 0:
        return None
    meta = {"requests": K, "step_scale": scale, "mem_budget_bytes": budget, "full_stream_requests": len(full),
            "full_stream_offered_pairs_per_s": full_pairs / full[-1].arrival_s, "arrival_span_s": reqs[-1].arrival_s,
            "fp64_cap_s": args.serve_fp64_cap_s, "chunk_steps": args.serve_chunk_steps,
            "max_parallel": args.serve_parallel or 3}
    return aggregate_serve(parts, meta)


def aggregate_serve(parts, meta):
    """Rank 0's summary of the serving measurement from every rank's record."""
    cat = lambda key: [x for p in parts for x in p[key]]
    pairs = sum(p["pairs"] for p in parts)
    ion_steps = sum(p["ion_steps"] for p in parts)
    wall = max(p["wall"] for p in parts)
    primary = {"wall_s": wall, "arrival_span_s": meta["arrival_span_s"],
               "offered_pairs_per_s": pairs / meta["arrival_span_s"],
               "pair_interactions_per_s": pairs / wall, "ion_steps_per_s": ion_steps / wall}
    primary.update(_pct(cat("lat")))
    wall07 = max(p["wall07"] for p in parts)
    span07 = max(max(p["arr07"]) for p in parts if p["arr07"])
    comp = {"wall_s": wall07, "arrival_span_s": span07, "offered_pairs_per_s": pairs / span07,
            "pair_interactions_per_s": pairs / wall07, "ion_steps_per_s": ion_steps / wall07}
    comp.update(_pct(cat("lat07")))
    # the same percentiles by request size: batched small, batched large, single-simulation
    ns = cat("ns") if all("ns" in p for p in parts) else None
    if ns:
        for name, lo, hi in (("n_le_256", 1, 256), ("n_257_2048", 257, 2048), ("n_gt_2048", 2049, 1 << 40)):
            for run, key in ((primary, "lat"), (comp, "lat07")):
                sel = [l for l, n in zip(cat(key), ns) if lo <= n <= hi]
                if sel:
                    run.setdefault("by_size", {})[name] = dict(_pct(sel), requests=len(sel))
    # the FP64 FIFO: a request not started within the cap counts as waiting until its
    # rank's run ended, so its percentiles are then lower bounds
    lat64 = [(l if l is not None else p["wall64"] - p["arrivals"][k])
             for p in parts for k, l in enumerate(p["lat64"])]
    served = sum(1 for p in parts for l in p["lat64"] if l is not None)
    fifo = {"wall_s": max(p["wall64"] for p in parts), "cap_s": meta["fp64_cap_s"],
            "note": "plain FP64 form, one simulation at a time in arrival order (same requests, same arrival times); "
                    "requests not started within the cap count as waiting until the end of the run (lower bounds)"}
    fifo.update(_pct(lat64))
    fifo["served"], fifo["not_served"] = served, len(lat64) - served
    fifo["percentiles_are_lower_bounds"] = served < len(lat64)
    return {"requests": meta["requests"], "ranks": len(parts), "requests_per_rank": [p["n"] for p in parts],
            "step_scale": meta["step_scale"],
            "step_budgets": f"the stream's budgets (1e3 .. 1e5) divided by {meta['step_scale']:g}",
            "mem_budget_bytes": meta["mem_budget_bytes"], "chunk_steps": meta.get("chunk_steps"),
            "max_parallel": meta.get("max_parallel"),
            "full_stream_requests": meta["full_stream_requests"],
            "full_stream_offered_pairs_per_s": meta["full_stream_offered_pairs_per_s"],
            "unstable_trap_redraws": sum(p["redraws"] for p in parts),
            "at_generated_arrivals": primary, "at_0.7_capacity": comp, "fp64_fifo_same_requests": fifo,
            "per_result_error": cat("errs"),
            "error_note": "relative RMS of the FP32 pair accelerations at each sampled result's final state "
                          "against the FP64 oracle (128 sampled ions); served results are bitwise equal alone "
                          "and in the mix (tests)"}


def plain_n64_measurement(it, torch, stream):
    """The plain method's workload: N = 64 Ca+ in the RF trap, 10 000 steps, in the plain
    FP64 form, and the FP32 form beside it; errors against the oracle at step 100 and at
    the end of the run."""
    import iongen
    import oracle
    w = iongen.plain_n64()
    q, m, qm0 = oracle.ion_arrays(w.species, w.species_of_ion)
    p = oracle.params(w.trap, qm0)
    x100, _, _ = oracle.run(w.x0, w.v0, q, m, p, 100)
    out = {"n_ions": w.n, "timesteps": w.steps}
    for name, prec in (("fp64_form", it.IONTRAP_PREC_FP64), ("fp32_form", it.IONTRAP_PREC_FP32)):
        pr = it.make_params(w.trap, precision=prec)
        with it.Simulation(w.species, w.species_of_ion, w.x0, w.v0, pr, stream=stream) as s:
            s.step(100)
            x, _, _, _ = s.state()
            traj = float(np.sqrt(((x - x100) ** 2).sum() / (x100 ** 2).sum()))
            s.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(w.steps)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            ferr = sampled_force_error(it, s, w, k=64)
            cfg = list(s.config())
        out[name] = {"us_per_timestep": 1e3 * ms / w.steps, "ion_steps_per_s": w.n * w.steps / (ms / 1e3),
                     "tile": cfg, "trajectory_rel_rms_vs_oracle_step100": traj,
                     "force_rel_rms_vs_oracle_final": ferr}
    return out


def oracle_timing(args):
    """The FP64 oracle on this host's cores: the plain N = 64 run and the N = 4096 run in
    full, and for the N = 32768 crystal 8 force evaluations plus a 10-step run."""
    import iongen
    import oracle
    out = {"cores": oracle.threads(), "cpu_model": None}
    try:
        lines = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout.splitlines()
        out["cpu_model"] = next(l.split(":", 1)[1].strip() for l in lines if l.startswith("Model name"))
    except Exception:
        try:
            out["cpu_model"] = next(l.split(":", 1)[1].strip() for l in open("/proc/cpuinfo")
                                    if l.lower().startswith(("model name", "cpu part")))
        except Exception:
            pass
    for name, gen in (("plain_n64", iongen.plain_n64), ("mix_n4096", iongen.mix_n4096)):
        w = gen()
        q, m, qm0 = oracle.ion_arrays(w.species, w.species_of_ion)
        p = oracle.params(w.trap, qm0)
        t0 = time.perf_counter()
        oracle.run(w.x0, w.v0, q, m, p, w.steps)
        dt = time.perf_counter() - t0
        out[name] = {"timesteps": w.steps, "seconds": dt, "ion_steps_per_s": w.n * w.steps / dt}
    w = iongen.crystal_n32768()
    q, m, qm0 = oracle.ion_arrays(w.species, w.species_of_ion)
    p = oracle.params(w.trap, qm0)
    t0 = time.perf_counter()
    for _ in range(8):
        oracle.coulomb_accel(w.x0, q, m)
    t_f = (time.perf_counter() - t0) / 8
    t0 = time.perf_counter()
    oracle.run(w.x0, w.v0, q, m, p, 10)
    t_r = (time.perf_counter() - t0) / 10
    out["crystal_n32768"] = {"force_evaluation_s": t_f, "seconds_per_timestep_10_step_run": t_r,
                             "ion_steps_per_s": w.n / t_r}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sample-steps", type=int, default=3000)
    ap.add_argument("--ref-sample-steps", type=int, default=100)
    ap.add_argument("--fp64-steps", type=int, default=50)
    ap.add_argument("--serve-requests", type=int, default=100)
    ap.add_argument("--tune-us", type=float, default=3000.0)
    ap.add_argument("--serve-step-scale", type=float, default=20.0)
    ap.add_argument("--serve-budget-mb", type=int, default=2048)
    ap.add_argument("--serve-fp64-cap-s", type=float, default=20.0)
    ap.add_argument("--serve-chunk-steps", type=int, default=100)
    ap.add_argument("--serve-parallel", type=int, default=0,
                    help="shared streams of the served requests the batched kernel does not take (0: 3)")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--only", choices=["serve"], default=None,
                    help="run one measurement leg alone and print its JSON (not the bench line)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
