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
# DRAM bytes (read + write) per timestep of the step kernel, from the ncu captures
# summarised in profiles/; valid only for that launch configuration.
PROFILED_TRAFFIC = {
    # one launch per timestep (profiles/step_f32_cw_mix_n4096.md)
    (128, 2, 1, 512, 3): (485376 + 0, "DRAM bytes per timestep launch (ncu, profiles/step_f32_cw_mix_n4096.md)"),
    # row-persistent form: its last capture (25.3 KB of DRAM traffic per timestep, 27 or 32
    # ions per CTA) predates a prologue proxy fence added since, so no figure is claimed
}
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
    if rank == 0 and not args.no_batched:
        extra["batched_512"] = batched_measurement(it, torch, stream)
    if rank == 0 and not args.no_serve:
        extra["serve"] = serve_measurement(it, torch, args.serve_requests, args.serve_step_scale,
                                           args.serve_budget_mb << 20, args.serve_fp64_subset)
    if rank == 0:
        probe = {}
        for kind, name in ((0, "ffma"), (1, "ffma2"), (2, "mufu_rsqrt"), (3, "dfma")):
            ops, mhz = it.iontrap_alu_probe(kind, 4000 if kind == 3 else 20000)
            probe[name] = round(ops, 2)
        probe["sm_mhz"] = round(mhz)
        extra["alu_probe_lane_ops_per_clk_per_sm"] = probe

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        rate, cores, dt = cpu_oracle_rate(w, args.cpu_sample_steps)
        cpu = {"value": rate, "unit": "ion-steps/s", "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_sample_steps} timesteps of the same N=4096 workload "
                         f"({dt:.1f} s, FP64 C/OpenMP)"}

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
                     "traffic": PROFILED_TRAFFIC.get(tuple(cfg[:5]), (None, None))[0],
                     "traffic_unit": PROFILED_TRAFFIC.get(tuple(cfg[:5]), (None, "not profiled for this tile"))[1],
                     "basis": f"{sms} SMs x {NOMINAL_SM_MHZ:.0f} MHz x {FP32_LANES_PER_SM} FP32 lanes / "
                              f"{opp} FP32 instr per ordered pair (MUFU roof "
                              f"{MUFU_PER_SM}/clk/SM not binding); achieved = N(N-1) per timestep / "
                              "mean time per timestep over the timed region",
                     "peak_source": "derived from SM count, nominal max SM clock and FP32 lane count",
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
    out["fp64_form_mix_n4096"] = {"ion_steps_per_s": n * k / (ms / 1e3),
                                  "pair_interactions_per_s": n * (n - 1) * k / (ms / 1e3),
                                  "us_per_timestep": 1e3 * ms / k, "timesteps": k}
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
                                            "cooling": "Ca+: bath 1e5/s 1 mK + laser (1e5, 0, 0)/s; NH3+: bath 2e5/s 2 mK"}
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
        out["mix_n4096_record_every_rf_period"] = {"ion_steps_per_s": n * k / (ms / 1e3), "us_per_timestep": 1e3 * ms / k,
                                                   "timesteps": k, "records": k // 20,
                                                   "fields": "x and the velocity averaged over 20 steps"}
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
        s.hessian()
        wall = time.perf_counter() - t0
    out["hessian_n2048"] = {"seconds": wall, "bytes": 9 * nh * nh * 8,
                            "note": "FP64 device kernels + device-to-host copy of the 3n x 3n matrix"}
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


def batched_measurement(it, torch, stream, steps=2000):
    """512 independent Ca+ ensembles (N log-uniform in [16, 2048]) advanced together by
    iontrap_step_many (batched resident kernel), 2000 steps."""
    import iongen
    stable = lambda species, trap: it.iontrap_stable(species, it.make_params(trap))
    ws = iongen.batched_512(stable=stable, steps=steps)
    sims = [it.Simulation(w.species, w.species_of_ion, w.x0, w.v0, it.make_params(w.trap), stream=stream)
            for w in ws]
    try:
        hs = [s.handle for s in sims]
        it.iontrap_step_many(hs, [100] * len(hs))  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it.iontrap_step_many(hs, [steps] * len(hs))
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        pick = np.random.default_rng(7).choice(len(ws), 8, replace=False)
        errs = [sampled_force_error(it, sims[k], ws[k], k=64, seed=int(k)) for k in pick]
    finally:
        for s in sims:
            s.close()
    ions = sum(w.n for w in ws)
    pairs = sum(w.n * (w.n - 1) for w in ws)
    return {"ensembles": len(ws), "ions": ions, "timesteps": steps, "ms": ms,
            "force_rel_rms_vs_oracle_max": max(errs), "error_sample": "8 ensembles, 64 ions each, after the run",
            "ion_steps_per_s": ions * steps / (ms / 1e3), "pair_interactions_per_s": pairs * steps / (ms / 1e3),
            "launches": 2 * ((steps + 999) // 1000)}


def serve_measurement(it, torch, count, step_scale, budget_bytes, fp64_subset):
    """The request stream (Poisson 200/s, N log-uniform in [8, 65536], Ca+ or 80/20
    Ca+/NH3+) with step budgets divided by step_scale, submitted at their arrival times
    to the continuous-batching server; latency = completion - arrival."""
    import iongen
    stable = lambda species, trap: it.iontrap_stable(species, it.make_params(trap))
    full = iongen.serve_stream(stable=stable)
    full_pairs = sum(r.n * r.n * r.steps for r in full)
    offered_full = full_pairs / full[-1].arrival_s
    reqs = full[:count]
    for r in reqs:
        r.steps = max(1, int(round(r.steps / step_scale)))
    work = [(iongen.request_workload(r), r) for r in reqs]
    srv = it.iontrap_server_create(mem_budget_bytes=budget_bytes, max_resident=4096, chunk_steps=100)
    lat, arrival, ids = [], {}, {}
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k = 0
        pending = len(work)
        while pending:
            now = time.perf_counter() - t0
            while k < len(work) and work[k][1].arrival_s <= now:
                w, r = work[k]
                rid = it.iontrap_server_submit(srv, w.species, w.species_of_ion, w.x0, w.v0, it.make_params(w.trap),
                                               r.steps)
                arrival[rid] = r.arrival_s
                ids[rid] = w.n
                k += 1
            for rid in it.iontrap_server_poll(srv):
                lat.append(time.perf_counter() - t0 - arrival[rid])
                it.iontrap_server_result(srv, rid, ids[rid])
                pending -= 1
            time.sleep(0.0002)
        wall = time.perf_counter() - t0
    finally:
        it.iontrap_server_destroy(srv)
    ion_steps = sum(r.n * r.steps for r in reqs)
    pairs = sum(r.n * (r.n - 1) * r.steps for r in reqs)
    lat_ms = np.array(lat) * 1e3
    out = {"requests": len(reqs), "step_scale": step_scale, "arrival_span_s": reqs[-1].arrival_s, "wall_s": wall,
           "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
           "ion_steps_per_s": ion_steps / wall, "pair_interactions_per_s": pairs / wall,
           "offered_pairs_per_s": pairs / reqs[-1].arrival_s, "mem_budget_bytes": budget_bytes,
           "full_stream_offered_pairs_per_s": offered_full, "full_stream_requests": len(full)}
    # baseline: the plain FP64 form, one simulation at a time in arrival order (subset)
    t = 0.0
    sub = work[:fp64_subset]
    for w, r in sub:
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        h = it.iontrap_create(w.species, w.species_of_ion, w.x0, w.v0,
                              it.make_params(w.trap, precision=it.IONTRAP_PREC_FP64))
        it.iontrap_step(h, r.steps)
        it.iontrap_state(h, w.n)
        t += time.perf_counter() - t1
        it.iontrap_destroy(h)
    sub_ion_steps = sum(r.n * r.steps for _, r in sub)
    ours_sub = sum(r.n * r.steps for _, r in sub)
    out["fp64_fifo_baseline"] = {"requests": len(sub), "ion_steps_per_s": sub_ion_steps / t, "seconds": t,
                                 "note": "plain FP64 form, one simulation at a time, first requests of the stream"}
    del ours_sub
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sample-steps", type=int, default=200)
    ap.add_argument("--ref-sample-steps", type=int, default=100)
    ap.add_argument("--fp64-steps", type=int, default=50)
    ap.add_argument("--serve-requests", type=int, default=800)
    ap.add_argument("--tune-us", type=float, default=3000.0)
    ap.add_argument("--serve-step-scale", type=float, default=1000.0)
    ap.add_argument("--serve-budget-mb", type=int, default=2048)
    ap.add_argument("--serve-fp64-subset", type=int, default=20)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
