"""Benchmark: PT-TTS hardness evaluation inside the RAO loop on GB300.

Workload (one instance per GPU): Chimera C_8 (N = 512, 1472 couplers), J
uniform on {+-1, +-2, +-3}, 32 temperatures geometric in beta [0.1, 4], 64
independent PT runs, TTS horizon S = 2^16 sweeps with the target taken from a
4x longer pass of the same runs (2^18 sweeps per evaluation), exchange every
sweep.  A step is one call of the engineering loop's public entry point
engineer_run(t, K, K): K consecutive RAO steps (Algorithm 1), whose K candidate
instances are PT-evaluated as one batched launch sequence (extra batches when a
candidate is kept early).

Reported: spin-flip attempts/s (value, device time), PT-TTS evaluations/s and
RAO steps/s, the end-to-end number through the same C-ABI call, the roofline
of the dominant kernel (pt_sweep_kernel, integer-issue bound), the CPU oracle
on a bounded sample, and SM clocks sampled during the timed region.

--impl reference times the CPU oracle (plain C, one thread) on a bounded
sample of the same workload per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "spin flips/s & PT-TTS evals/s; log-TTS gain per GPU-s, surrogate vs plain"
UNIT = "spin-flip attempts/s"

# Algorithmic integer operations per spin-flip attempt (counted from the
# method, not from the compiled code):
#   Philox4x32-10, 1/4 call per attempt: 10 rounds x (2 widening multiplies,
#     2 three-input xors, 2 key-schedule adds) / 4            = 15
#   local field over 6 neighbours: 6 multiply-adds            =  6
#   k = -s_i h_i                                              =  1
#   acceptance: clamp, table load, 2 compares, or             =  5
#   flip, energy and accept-count updates                     =  3
#   spin loads (4 words per 4 spins) and store (1 per 4)      =  1.25
OPS_PER_ATTEMPT = 31.25
# Integer issue peak per SM and clock: 4 sub-partitions x 32 lanes.
INT_LANES_PER_SM_CLK = 128
# DRAM bytes (read + write) of one sweep-kernel launch, taken from one ncu
# capture of the C_8 / 32-temperature / 1024-run launch (dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by (team, slot_parallel, runs_per_cta, runs).
# It is a profiled constant, not measured in the bench run: a launch reads the
# runs' state once and its write-back stays in L2, so the figure does not
# depend on the sweeps per launch.  Any other schedule reports null, and so
# does every schedule while the kernel has changed since the last capture.
PROFILED_TRAFFIC = {(4, 32, 1, 1024): 17554176}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def measured_int_issue(P, stream, peak_ops, iters=1 << 18, reps=3):
    """The integer-issue microbenchmark (pt_int_issue_rate) of every kind, run
    outside the timed region: measured T ops/s and the fraction of the
    derived peak, so the derived roofline can be read against the sustained
    rate of the instruction kinds the sweep is made of."""
    out = {}
    for kind in P.INT_ISSUE_KINDS:
        ops, ms = P.int_issue_rate(kind, iters=iters, reps=reps, stream=stream)
        out[kind] = {"Tops_s": ops / 1e12, "of_derived_peak": ops / peak_ops if peak_ops else None,
                     "ms_per_launch": ms}
    return out


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            if self.path:
                self.fh.close()
                os.unlink(self.path)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=ws)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(ws, x):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def workload():
    cfg = W.CONFIGS["c8_single"]
    return cfg


def oracle_sample(cfg, sweeps, runs):
    """CPU oracle on a bounded sample: `runs` runs x all slots x `sweeps` sweeps."""
    import oracle
    oracle.build()
    J = W.random_couplers(cfg["L"], cfg["seed"], 0)
    betas = W.beta_ladder(cfg["n_temps"], cfg["beta_min"], cfg["beta_max"])
    st = oracle.PTState(cfg["L"], J, betas, runs, cfg["seed"], 0)
    t0 = time.perf_counter()
    st.sweeps(sweeps, cfg["exchange_every"])
    dt = time.perf_counter() - t0
    attempts = sweeps * runs * cfg["n_temps"] * 8 * cfg["L"] ** 2
    return attempts / dt, attempts, dt


def _oracle_worker(job):
    """One host process of the parallel CPU baseline: the oracle sample on instance uid `job[2]`."""
    cfg, sweeps, uid, runs = job
    import oracle
    J = W.random_couplers(cfg["L"], cfg["seed"], uid)
    betas = W.beta_ladder(cfg["n_temps"], cfg["beta_min"], cfg["beta_max"])
    st = oracle.PTState(cfg["L"], J, betas, runs, cfg["seed"], uid)
    t0 = time.perf_counter()
    st.sweeps(sweeps, cfg["exchange_every"])
    return sweeps * runs * cfg["n_temps"] * 8 * cfg["L"] ** 2, time.perf_counter() - t0


def oracle_sample_parallel(cfg, sweeps, runs, procs):
    """The oracle on all host cores: `procs` processes (spawned, so none inherits
    a CUDA context), each running the sample on its own instance (uid 0..procs-1),
    which is the path's own unit of parallelism.  Returns (attempts/s over the
    wall time of the slowest process, attempts, seconds)."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    with mp.get_context("spawn").Pool(procs) as pool:
        pool.map(_oracle_worker, [(cfg, 1, u, 1) for u in range(procs)])      # start-up, imports
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, [(cfg, sweeps, u, runs) for u in range(procs)])
        dt = time.perf_counter() - t0
    att = sum(r[0] for r in res)
    return att / dt, att, dt


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    cfg = workload()
    sweeps, runs = 32, cfg["n_runs"]
    procs = args.cpu_procs or os.cpu_count() or 1
    oracle_sample_parallel(cfg, 2, runs, procs)
    tot_att, tot_t = 0, 0.0
    for _ in range(args.warmup):
        oracle_sample_parallel(cfg, 4, runs, procs)
    for _ in range(args.steps):
        _, att, dt = oracle_sample_parallel(cfg, sweeps, runs, procs)
        tot_att += att
        tot_t += dt
    v = tot_att / tot_t
    per_eval = cfg["sweeps"] * cfg["pass_mult"] * cfg["n_runs"] * cfg["n_temps"] * 8 * cfg["L"] ** 2
    sample = (f"{procs} processes x ({runs} runs x {cfg['n_temps']} slots x {sweeps} sweeps) of "
              f"{procs} C_8 instances per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": "c8_single: C_8 N=512, 32 temps beta [0.1,4], 64 runs, S=2^16, 4x target pass",
                   "sample": sample},
        "pt_tts_evals_per_s": v / per_eval,
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_gpu(args):
    import torch

    ws, rank, local = dist_setup()
    import paper_1605_03607_gb300 as P
    from paper_1605_03607_gb300 import build as B
    B.build()
    P.select_device(local)
    torch.cuda.set_device(local)
    cfg = workload()
    L, NT, R, S, pm = cfg["L"], cfg["n_temps"], cfg["n_runs"], cfg["sweeps"], cfg["pass_mult"]
    N = 8 * L * L
    spec = args.speculation
    uid = rank                                       # weak scaling: one instance per GPU
    J = W.random_couplers(L, cfg["seed"], uid)
    betas = W.beta_ladder(NT, cfg["beta_min"], cfg["beta_max"])
    stream = torch.cuda.current_stream()
    h = P.PTHandle(L, J, betas, R, cfg["seed"], uid, stream=stream.cuda_stream)
    if args.mapping:
        h.set_mapping(*[int(x) for x in args.mapping.split(",")])
    if args.schedule:
        h.set_schedule(*[int(x) for x in args.schedule.split(",")])
    elif not args.no_autotune and not args.mapping:
        h.autotune(n_inst=spec, trial_sweeps=64)
    h.set_timing(True)
    h.engineer_begin(S=S, pass_mult=pm, exchange_every=cfg["exchange_every"], base_uid=uid)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")   # > 129 MB L2
    step = 0
    for _ in range(args.warmup):
        h.engineer_run(step, spec, spec)
        step += spec
    h.eval_stats(reset=True)
    h.set_timing(True)
    n0 = h.launch_count()
    sampler = ClockSampler(local)
    barrier(ws)
    torch.cuda.synchronize()
    sampler.start()
    dev_ms, wall_s = 0.0, 0.0
    accepted = 0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        e0.record(stream)
        res = h.engineer_run(step, spec, spec)
        e1.record(stream)
        e1.synchronize()
        wall_s += time.perf_counter() - w0
        dev_ms += e0.elapsed_time(e1)
        accepted += int(res["accepted"].sum())
        step += spec
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop()
    launches = h.launch_count() - n0
    tts_now, hits_now = h.engineer_state()
    evals, batches, eval_ms = h.eval_stats()
    sweep_ms, sweep_launches = h.sweep_timing_total()
    attempts = evals * R * NT * N * S * pm
    t_dev = max_over_ranks(ws, dev_ms / 1e3)
    t_wall = max_over_ranks(ws, wall_s)
    tot_attempts = sum_over_ranks(ws, attempts)
    tot_evals = sum_over_ranks(ws, evals)
    tot_steps = sum_over_ranks(ws, args.steps * spec)
    peaks, peak_kind = load_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak_ops = sms * INT_LANES_PER_SM_CLK * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    achieved_ops = attempts * OPS_PER_ATTEMPT / (sweep_ms / 1e3) if sweep_ms > 0 else 0.0
    # h2d per step: packed candidate couplers + instance descriptors; d2h: 3 ints per candidate
    h2d = batches / max(args.steps, 1) * (spec * (L * L * 16 * 4) + spec * 128)
    d2h = batches / max(args.steps, 1) * spec * 12
    if rank != 0:
        h.close()
        return 0
    issue = measured_int_issue(P, stream.cuda_stream, peak_ops)
    cpu = None
    if ws == 1 and not args.no_cpu:
        v1, att1, dt1 = oracle_sample(cfg, args.cpu_sweeps, R)
        procs = args.cpu_procs or os.cpu_count() or 1
        v, att, dt = oracle_sample_parallel(cfg, args.cpu_sweeps, R, procs)
        cpu = {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle",
               "sample": f"{procs} processes, each {R} runs x {NT} slots x {args.cpu_sweeps} sweeps of its own "
                         f"C_8 instance ({att:.3g} attempts, {dt:.1f} s)",
               "single_thread": {"value": v1, "cores": 1,
                                 "sample": f"{R} runs x {NT} slots x {args.cpu_sweeps} sweeps "
                                           f"({att1:.3g} attempts, {dt1:.1f} s)"}}
    line = {
        "metric": METRIC, "value": tot_attempts / t_dev, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": "c8_single: C_8 N=512 (1472 couplers, J in {+-1,+-2,+-3}), 32 temps "
                               "beta geometric [0.1,4], 64 PT runs, S=2^16, target from 4x pass, "
                               "exchange every sweep",
                   "step": f"engineer_run: {spec} RAO steps, candidates evaluated in batches of {spec}",
                   "speculation": spec, "schedule": list(h.schedule()), "team": h.mapping(),
                   "l2": "flushed between steps",
                   "parallelism": f"{ws} independent instance(s), one per GPU"},
        "pt_tts_evals_per_s": tot_evals / t_dev,
        "rao_steps_per_s": tot_steps / t_dev,
        "accepted_moves": accepted,
        "instance_state": {"tts_sweeps": tts_now, "n_hit": hits_now, "runs": R, "horizon_S": S,
                           "unsolved": bool(tts_now > S),
                           "note": "TTS of the engineered instance after the timed steps; at the unsolved "
                                   "cap (TTS = S + 1) no candidate can be kept"},
        "e2e": {"value": tot_attempts / t_wall, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "pt_tts_evals_per_s": tot_evals / t_wall},
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "achieved": achieved_ops / 1e12, "peak": peak_ops / 1e12,
                     "unit": "Tops/s (int32 issue)", "frac": achieved_ops / peak_ops if peak_ops else None,
                     "traffic": PROFILED_TRAFFIC.get((h.mapping(), *h.schedule()[:2], R * spec)),
                     "traffic_source": "profiled constant (one ncu capture of this schedule), not measured "
                                       "in this run",
                     "kernel": "pt_sweep_kernel",
                     "ops_per_attempt": OPS_PER_ATTEMPT,
                     "avg_launch_ms": sweep_ms / max(sweep_launches, 1), "launches": sweep_launches,
                     "peak_source": f"{sms} SMs x {INT_LANES_PER_SM_CLK} lanes x "
                                    f"{peaks.get('sm_max_mhz', 2070.0)} MHz ({peak_kind} max clock)",
                     "measured_int_issue": issue},
        "cpu_baseline": cpu,
        "clocks": clocks,
    }
    h.close()
    if ws == 1 and not args.no_batched:
        # the batched configuration, measured after (outside) the timed region above
        line["batched"] = measure_batched(args, steps=args.batched_steps, warmup=1)
    print(json.dumps(line))
    return 0


def measure_batched(args, steps, warmup):
    """Batched workload: 256 instances mixed over C_4/8/12/16 with 24..48
    temperatures, 32 runs each; a step is fresh runs + `batch_sweeps` sweeps of
    every run (one graph replay of the persistent launch) + per-instance TTS.
    Returns the measurement as a dict (attempts/s, PT-TTS evaluations/s,
    roofline of the persistent sweep kernel, clocks)."""
    import torch
    import paper_1605_03607_gb300 as P
    from paper_1605_03607_gb300 import build as B
    B.build()
    cfg = W.CONFIGS["batched_256"]
    inst = W.batched_instances(cfg)
    sweeps = args.batch_sweeps
    attempts = sum(cfg["n_runs"] * len(x["betas"]) * 8 * x["L"] ** 2 for x in inst) * sweeps
    stream = torch.cuda.current_stream()
    b = P.PTBatch(inst, cfg["n_runs"], cfg["seed"], stream=stream.cuda_stream)
    if args.batch_mapping:
        # "L:team,slot_parallel,runs_per_cta;..." (team 0: cell-major)
        for item in args.batch_mapping.split(";"):
            Ls, rest = item.split(":")
            team, sp, ipc = (int(x) for x in rest.split(","))
            b.set_mapping(team, int(Ls), sp, ipc)
    elif not args.no_autotune:
        b.autotune(trial_sweeps=32)
    for _ in range(warmup):
        b.reset()
        b.run(sweeps, cfg["exchange_every"])
    sampler = ClockSampler(0)
    torch.cuda.synchronize()
    sampler.start()
    kern_ms, wall = 0.0, 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_solved = 0
    for _ in range(steps):
        b.reset()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        e0.record(stream)
        b.run(sweeps, cfg["exchange_every"])
        tts, _, _ = b.tts(sweeps)
        e1.record(stream)
        e1.synchronize()
        wall += time.perf_counter() - w0
        kern_ms += b.info()["last_run_ms"]
        n_solved = int(np.sum(tts <= sweeps))
    clocks = sampler.stop()
    peaks, peak_kind = load_peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak_ops = sms * INT_LANES_PER_SM_CLK * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    achieved = attempts * steps * OPS_PER_ATTEMPT / (kern_ms / 1e3)
    sched = {L: b.schedule(L) + (b.mapping(L),) for L in (4, 8, 12, 16)}
    out = {
        "workload": "batched_256: 256 instances, 64 each of C_4/C_8/C_12/C_16, 24..48 temps (beta [0.1,4]), "
                    "32 runs each, 2^14 sweeps, one persistent graph-captured launch per size group",
        "metric": "spin-flip attempts/s", "value": attempts * steps / wall, "unit": UNIT,
        "steps": steps, "warmup": warmup, "sweeps_per_step": sweeps,
        "kernel_attempts_per_s": attempts * steps / (kern_ms / 1e3),
        "pt_tts_evals_per_s": len(inst) * steps / wall,
        "instances_solved_within_S": n_solved,
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                     "unit": "Tops/s (int32 issue)", "frac": achieved / peak_ops,
                     "kernel": "pt_sweep_kernel (persistent)", "ops_per_attempt": OPS_PER_ATTEMPT,
                     "avg_launch_ms": kern_ms / max(steps, 1), "peak_source": peak_kind},
        "schedule": {str(k): v for k, v in sched.items()}, "info": b.info(), "clocks": clocks,
        "timing": "value over the host wall clock of reset + run + TTS per step; kernel_attempts_per_s "
                  "and the roofline over the graph replay's CUDA-event time"}
    b.close()
    return out


def run_batched(args):
    import torch
    import paper_1605_03607_gb300 as P
    out = measure_batched(args, steps=args.steps, warmup=args.warmup)
    peaks, _ = load_peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak_ops = sms * INT_LANES_PER_SM_CLK * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    out["roofline"]["measured_int_issue"] = measured_int_issue(P, torch.cuda.current_stream().cuda_stream, peak_ops)
    print(json.dumps(out))
    return 0


def run_mixing(args):
    """Temperature random walk (Sec. III.B): EMCS = 10 Metropolis sweeps + one
    exchange pass, on the C_8 bench instance with 30 temperatures (beta
    geometric in [0.1, 4]) and `mixing_runs` independent chains.  Reports the
    sweep rate with the walk tracked and untracked, the paper's first mixing
    criterion (the copy with the least hot-half time spends >= 20 % of the run
    there) and round trips per copy; the round-trip time (sweeps per completed
    cold -> hot -> cold trip) stands in for the mixing time in the second
    criterion (run >= 20 tau)."""
    import torch
    import paper_1605_03607_gb300 as P
    from paper_1605_03607_gb300 import build as B
    B.build()
    cfg = workload()
    L, NT, R, X = cfg["L"], 30, args.mixing_runs, 10
    n_sweeps = X * args.mixing_emcs
    J = W.random_couplers(L, cfg["seed"], 0)
    betas = W.beta_ladder(NT, cfg["beta_min"], cfg["beta_max"])
    h = P.PTHandle(L, J, betas, R, cfg["seed"], 0)
    if not args.no_autotune:
        h.autotune(n_inst=1, trial_sweeps=64)
    att = float(R) * NT * 8 * L * L * n_sweeps
    rates = {}
    sampler = ClockSampler(0)
    sampler.start()
    for walk in (False, True):
        h.set_walk_stats(walk)
        h.reset(0)
        h.sweep(X * 64, X)                       # warm-up launches
        h.reset(0)
        h.set_timing(True)
        h.sweep(n_sweeps, X)
        ms, n = h.sweep_timing_total()
        rates[walk] = att / (ms / 1e3)
    clocks = sampler.stop()
    hot, trips, passes = h.walk_stats()
    frac = hot.astype(np.float64) / max(passes, 1)
    mean_trips = float(trips.mean())
    tau_rt = n_sweeps / mean_trips if mean_trips > 0 else None
    print(json.dumps({
        "workload": "mixing: C_8 N=512, 30 temps beta geometric [0.1,4], EMCS = 10 sweeps + 1 exchange",
        "metric": "spin-flip attempts/s (walk tracked)", "value": rates[True], "unit": UNIT,
        "untracked_attempts_per_s": rates[False], "tracking_cost": 1.0 - rates[True] / rates[False],
        "chains": R, "emcs": args.mixing_emcs, "sweeps": n_sweeps, "exchange_passes": passes,
        "schedule": list(h.schedule()), "team": h.mapping(),
        "walk": {"min_hot_fraction": float(frac.min()), "median_hot_fraction": float(np.median(frac)),
                 "criterion_hot_half": bool(frac.min() >= 0.2),
                 "round_trips_per_copy_mean": mean_trips, "round_trips_min": int(trips.min()),
                 "sweeps_per_round_trip": tau_rt,
                 "criterion_20_tau": bool(tau_rt is not None and n_sweeps >= 20 * tau_rt)},
        "clocks": clocks, "data": "synthetic"}))
    h.close()
    return 0


def run_surrogate(args):
    """Surrogate training step (config 4's shape): forward, backward and Adam on
    a batch of 256 seeded C_8 instances with random log10-TTS targets.  Reports
    steps/s, graphs/s and the GEMM rate of the step's linear maps against the
    measured BF16 peak (the maps are K = 128 -> N = 64, HBM-bound; DRAM
    throughput comes from the ncu summary)."""
    import torch
    import paper_1605_03607_gb300 as P
    from paper_1605_03607_gb300 import build as B
    B.build()
    L, Bsz, H, layers = 8, 256, 64, 4
    N, E = 8 * L * L, W.chimera_n_edges(L)
    J = np.stack([W.random_couplers(L, 20160514, i) for i in range(Bsz)])
    t = np.random.default_rng(20160514).uniform(1.0, 4.0, Bsz)
    m = P.Surrogate(hidden=H, layers=layers)
    m.set_params(W.surrogate_init_params(20160514, H, layers))
    for _ in range(args.warmup):
        m.train_step(L, J, t)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(0)
    sampler.start()
    w0 = time.perf_counter()
    e0.record()
    for _ in range(args.steps):
        m.train_step(L, J, t)
    e1.record()
    e1.synchronize()
    wall = time.perf_counter() - w0
    clocks = sampler.stop()
    # the step's own launches run on the library's stream; the host waits for
    # each step's loss, so the wall clock bounds the device time
    ms = wall * 1e3 / args.steps
    flops = 3.0 * layers * 2.0 * 2 * H * H * Bsz * (3 * E + N)     # fwd + dX + dW of the 3 maps per layer
    peaks, kind = load_peaks()
    achieved = flops / (ms / 1e3) / 1e12
    print(json.dumps({
        "workload": f"surrogate train step: {Bsz} C_8 graphs (N={N}, E={E}), hidden {H}, {layers} layers",
        "metric": "surrogate training steps/s", "value": 1e3 / ms, "unit": "steps/s",
        "graphs_per_s": Bsz * 1e3 / ms, "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
        "dtype": "bf16 (fp32 accumulate)",
        "tensor": {"gemm_tflops": achieved, "peak": float(peaks.get("bf16_tflops", 1900.0)),
                   "frac": achieved / float(peaks.get("bf16_tflops", 1900.0)), "flops_per_step": flops,
                   "peak_source": kind},
        "clocks": clocks, "data": "synthetic"}))
    m.close()
    return 0


def run_lao(args):
    """Loop adaptive optimisation (Algorithm 2) on a planted C_8 instance:
    350 frustrated loops (length 4 w.p. 0.1, else 6; weights 1..5, the paper's), PT-TTS of
    every candidate against its known ground-state energy (one pass of
    S = 2^16 sweeps: the planted instance's TTS is about 26,000 sweeps, so a
    smaller horizon leaves every candidate at the unsolved cap), candidates in
    speculative batches of 16.  A step is one
    batch; reports LAO steps/s, PT-TTS evaluations/s and the sweep kernel's
    rate against the integer-issue roofline."""
    import torch
    import paper_1605_03607_gb300 as P
    from paper_1605_03607_gb300 import build as B
    B.build()
    cfg = workload()
    L, NT, R = cfg["L"], cfg["n_temps"], cfg["n_runs"]
    S, spec, M = 1 << 16, 16, 350
    betas = W.beta_ladder(NT, cfg["beta_min"], cfg["beta_max"])
    h = P.PTHandle(L, np.zeros(W.chimera_n_edges(L), np.int8), betas, R, cfg["seed"], 0)
    if not args.no_autotune:
        h.autotune(n_inst=spec, trial_sweeps=64)
    tts0 = h.lao_begin(S, 7, M, 5)
    e_gs0 = h.lao_state()["E_gs"]
    step = 1
    accepted_warmup = 0
    for _ in range(args.warmup):
        accepted_warmup += int(h.lao_run(step, spec, spec)["accepted"].sum())
        step += spec
    tts_warm = h.lao_state()["tts"]
    h.eval_stats(reset=True)
    h.set_timing(True)
    sampler = ClockSampler(0)
    torch.cuda.synchronize()
    sampler.start()
    w0 = time.perf_counter()
    accepted = 0
    for _ in range(args.steps):
        res = h.lao_run(step, spec, spec)
        accepted += int(res["accepted"].sum())
        step += spec
    wall = time.perf_counter() - w0
    clocks = sampler.stop()
    evals, batches, eval_ms = h.eval_stats()
    sweep_ms, launches = h.sweep_timing_total()
    attempts = evals * R * NT * 8 * L * L * S
    peaks, kind = load_peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak_ops = sms * INT_LANES_PER_SM_CLK * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    achieved = attempts * OPS_PER_ATTEMPT / (sweep_ms / 1e3)
    st = h.lao_state()
    # ground / first-excited overlaps of the engineered instance (Sec. III.B): one
    # fresh PT pass of the handle's runs, then per run its coldest replica at
    # each of the two levels
    h.reset(1)
    h.sweep(S, 1)
    ov = h.overlaps(st["E_gs"])
    ov["ratio_gs_es_over_gs_gs"] = (ov["q_gs_es"] / ov["q_gs_gs"]) if ov["q_gs_gs"] > 0 and ov["q_gs_es"] >= 0 else None
    print(json.dumps({
        "workload": f"lao: planted C_8 ({M} loops, weights 1..5), 32 temps beta [0.1,4], 64 runs, S=2^16 known target",
        "table_rows": h.table_rows(),
        "metric": "LAO steps/s", "value": args.steps * spec / wall, "unit": "steps/s",
        "pt_tts_evals_per_s": evals / wall, "attempts_per_s": attempts / (eval_ms / 1e3),
        "steps": args.steps, "warmup": args.warmup, "speculation": spec, "accepted": accepted,
        "accepted_warmup": accepted_warmup, "tts_initial": tts0, "tts_after_warmup": tts_warm,
        "tts_final": st["tts"], "unsolved_cap": S + 1, "E_gs_initial": e_gs0, "E_gs_final": st["E_gs"],
        "overlaps_final": ov,
        "schedule": list(h.schedule()), "team": h.mapping(),
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                     "unit": "Tops/s (int32 issue)", "frac": achieved / peak_ops, "kernel": "pt_sweep_kernel",
                     "ops_per_attempt": OPS_PER_ATTEMPT, "peak_source": kind},
        "clocks": clocks, "data": "synthetic"}))
    h.close()
    return 0


GUIDED_SHAPES = {
    # C_4: 16 temperatures in [0.1, 3], 64 runs, horizon 2^12 with the 4x target pass
    "c4": dict(L=4, n_temps=16, beta_min=0.1, beta_max=3.0, n_runs=64, S=1 << 12, pass_mult=4, max_sweeps=0),
    # C_8 (the single-instance configuration): 32 temperatures in [0.1, 4], 64 runs, 2^14 with the 4x pass
    "c8": dict(L=8, n_temps=32, beta_min=0.1, beta_max=4.0, n_runs=64, S=1 << 14, pass_mult=4, max_sweeps=0),
    # C_16 (the guided configuration): 48 temperatures in [0.05, 5], 32 runs, doubling budget 2^12 .. 2^20
    "c16": dict(L=16, n_temps=48, beta_min=0.05, beta_max=5.0, n_runs=32, S=1 << 12, pass_mult=1,
                max_sweeps=1 << 20),
}


def run_guided_experiment(args):
    """Surrogate-guided vs plain engineering at equal GPU time and identical
    acceptance.  Every arm runs engineer_guided_step: each step draws 64
    proposals, PT-evaluates 4 of them in one batched launch and keeps the
    largest TTS if it beats the current one.  The arms differ only in which 4
    are evaluated:
      plain      proposals 0..3 (no ranking);
      untrained  the 4 ranked best by a network with initial weights;
      online     the 4 ranked best by a network retrained every 8 steps on
                 the loop's 1024 most recent evaluations (differences
                 candidate - base, guided.train_pairs), the plain choice
                 until its first training; training time counts against its
                 budget.
    From each of --guided-test-instances seeded instances every arm runs for
    --guided-seconds; reported: gain in log10 TTS per GPU-second (up to the
    first unsolved TTS), per-arm mean and standard error, paired differences,
    and the noise floor of log10 TTS (one instance, 16 keys)."""
    import paper_1605_03607_gb300 as P
    from paper_1605_03607_gb300 import build as B
    from paper_1605_03607_gb300 import guided as G
    B.build()
    sh = GUIDED_SHAPES[args.guided_shape]
    L, NT, R = sh["L"], sh["n_temps"], sh["n_runs"]
    S, pm, mx = sh["S"], sh["pass_mult"], sh["max_sweeps"]
    seed = 20160515
    cap = (mx if mx else S) + 1
    betas = W.beta_ladder(NT, sh["beta_min"], sh["beta_max"])
    arms = ("plain", "untrained", "online")
    per = {a: [] for a in arms}
    detail = {a: [] for a in arms}
    noise = None
    for k in range(args.guided_test_instances):
        uid = 900 + k
        J0 = W.random_couplers(L, seed, uid)
        if k == 0:
            with P.PTHandle(L, J0, betas, R, seed, uid) as h:
                t = h.tts_eval_many(np.repeat(J0[None], 16, 0), np.arange(16) + 10_000_000, S, pm, mx)["tts"]
            ok = t < cap
            noise = {"instance_uid": uid, "keys": 16, "solved": int(ok.sum()),
                     "log10_tts_std": float(G.log10_tts(t[ok]).std(ddof=1)) if ok.sum() > 1 else None,
                     "tts_median": int(np.median(t))}
        for arm in arms:
            model = None
            if arm != "plain":
                model = P.Surrogate()
                model.set_params(W.surrogate_init_params(1))
            with P.PTHandle(L, J0, betas, R, seed, uid) as h:
                if not args.no_autotune and k == 0 and arm == "plain":
                    h.autotune(n_inst=4, trial_sweeps=32)
                h.engineer_begin(S=S, pass_mult=pm, exchange_every=1, base_uid=uid, max_sweeps=mx)
                trace, npairs = G.run_loop(h, L, args.guided_seconds, model=model, online=(arm == "online"))
            if model is not None:
                model.close()
            gain = G.gain_per_second(trace, cap=cap)
            per[arm].append(gain)
            detail[arm].append({"uid": uid, "gain_log10_tts_per_gpu_s": gain, "tts_initial": int(trace[0][1]),
                                "tts_final": int(trace[-1][1]), "gpu_s": trace[-1][0], "steps": trace[-1][2],
                                "evaluated": npairs})

    def mean_se(v):
        v = np.asarray(v, np.float64)
        return {"mean": float(v.mean()), "se": float(v.std(ddof=1) / np.sqrt(len(v))) if len(v) > 1 else None}

    print(json.dumps({
        "workload": f"guided_vs_plain ({args.guided_shape})",
        "metric": "log-TTS gain per GPU-s, surrogate vs plain", "unit": "log10 TTS / GPU-s",
        "config": {"shape": {k: v for k, v in sh.items()}, "proposals": 64, "evaluated_per_step": 4,
                   "acceptance": "best of the 4 evaluated, kept if its TTS beats the current one (all arms)",
                   "online_training": "every 8 steps, 4 epochs of train_pairs over the 1024 most recent pairs, "
                                      "lr 1e-3; no ranking before the first training",
                   "gpu_seconds_per_arm": args.guided_seconds, "instances": args.guided_test_instances,
                   "gain": "until the TTS first reaches the unsolved value, or the budget ends"},
        "noise_floor": noise,
        "arms": {a: dict(mean_se(per[a]), instances=detail[a]) for a in arms},
        "online_minus_plain": mean_se(np.asarray(per["online"]) - np.asarray(per["plain"])),
        "online_minus_untrained": mean_se(np.asarray(per["online"]) - np.asarray(per["untrained"])),
        "untrained_minus_plain": mean_se(np.asarray(per["untrained"]) - np.asarray(per["plain"])),
        "data": "synthetic"}))
    return 0


def run_int_issue(args):
    """The integer-issue microbenchmark alone: every kind, with the SM clock
    sampled while it runs."""
    import torch
    import paper_1605_03607_gb300 as P
    from paper_1605_03607_gb300 import build as B
    B.build()
    stream = torch.cuda.current_stream()
    peaks, peak_kind = load_peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = sms * INT_LANES_PER_SM_CLK * max_mhz * 1e6
    P.int_issue_rate(0, iters=1 << 16, reps=args.warmup or 1, stream=stream.cuda_stream)
    sampler = ClockSampler(0)
    sampler.start()
    issue = measured_int_issue(P, stream.cuda_stream, peak_ops, reps=max(args.steps, 1) * 5)
    clocks = sampler.stop()
    mhz = (clocks or {}).get("sm_mhz") or max_mhz
    for v in issue.values():
        v["lanes_per_sm_clk"] = v["Tops_s"] * 1e12 / (sms * mhz * 1e6)
    print(json.dumps({"workload": "int_issue", "metric": "32-bit integer operations/s by instruction kind",
                      "unit": "Tops/s", "derived_peak": peak_ops / 1e12,
                      "derived_peak_source": f"{sms} SMs x {INT_LANES_PER_SM_CLK} lanes x {max_mhz} MHz "
                                             f"({peak_kind} max clock)",
                      "kinds": issue, "clocks": clocks}))
    return 0


def run_profile_case(args):
    """A fixed, small sequence of sweep-kernel launches (for ncu captures):
    fresh runs, then `profile_sweeps` launches of sweeps_per_launch sweeps each,
    through pt_sweep.  Default shape: the bench instance with 64 x
    profile_instances runs; --profile-shape L,NT,R picks a seeded C_L instance
    with NT temperatures (beta geometric in [0.1, 4]) and R runs."""
    import paper_1605_03607_gb300 as P
    from paper_1605_03607_gb300 import build as B
    B.build()
    cfg = workload()
    if args.profile_shape:
        L, NT, R = (int(x) for x in args.profile_shape.split(","))
        J = W.random_couplers(L, cfg["seed"], 0)
        betas = W.beta_ladder(NT, cfg["beta_min"], cfg["beta_max"])
    else:
        L, R = cfg["L"], cfg["n_runs"] * args.profile_instances
        J = W.random_couplers(L, cfg["seed"], 0)
        betas = W.beta_ladder(cfg["n_temps"], cfg["beta_min"], cfg["beta_max"])
    h = P.PTHandle(L, J, betas, R, cfg["seed"], 0)
    if args.mapping:
        h.set_mapping(*[int(x) for x in args.mapping.split(",")])
    if args.schedule:
        h.set_schedule(*[int(x) for x in args.schedule.split(",")])
    spl = h.schedule()[2]
    h.set_timing(True)
    for _ in range(args.profile_sweeps):
        h.sweep(spl, cfg["exchange_every"])
    ms, n = h.sweep_timing_total()
    att = args.profile_sweeps * spl * h.R * h.NT * h.N
    print(json.dumps({"profile_case": True, "L": L, "n_temps": h.NT, "launches": n, "ms": ms,
                      "attempts_per_s": att / (ms / 1e3), "runs": h.R, "schedule": list(h.schedule()),
                      "team": h.mapping()}))
    h.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c8_single", choices=["c8_single", "batched_256", "guided", "mixing",
                                                                      "surrogate", "lao", "int_issue"])
    ap.add_argument("--mixing-runs", type=int, default=1024, help="mixing workload: independent PT chains")
    ap.add_argument("--mixing-emcs", type=int, default=1 << 14, help="mixing workload: EMCS per run")
    ap.add_argument("--guided-shape", default="c4", choices=sorted(GUIDED_SHAPES))
    ap.add_argument("--guided-seconds", type=float, default=45.0)
    ap.add_argument("--guided-test-instances", type=int, default=4)
    ap.add_argument("--batch-sweeps", type=int, default=1 << 14)
    ap.add_argument("--batch-mapping", default="",
                    help="batched workload: 'L:team,slot_parallel,runs_per_cta;...' instead of the autotuner")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="default workload: skip the batched measurement that follows the timed steps")
    ap.add_argument("--batched-steps", type=int, default=2,
                    help="default workload: timed steps of the batched measurement")
    ap.add_argument("--profile-sweeps", type=int, default=0,
                    help="profiling case: this many sweep launches on the bench instance, then exit")
    ap.add_argument("--profile-shape", default="", help="profiling case: L,n_temps,runs of a seeded C_L instance")
    ap.add_argument("--profile-instances", type=int, default=4,
                    help="profiling case: runs = 64 x this (as many runs as a speculative batch)")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--speculation", type=int, default=16)
    ap.add_argument("--schedule", default="", help="slot_parallel,runs_per_cta,sweeps_per_launch")
    ap.add_argument("--mapping", default="", help="team,slot_parallel,runs_per_cta (team 0: cell-major); "
                    "skips the autotuner")
    ap.add_argument("--cpu-sweeps", type=int, default=256)
    ap.add_argument("--cpu-procs", type=int, default=0, help="host processes of the CPU baseline (0: all cores)")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gb300":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_sweeps > 0:
        return run_profile_case(args)
    if args.workload == "batched_256":
        return run_batched(args)
    if args.workload == "mixing":
        return run_mixing(args)
    if args.workload == "surrogate":
        return run_surrogate(args)
    if args.workload == "lao":
        return run_lao(args)
    if args.workload == "guided":
        return run_guided_experiment(args)
    if args.workload == "int_issue":
        return run_int_issue(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
