#!/usr/bin/env python3
"""Throughput of the UC-ACOPF component-ADMM sweep on B300.

One step = one inner ADMM sweep (UC dynamic program, generator and line
subproblems, bus and duplicate-UC updates, z/y updates, residual reductions,
outer control) over every instance of the workload.  Default workload: the
largest single-GPU configuration, a synthetic 2000-bus / 3200-line /
500-generator grid over T = 24 hourly periods in 16 load scenarios, batched in
one launch sequence (FP64 throughout).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ucac|reference]

--impl reference times the FP64 CPU oracle (plain C, single thread) on a
bounded sample of the same workload and prints the same JSON line.
With N > 1 (torchrun) every rank runs its own replica of the workload
(independent instances, no collective on the data path: weak scaling).
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2310_13145_b300 import synth  # noqa: E402

METRIC = "ADMM sweeps/s (one sweep = all instances of the workload)"
UNIT = "sweeps/s"

# FP64 work of the line kernel per line-period solve (the unit a launch
# processes), counted by the hardware: (DADD + DMUL + 2 DFMA) thread
# instructions of one launch (ncu smsp__sass_thread_inst_executed_op_d*_pred_on)
# divided by the launch's line-period solves.  16 x 2000-bus scenarios:
# 501.6 M FLOP over 1,228,800 solves at sweep 31 (408.2 per solve; 180 per
# counted Newton iteration); the work per solve hardly moves over a run
# (472.0 per solve at sweep 701 against 469.2 at sweep 31 in an earlier
# capture), while the Newton count does.  The W-form kernel: 10,340.8 M
# FLOP at sweep 31 (8,415 per solve).  The captures and their commands are
# summarised under profiles/.
LINE_FLOP_PER_SOLVE = {"polar": 408.2, "w": 8415.3}
FP64_NOMINAL_TFLOPS = 1.25
# DRAM bytes (read + write) of one launch of the polar line kernel on the
# 16 x 2000-bus workload, from the same ncu capture of sweep 31; None for a
# form or workload not captured
LINE_TRAFFIC = {("polar", "c5_2000bus_T24x16"): 377.8e6}
# FP64 pipe cycles active over the line kernel's active cycles, from the same
# capture (sm__pipe_fp64_cycles_active, sweep 31)
LINE_FP64_BUSY = {"polar": 0.602, "w": 0.876}
# Algorithmic bytes (FP64 reads + writes each kernel must make) per unit of
# the streaming x-bar and generator kernels, from their data layout (a row
# keeps w = z + y/rho beside its next x-step target):
#  k_bus per line-period: 4 flow-end rows x (a, w, y, lambda, old copy read;
#    z, y, next target, w, copy written) 80 B + 4 w/theta-end rows x (a, w,
#    y, lambda read; z, y, next target, w written) 64 B = 576 B; per
#    gen-period the rows gp, gq, tc 3 x 64 B + pbar, qbar read and written
#    32 B = 224 B; per bus-period loads Pd, Qd and w, theta read and written
#    48 B;
#  k_ucbar per gen-period: 9 rows (on, sd, pl, pu, ql, qu, rd; su, ru of the
#    next period) x 64 B + ubar_on, ubar_sd, ubar_su read and written 48 B +
#    the objective's p, u_on, u_su, u_sd 32 B = 656 B;
#  k_gen per gen-period: 9 targets and p, phat read 88 B; p, q, phat and six
#    slacks 72 B and 9 row values 72 B written = 232 B.
STREAM_BYTES = {"k_bus": (576, 224, 48), "k_ucbar": (0, 656, 0), "k_gen": (0, 232, 0)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ucac", choices=["ucac", "reference"])
    ap.add_argument("--mode", default="sweep", choices=["sweep", "dp"],
                    help="dp: the UC dynamic program alone on 1,000 and 10,000 generators (Fig. 1 workload)")
    ap.add_argument("--workload", default="c5_2000bus_T24x16", choices=sorted(synth.CONFIGS))
    ap.add_argument("--instances", type=int, default=None, help="use only the first N instances (profiling)")
    ap.add_argument("--line-form", default="polar", choices=["polar", "w"])
    ap.add_argument("--no-ttc", action="store_true", help="skip the time-to-1e-4 run")
    ap.add_argument("--ttc-max-sweeps", type=int, default=6000)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned warm-start arm")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-instance batching comparison")
    ap.add_argument("--no-uc-warm", action="store_true", help="skip the UC warm-start time-to-1e-4 run")
    ap.add_argument("--uc-warm-sweeps", type=int, default=300, help="relaxed sweeps of the UC warm start")
    return ap.parse_args()


def dist_info():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def reduce_max(x: float, world: int, device="cpu") -> float:
    """Maximum of x over all ranks (the whole job ends when the slowest rank does)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(steps: int, world: int, max_ms: float) -> float:
    """Sweeps per second of the whole job: every rank runs `steps` sweeps of its
    own replica of the workload (weak scaling)."""
    return steps * world / (max_ms * 1e-3)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock and throttle-reason samples around a timed region.

    Sampling starts before the warm-up and waits for its first sample
    (nvidia-smi needs ~0.1-0.3 s, longer than a short timed region); one
    sample every 50 ms, each stamped with nvidia-smi's own wall-clock
    timestamp; mark(True) and
    mark(False) stamp the region's start and end on the host, and stop()
    keeps the samples taken within 0.1 s of the region (at least the last
    one before it and the first one after it, waiting for that one)."""
    FIELDS = "timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # the first sample, so that one precedes the timed region
        deadline = time.time() + 3.0
        while time.time() < deadline and not self._rows():
            time.sleep(0.05)

    def mark(self, begin):
        now = datetime.datetime.now()
        if begin:
            self.t0 = now
        else:
            self.t1 = now

    def _rows(self):
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(p[0], "%Y/%m/%d %H:%M:%S.%f")
                rows.append((ts, float(p[2]), float(p[3]), p[6], p[7], p[8], p[9]))
            except ValueError:
                continue
        return rows

    def stop(self):
        if self.proc is None:
            return None
        t1 = self.t1 or datetime.datetime.now()
        deadline = time.time() + 2.0
        while time.time() < deadline and not any(r[0] > t1 for r in self._rows()):
            time.sleep(0.05)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = self._rows()
        os.unlink(self.path)
        return clock_summary(rows, self.t0, t1)


def clock_summary(rows, t0, t1):
    """Median SM clock, maximum clock and throttle reasons of the samples
    (timestamp, sm_mhz, sm_max_mhz, hw_slowdown, hw_thermal_slowdown,
    sw_thermal_slowdown, sw_power_cap) taken within 0.1 s of [t0, t1], plus
    the last sample before and the first after; None without samples."""
    if not rows:
        return None
    t0 = t0 or rows[0][0]
    pad = datetime.timedelta(seconds=0.1)
    keep = [r for r in rows if t0 - pad <= r[0] <= t1 + pad]
    before = [r for r in rows if r[0] < t0 - pad]
    after = [r for r in rows if r[0] > t1 + pad]
    if before:
        keep.insert(0, before[-1])
    if after:
        keep.append(after[0])
    reasons = set()
    for r in keep:
        for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), r[3:]):
            if val.lower() == "active":
                reasons.add(name)
    return {"sm_mhz": statistics.median(r[1] for r in keep), "sm_max_mhz": max(r[2] for r in keep),
            "reasons": sorted(reasons), "samples": len(keep),
            "window_s": round((keep[-1][0] - keep[0][0]).total_seconds(), 3)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------------ CPU oracle
def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_sweep_rate(grids, budget_s, warm=1, threads=1):
    """Times the oracle (plain C; one thread, or `threads` threads of its
    OpenMP build) on one instance of the workload; returns (workload
    sweeps/s, sample description)."""
    import oracle
    omp = threads > 1
    oracle.build(omp=omp)
    if omp:
        oracle.threads(threads)
    g = grids[0]
    o = oracle.Oracle(g, omp=omp)
    o.sweep(warm)
    n, t0 = 0, time.perf_counter()
    while True:
        o.sweep()
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or n >= 50:
            break
    per_instance = el / n
    rate = 1.0 / (per_instance * len(grids))
    return rate, (f"{n} oracle sweep(s) of instance 0 of {len(grids)} (after {warm} warm-up) on {threads} "
                  f"thread(s), scaled to the batch")


def reference_arm(a, grids):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    import oracle
    # the oracle on every host core (its OpenMP build: the x-step subproblems
    # in parallel, the same bits as the single-thread build)
    ncores = os.cpu_count() or 1
    oracle.build(omp=True)
    oracle.threads(ncores)
    # bounded sample: every step is one oracle sweep over one instance restricted
    # to its first T_s periods, T_s chosen so that the whole run takes ~2 min.
    g0 = grids[0]
    probe = oracle.Oracle(g0, omp=True)
    probe.sweep(2)
    t0 = time.perf_counter()
    probe.sweep()
    t_full = time.perf_counter() - t0
    n_steps = a.steps + a.warmup
    budget = 120.0 / max(n_steps, 1)
    Ts = int(max(1, min(g0.T, np.floor(g0.T * budget / max(t_full, 1e-9)))))
    gs = g0.copy()
    gs.T = Ts
    gs.Pd = np.ascontiguousarray(g0.Pd[:Ts])
    gs.Qd = np.ascontiguousarray(g0.Qd[:Ts])
    o = oracle.Oracle(gs, omp=True)
    for _ in range(a.warmup):
        o.sweep()
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        o.sweep()
        times.append(time.perf_counter() - t0)
    per_period = (sum(times) / len(times)) / Ts
    val = 1.0 / (per_period * g0.T * len(grids))
    sample = f"oracle sweeps over instance 0 restricted to its first {Ts} of {g0.T} periods, scaled to the batch"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 / val, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded grids shaped like the paper's workloads)",
            "config": {"workload": a.workload, "instances": len(grids)},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": ncores, "kind": "oracle (OpenMP build)",
                             "sample": sample, "cpu": cpu_model()},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def dp_inputs(ng, T, seed):
    """Seeded UC subproblems: duplicate-row targets around the relaxed schedule,
    costs and minimum up/down times of the synthetic fleet."""
    rng = np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, ng, T])))
    return dict(tau_on=rng.uniform(-0.2, 1.2, (T, ng)), tau_su=rng.uniform(-0.2, 0.5, (T, ng)),
                tau_sd=rng.uniform(-0.2, 0.5, (T, ng)), c0=rng.uniform(100, 500, ng), csu=rng.uniform(200, 1000, ng),
                csd=np.zeros(ng), TU=rng.integers(1, 9, ng).astype(np.int32), TD=rng.integers(1, 9, ng).astype(np.int32),
                u0=rng.integers(0, 2, ng).astype(np.int32), K0=np.zeros(ng, np.int32))


def dp_mode(a):
    """The DP-only workload of Fig. 1: time of one UC-subproblem solve for all
    generators, GPU (ucac_ucdp) against the oracle's C loop on one core; the
    decisions and costs are checked bit for bit."""
    import torch
    import oracle
    from paper_2310_13145_b300 import build, ucac
    build.build()
    oracle.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream().cuda_stream
    rows = []
    rho = 1e4
    for ng in (1000, 10000):
        for T in (24, 48, 96, 168):
            x = dp_inputs(ng, T, 7)
            f64 = lambda v: torch.as_tensor(v, dtype=torch.float64, device=dev)
            i32 = lambda v: torch.as_tensor(v, dtype=torch.int32, device=dev)
            A = [f64(x["tau_on"]), f64(x["tau_su"]), f64(x["tau_sd"]), f64(x["c0"]), f64(x["csu"]), f64(x["csd"]),
                 i32(x["TU"]), i32(x["TD"]), i32(x["u0"]), i32(x["K0"])]
            u = torch.zeros((T, ng), dtype=torch.int8, device=dev)
            cost = torch.zeros(ng, dtype=torch.float64, device=dev)
            nb = ucac.ucac_ucdp_workspace_bytes(ng, T)
            ws = torch.empty(nb, dtype=torch.uint8, device=dev)
            args = [t.data_ptr() for t in A] + [u.data_ptr(), cost.data_ptr(), ws.data_ptr(), nb, stream]
            for _ in range(3):
                ucac.ucac_ucdp(ng, T, rho, *args)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 50
            e0.record()
            for _ in range(reps):
                ucac.ucac_ucdp(ng, T, rho, *args)
            e1.record()
            torch.cuda.synchronize()
            gpu_ms = e0.elapsed_time(e1) / reps
            t0 = time.perf_counter()
            uo, co = oracle.ucdp_batch(rho, x["tau_on"], x["tau_su"], x["tau_sd"], x["c0"], x["csu"], x["csd"],
                                       x["TU"], x["TD"], x["u0"], x["K0"])
            cpu_ms = (time.perf_counter() - t0) * 1e3
            exact = bool(np.array_equal(uo, u.cpu().numpy()) and np.array_equal(co, cost.cpu().numpy()))
            rows.append({"n_gen": ng, "T": T, "gpu_ms": gpu_ms, "cpu_ms": cpu_ms, "speedup": cpu_ms / gpu_ms,
                         "bit_exact": exact})
    print(json.dumps({"metric": "UC dynamic program (Algorithm 2) time per solve of all generators",
                      "unit": "ms", "higher_is_better": False, "workload": "dp_fig1 (1,000 and 10,000 generators, "
                      "T = 24..168, seeded targets)", "cpu": "oracle C loop, 1 core", "rows": rows}), flush=True)


def main():
    a = parse()
    rank, world, local = dist_info()
    if a.mode == "dp":
        if rank == 0:
            dp_mode(a)
        return
    grids = synth.config_instances(a.workload, a.instances)
    if a.impl == "reference":
        reference_arm(a, grids)
        return
    import torch
    from paper_2310_13145_b300 import build, ucac
    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    stream = torch.cuda.Stream()
    params = ucac.ucac_default_params()
    params.line_form = ucac.UCAC_LINE_POLAR if a.line_form == "polar" else ucac.UCAC_LINE_W
    h = ucac.Handle(grids, params=params, stream=stream.cuda_stream)
    tuning, cache = None, None
    if not a.no_autotune:
        cache = os.path.join(os.path.expanduser("~"), ".cache", "ucac", "autotune.txt")
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        tuning = h.autotune(3, cache)
    clk = ClockSampler(local)
    clk.start()
    with torch.cuda.stream(stream):
        h.enqueue(a.warmup)
        stream.synchronize()
        if world > 1:
            torch.distributed.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        clk.mark(True)
        e0.record(stream)
        h.enqueue(a.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        clk.mark(False)
        clocks = clk.stop()
    ms = reduce_max(e0.elapsed_time(e1), world, device="cuda")
    value = whole_job_value(a.steps, world, ms)
    # per-kernel device times (events on the handle's stream) and iteration counts
    r = h.residuals(0)
    kt = h.kernel_times(4)
    newton = sum(h.residuals(k)["newton"] for k in range(len(grids)))
    al = sum(h.residuals(k)["al"] for k in range(len(grids)))
    # per-solve device counters of the last sweep: histograms over all instances
    nhist, ahist = None, None
    for k in range(len(grids)):
        nw, na = h.line_counts(k)
        hn, ha = ucac.count_histogram(nw), ucac.count_histogram(na, top=4)
        nhist = hn if nhist is None else [x + y for x, y in zip(nhist, hn)]
        ahist = ha if ahist is None else [x + y for x, y in zip(ahist, ha)]
    fp64 = ucac.ucac_probe_fp64(5, stream.cuda_stream)
    torch.cuda.synchronize()
    t_br = kt["k_branch"] * 1e-3
    sz = synth.stack_sizes(grids)
    fps = LINE_FLOP_PER_SOLVE.get(a.line_form)
    achieved = fps * sz["branch_periods"] / t_br / 1e12 if fps else None
    peaks = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2032.0))
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    roofline = {"bound": "alu", "kernel": "k_branch (line subproblems, %s form)" % a.line_form,
                "achieved": achieved, "peak": fp64 / 1e12, "unit": "TFLOP/s",
                "frac": achieved / (fp64 / 1e12) if achieved else None,
                "traffic": LINE_TRAFFIC.get((a.line_form, a.workload)) if a.instances is None else None,
                "traffic_unit": "bytes per launch (ncu, sweep 31)",
                "flop_per_unit": fps, "units_per_launch": sz["branch_periods"],
                "flop_source": "ncu DADD + DMUL + 2 DFMA per line-period solve (sweep 31)",
                "peak_source": "measured FP64 FMA probe on this GPU, events (nominal %.2f)" % FP64_NOMINAL_TFLOPS,
                # the FP64 pipe's own rate at the maximum SM clock: 2 FMA lanes per SM per clock
                "peak_pipe_at_max_clock": 2 * 2 * n_sm * sm_mhz * 1e6 / 1e12,
                "frac_of_pipe_at_max_clock": (achieved / (4 * n_sm * sm_mhz * 1e6 / 1e12)) if achieved else None,
                "fp64_pipe_busy": LINE_FP64_BUSY.get(a.line_form),
                "note": "FLOP are the FP64 instructions the kernel executes; the common Newton step takes the "
                        "line-limit gradients in FP32 (660.8 FLOP per solve before it, 469.2 after, with 22% less "
                        "time; 408.2 since the common step forms no FP64 bound distances and the evaluation doubles on "
                        "the integer units), and the FP64 pipe is "
                        "busy 60% of the active cycles beside the per-lane solves' dependency and memory waits: "
                        "removing FP64 work the solve does not need lowers this FLOP-based fraction while the "
                        "kernel gets faster" if a.line_form == "polar" else None,
                "newton_per_sweep": newton, "al_per_sweep": al,
                "solves_by_newton_iterations": {"bins": "0..7, 8 or more", "counts": nhist},
                "solves_by_multiplier_rounds": {"bins": "0..3, 4 or more", "counts": ahist},
                "kernel_ms": kt}
    # streaming kernels: algorithmic bytes per launch / event time / measured HBM copy rate
    hbm = float(peaks.get("hbm_gbs", 6314.0))
    streaming = {}
    for kname, (per_bp, per_gp, per_up) in STREAM_BYTES.items():
        nbytes = per_bp * sz["branch_periods"] + per_gp * sz["gen_periods"] + per_up * sz["bus_periods"]
        gbs = nbytes / (kt[kname] * 1e-3) / 1e9
        streaming[kname] = {"bytes_per_launch": nbytes, "ms": kt[kname], "achieved_gbs": gbs, "hbm_frac": gbs / hbm}
    roofline["streaming"] = streaming
    roofline["hbm_peak_gbs"] = hbm
    # end to end through the public API: create from pinned host arrays, sweeps,
    # read back the solution and the residual record
    e2e = None
    if not a.no_e2e:
        e2e = e2e_run(ucac, grids, a.steps, stream, params, cache)
    ttc = None
    if not a.no_ttc:
        ttc = time_to_tolerance(ucac, grids, stream, params, a.ttc_max_sweeps, cache)
    ucw = None
    if not a.no_ttc and not a.no_uc_warm:
        # start and penalty variants on the 3 x 118-bus batch: the UC warm
        # start (Sec. IV-A) against the all-on start, and the adaptive
        # penalty (on the 2000-bus scenarios the UC warm start does not
        # converge within the sweep cap)
        g2 = synth.config_instances("c2_118bus_T24x3")
        pa = ucac.ucac_default_params(line_form=params.line_form, rho_every=10)
        ucw = {"workload": "c2_118bus_T24x3",
               "all_on_start": time_to_tolerance(ucac, g2, stream, params, a.ttc_max_sweeps),
               "uc_warm_start": time_to_tolerance(ucac, g2, stream, params, a.ttc_max_sweeps,
                                                  uc_warm=a.uc_warm_sweeps),
               "adaptive_penalty_every10": time_to_tolerance(ucac, g2, stream, pa, a.ttc_max_sweeps)}
    learned = None
    if not a.no_learned:
        learned = learned_arm(ucac, grids, stream, params, a, cache)
    batch = None
    if not a.no_batch:
        batch = batch_arm(ucac, stream, params, cache)
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        v, sample = oracle_sweep_rate(grids, budget_s=12.0)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
        # the same oracle with its x-step subproblems on every host core
        ncores = os.cpu_count() or 1
        v2, sample2 = oracle_sweep_rate(grids, budget_s=8.0, threads=ncores)
        cpu["all_cores"] = {"value": v2, "unit": UNIT, "cores": ncores, "kind": "oracle (OpenMP build)",
                            "sample": sample2, "cpu": cpu_model()}
    h.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded grids shaped like the paper's workloads)",
                "config": {"workload": a.workload, "instances": len(grids), "line_form": a.line_form,
                           "block_sizes": tuning,
                           "parallelism": "replicas" if world > 1 else "single",
                           "l2": "state larger than L2 (no flush needed)", "r_p_inst0": r["r_p"]},
                "gpu_launches": 6 * a.steps, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "time_to_1e-4": ttc, "variants_118bus": ucw, "learned": learned, "batch64": batch,
                "clocks": clocks}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def learned_arm(ucac, grids, stream, params, a, cache):
    """The learned warm start: train the default network (outside any timed
    region), then sweeps/s with it switched on over the same sweeps as the
    plain measurement (a fresh handle: cold start, the same warm-up and timed
    sweeps, the same block sizes), and the time to 1e-4 from a cold start
    with it."""
    import torch
    from paper_2310_13145_b300 import warmstart
    t0 = time.perf_counter()
    wp, info = warmstart.train_default()
    info["seconds"] = time.perf_counter() - t0
    hl = ucac.Handle(grids, params=params, stream=stream.cuda_stream)
    if cache is not None:
        hl.autotune(3, cache)  # cache hit: the bench handle's block sizes
    with torch.cuda.stream(stream):
        hl.set_warm_start(wp)
        hl.enqueue(a.warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        hl.enqueue(a.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    kt = hl.kernel_times(4)
    taken = sum(hl.warm_start_stats(k)[0] for k in range(len(grids)))
    errs = sum(hl.warm_start_stats(k)[1] for k in range(len(grids)))
    hl.close()
    out = {"sweeps_per_s": a.steps / (ms * 1e-3), "ms_per_step": ms / a.steps, "kernel_ms": kt,
           "starts_from_network": taken, "tensor_core_errors": errs, "training": info}
    if not a.no_ttc:
        out["time_to_1e-4"] = time_to_tolerance(ucac, grids, stream, params, a.ttc_max_sweeps, cache, warm=wp)
    return out


def batch_arm(ucac, stream, params, cache, warmup=5, sweeps=50):
    """The batching pattern on 64 instances of uneven size and horizon
    (buses 30..500, T in {12, 18, 24}): sweeps/s of one handle holding all
    of them (one graph replay per sweep, autotuned block sizes) against one
    handle per instance (64 graph replays per sweep), the same sweeps from
    the cold start on the same stream, CUDA events around the timed sweeps."""
    import torch
    grids = synth.config_instances("c4_batch64")

    def timed(handles):
        with torch.cuda.stream(stream):
            for hh in handles:
                hh.enqueue(warmup)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(sweeps):
                for hh in handles:
                    hh.enqueue(1)
            e1.record(stream)
            torch.cuda.synchronize()
        return sweeps / (e0.elapsed_time(e1) * 1e-3)

    hb = ucac.Handle(grids, params=params, stream=stream.cuda_stream)
    tuning = hb.autotune(3, cache) if cache is not None else None
    batched = timed([hb])
    hb.close()
    singles = [ucac.Handle([g], params=params, stream=stream.cuda_stream) for g in grids]
    separate = timed(singles)
    for hh in singles:
        hh.close()
    return {"workload": "c4_batch64", "instances": len(grids), "sweeps": sweeps,
            "batched_sweeps_per_s": batched, "one_handle_per_instance_sweeps_per_s": separate,
            "speedup": batched / separate, "block_sizes": tuning}


def time_to_tolerance(ucac, grids, stream, params, max_sweeps, cache=None, warm=None, uc_warm=0):
    """Cold start to convergence of every instance (r_p, r_d <= 1e-4 RMS and
    z_rms <= 1e-4, the inner and outer stops of Algorithm 1) through the public
    API: create from host arrays, ucac_iterate with host checks every 50
    sweeps (the checks are inside the timed region).  warm: parameters of the
    learned warm start (loaded inside the timed region) or None; uc_warm > 0:
    the UC warm start with that many relaxed sweeps, inside the timed region
    (its sweeps are counted in `sweeps`)."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = ucac.Handle(grids, params=params, stream=stream.cuda_stream)
    if cache:
        h.autotune(3, cache)  # cache hit: applies the tuned block sizes
    if warm is not None:
        h.set_warm_start(warm)
    t1 = time.perf_counter()
    done, rc = 0, 0
    if uc_warm:
        h.uc_warm_start(uc_warm, 0.5)
        done = uc_warm
    while done < max_sweeps + uc_warm and rc != 1:
        rc = h.iterate(params.check_every)
        done += params.check_every
    t2 = time.perf_counter()
    rs = [h.residuals(k) for k in range(len(grids))]
    taken = sum(h.warm_start_stats(k)[0] for k in range(len(grids))) if warm is not None else 0
    committed = 0
    for k, g in enumerate(grids):
        committed += int(np.sum(ucac.ucac_solution(h.h, k, g.T, g.n_gen, g.n_bus, g.n_branch)["u_on"]))
    h.close()
    return {"converged": rc == 1, "seconds": t2 - t0, "create_s": t1 - t0, "iterate_s": t2 - t1,
            "newton_total": sum(r["newton_total"] for r in rs), "al_total": sum(r["al_total"] for r in rs),
            "starts_from_network": taken,
            "sweeps": done, "check_every": params.check_every,
            # (a converged instance takes no further sweep: the last one to
            # converge fixes the run's length, up to the check interval)
            "instance_sweeps_max": max(r["sweeps"] for r in rs),
            "objective_mean": statistics.mean(r["objective"] for r in rs),
            "r_p_max": max(r["r_p"] for r in rs), "r_d_max": max(r["r_d"] for r in rs),
            "z_rms_max": max(r["z_rms"] for r in rs), "inf_norm_max": max(r["inf_norm_viol"] for r in rs),
            "outer_max": max(r["outer"] for r in rs),
            "committed_unit_periods": committed,
            "variant": ("learned warm start + batched" if warm is not None else
                        "UC warm start (%d relaxed sweeps)" % uc_warm if uc_warm else "plain (no learned warm start)")}


def e2e_run(ucac, grids, steps, stream, params, cache=None):
    import torch
    # pinned host copies of every grid array
    pinned = []
    for g in grids:
        gg = g.copy()
        for name, val in vars(g).items():
            if isinstance(val, np.ndarray):
                t = torch.from_numpy(np.ascontiguousarray(val)).pin_memory()
                setattr(gg, name, t.numpy())
        pinned.append(gg)
    h2d = sum(sum(v.nbytes for v in vars(g).values() if isinstance(v, np.ndarray)) for g in pinned)
    # page-locked result arrays, allocated like the pinned inputs before the timed region
    pin = lambda shape, dt: torch.empty(shape, dtype=torch.from_numpy(np.zeros(0, dt)).dtype).pin_memory().numpy()  # noqa: E731
    outs = [ucac.solution_arrays(g.T, g.n_gen, g.n_bus, g.n_branch, alloc=pin) for g in grids]
    d2h = sum(sum(a.nbytes for a in o.values()) for o in outs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = ucac.Handle(pinned, params=params, stream=stream.cuda_stream)
    if cache:
        h.autotune(3, cache)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    ucac.ucac_iterate(h.h, steps)
    t2 = time.perf_counter()
    for k, g in enumerate(grids):
        ucac.ucac_solution(h.h, k, g.T, g.n_gen, g.n_bus, g.n_branch, out=outs[k])
        h.residuals(k)
    t3 = time.perf_counter()
    h.close()
    el = t3 - t0
    return {"value": steps / el, "unit": UNIT, "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps,
            "create_s": t1 - t0, "sweeps_s": t2 - t1, "readback_s": t3 - t2,
            "sweeps_per_s_without_create_and_readback": steps / (t2 - t1),
            "note": "create from pinned host arrays + ucac_iterate (host checks every check_every sweeps) + "
                    "ucac_solution into pinned result arrays + ucac_residuals of every instance, amortised over "
                    "the steps; create, sweeps and readback are also given separately"}


if __name__ == "__main__":
    main()
