"""Benchmark: point-samples per second of the frozen-coefficient Picard sweep on GB300.

One step = one full Picard solve (Algorithm 1: initial iterate + K sweeps + residuals) of
the 45-D multi-rocket workload, the largest single-GPU configuration: 262,144 states (15
planar agents, positions N(0, 2^2), headings uniform in [-pi, pi]), N = 131,072 samples
per state and sweep, K = 30 sweeps, nu = 0.05 (delta = 0.1), T = 2.  metric value =
M * N * K / (device time of the step); the inputs are resident in HBM before the step
starts.  e2e repeats the measurement through hjg_value_grad with pinned host buffers
(state upload and value/gradient download inside the timed region).  The 6-D two-rocket
workload (65,536 states, N = 65,536, K = 20) is timed the same way under its own key.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload rockets45|rockets6|mixed|surrogate]

--impl reference times the FP64 CPU oracle (the test oracle, as it stands) on a bounded
sample of the same workload on the host cores.  Multi-GPU (torchrun): the state set is
sharded over the ranks in contiguous blocks (each rank's Philox counters offset by its
block's first global index, so it draws the samples of the unsharded solve) and the
per-sweep residual parts are combined by one all-reduce per solve (strong scaling: the
total work is fixed); rank 0 prints the max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import hjg_inputs  # noqa: E402

METRIC = "point-samples/s per Picard sweep (v+grad v)"
UNIT = "point-samples/s"
W = hjg_inputs.ROCKETS45          # the headline workload
W_EXTRA = hjg_inputs.ROCKETS6     # timed the same way, reported under its own key
BENCH_WORKLOADS = {"rockets45": hjg_inputs.ROCKETS45, "rockets6": hjg_inputs.ROCKETS6}
# The paper's own throughput on this path, for context only (its timings are CPU-only): its
# 3-D slice runs (1,600 states, N = 14,000, 12 sweeps in 13.5 s; N = 20,000, 15 sweeps in
# 23.6 s) give about 2.0e7 point-samples/s.
PAPER_CONTEXT = {"value": 2.0e7, "unit": UNIT,
                 "hardware": "one core of an Intel Core i7-14700K, JAX on the CPU backend",
                 "derived_from": "3-D slice timings (states x N x sweeps / time)"}

# Per-point-sample work of the sweep on the pipes that share its time (counts for each
# workload's game; the block index sits in the Philox counter words the first round does
# not multiply, so 4 of the 20 multiplies of a block depend only on the state and sweep and
# are not per-sample work):
#   Philox blocks per sample (eight normals per block): n / 8 for n <= 8 (packed slots),
#   ceil(n/8) above
#   high halves of the 32x32 products (mul.hi.u32, 32 per SM and clock): 16 per block
#   MUFU (XU pipe, 16 per SM and clock): log2 and sqrt per Box-Muller pair -- the pair's
#   cos and sin come from the 4,096-entry shared-memory table of the 12-bit angle field --,
#   one sqrt for the target distance and one exp2 weight at half cost: n + 1.5
#   issue (4 warp instructions = 128 thread instructions per SM and clock): the kernel's
#   own thread instructions per point-sample, per launch variant, from ncu
#   (smsp__inst_executed.sum x 32 / point-samples on each workload's small ncu case, one
#   capture per variant) -- measured, not algorithmic
#   mufu_equivalent: the 2n + 1.5 transcendental evaluations of the Box-Muller transform
#   with cos and sin on the MUFU pipe, the accounting before the table, over the MUFU peak;
#   kept for comparison only, it is no pipe's load
BLOCKS_PER_SAMPLE = {"double_int2": 2 / 8, "dubins3": 3 / 8, "rockets_rel3": 3 / 8, "rockets6": 6 / 8,
                     "rockets45": 6.0}
GAME_N = {"double_int2": 2, "dubins3": 3, "rockets_rel3": 3, "rockets6": 6, "rockets45": 45}
MUFU_PER_SAMPLE = {g: n + 1.5 for g, n in GAME_N.items()}
MUFU_EQUIV_PER_SAMPLE = {g: 2 * n + 1.5 for g, n in GAME_N.items()}
INSTR_PER_SAMPLE = {
    "rockets45": {0: 658.5, 1: 658.7, 2: 657.9, 3: 657.9, 4: 660.5, 5: 678.8, 6: 680.0, 7: 685.1,
                  8: 683.0, 9: 647.9, 10: 647.9, 11: 679.9},
    "rockets6": {0: 84.0, 1: 83.6, 2: 87.0, 3: 81.3, 4: 82.4, 5: 83.0, 6: 88.3, 7: 81.8, 8: 89.6,
                 9: 88.5, 10: 82.6, 11: 91.8},
    # the other games at their workloads' N (the per-state work is part of the count)
    "dubins3": {0: 56.1, 1: 54.0, 2: 56.6, 3: 54.0, 4: 54.3, 5: 54.6, 6: 57.2, 7: 54.7, 8: 58.2,
                9: 57.5, 10: 54.8, 11: 58.9},
    "rockets_rel3": {0: 63.4, 1: 60.3, 2: 63.2, 3: 60.3, 4: 61.6, 5: 58.5, 6: 61.2, 7: 58.6, 8: 67.4,
                     9: 64.1, 10: 58.7, 11: 65.7},
    "double_int2": {0: 55.3, 1: 53.4, 2: 58.5, 3: 53.4, 4: 55.4, 5: 49.0, 6: 54.1, 7: 49.5, 8: 64.2,
                    9: 58.9, 10: 49.3, 11: 58.9},
}
IMUL_PER_BLOCK = 16
# GB300 unit counts and clock: 152 SMs at 2070 MHz; per SM and clock 16 MUFU operations,
# 32 high-half integer multiplies and 4 issued warp instructions.
SMS = 152
SM_MAX_MHZ = 2070.0
MUFU_PER_SM_CLK = 16
IMUL_PER_SM_CLK = 32
ISSUE_PER_SM_CLK = 4 * 32

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one sweep launch of each
# workload at its full M and K, from one-pass ncu captures of the sweep kernel.  The
# traffic does not depend on N (samples never touch memory; each state's rows are read and
# written once per launch).  A workload without a capture of the current kernel has none.
# rockets45: 110,972,672 B read + 72,240,384 B written, captured at the full 262,144 states and
# K = 30 with N = 1,024 (launch variant 3); see profiles/.
DRAM_BYTES_LAUNCH = {"rockets45": 110972672.0 + 72240384.0,
                     # rockets6: 5,066,496 B read + 0 B written at M = 65,536, K = 20, N = 1,024
                     # (launch variant 7)
                     "rockets6": 5066496.0 + 0.0}


def roofline(game, samples, kernel_s, full_size=False, variant=None):
    """Binding-pipe roofline of the sweep kernel: operations per second over the pipe's peak
    at the maximum SM clock, for the MUFU and high-half-multiply pipes (algorithmic counts)
    and, where the launch variant's instruction count was measured, the issue port; the
    bound is the pipe closest to its peak."""
    clk = SMS * SM_MAX_MHZ * 1e6
    pipes = {
        "int_mul_hi": (samples * BLOCKS_PER_SAMPLE[game] * IMUL_PER_BLOCK, IMUL_PER_SM_CLK * clk),
        "mufu": (samples * MUFU_PER_SAMPLE[game], MUFU_PER_SM_CLK * clk),
    }
    ips = INSTR_PER_SAMPLE.get(game, {}).get(variant)
    if ips:
        pipes["issue"] = (samples * ips, ISSUE_PER_SM_CLK * clk)
    fr = {k: (ops / kernel_s) / peak for k, (ops, peak) in pipes.items()}
    bind = max(fr, key=fr.get)
    ops, peak = pipes[bind]
    traffic = DRAM_BYTES_LAUNCH.get(game) if full_size else None
    return {"bound": "alu", "pipe": bind, "achieved": ops / kernel_s / 1e9, "peak": peak / 1e9,
            "unit": "Gop/s", "frac": fr[bind], "traffic": traffic,
            "hbm_gbs": traffic / kernel_s / 1e9 if traffic else None,
            "ops_per_point_sample": ops / samples,
            "ops_kind": "thread instructions (measured by ncu for this launch variant)" if bind == "issue"
            else "algorithmic operations",
            "other_pipes": {k: round(v, 4) for k, v in fr.items() if k != bind},
            "mufu_equivalent_frac": round(samples * MUFU_EQUIV_PER_SAMPLE[game] / kernel_s / (MUFU_PER_SM_CLK * clk), 4),
            "peak_basis": "per-SM-per-clock pipe rate x 152 SMs x 2070 MHz"}


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value, device):
    """The largest value over the ranks of the default process group: the slowest rank's
    time, which the whole job's throughput is divided by."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def flush_l2(buf):
    buf.fill_(1.0)


def shard_solve(solve_parts, M, world, rank, group=None):
    """One rank's share of a sharded solve of M states: solve_parts(lo, hi) solves the
    contiguous block [lo, hi) (its Philox counters offset by lo) and returns (that block's
    per-sweep residual parts [K, 3] = (sum dv^2, sum v^2, max |dv|), anything else); one
    all-reduce over the ranks gives every rank the global residual of Algorithm 1.
    Returns (lo, hi, relative L2 residual [K], sup-norm change [K], anything else)."""
    from paper_2605_18566_gb300 import sharding
    lo, hi = sharding.shard_bounds(M, world, rank)
    parts, extra = solve_parts(lo, hi)
    rel, sup = sharding.combine_residual_parts(parts, group)
    return lo, hi, rel, sup, extra


def sweeps_to_floor(resid):
    """Residual floor = median of the last three sweeps' residuals; sweeps to the floor =
    the first sweep k from which on every residual stays within 10 % of the floor (a
    residual that first dips below the band and then rises back to it has not settled).
    Also the smallest residual and its sweep: a floor well above the minimum means the
    iteration moved away from its best iterate again."""
    r = np.asarray(resid, dtype=np.float64)
    floor = float(np.median(r[-3:]))
    inside = np.abs(r - floor) <= 0.1 * floor
    k = len(r)
    while k > 0 and inside[k - 1]:
        k -= 1
    return {"floor": floor, "sweeps": k + 1, "settled": bool(k < len(r)), "min": float(r.min()),
            "min_sweep": int(np.argmin(r)) + 1,
            "definition": "floor = median of the last 3 residuals; sweeps = first k such that every "
                          "residual from sweep k on is within 10 % of the floor (K + 1: not settled)"}


def sweep_diagnostics(w, x, n_states=4096, stream=None):
    """Per-sweep diagnostics of the benchmark trajectory on its first n_states states (the
    same global indices and draws as the full solve, one sweep per launch): the fraction of
    states whose frozen coefficient c changes sign, the fraction whose |c| sits at a clip
    bound, and the minimum and median ESS of each sweep."""
    import torch
    from paper_2605_18566_gb300 import Solver
    xs = x[:n_states].contiguous()
    s = Solver(w.game, w.nu, w.T, w.N, w.K, radius=w.radius, seed=0, stream=stream,
               speed=list(w.speed) or None)
    s.set_points(xs)
    c_prev = s.get_state()["c"]
    flips, clipped, ess_min, ess_med = [], [], [], []
    for _ in range(w.K):
        s.picard_sweep(1)
        st = s.get_state()
        d = s.diagnostics()
        c = st["c"]
        flips.append(round(float((torch.sign(c) != torch.sign(c_prev)).float().mean()), 5))
        clipped.append(round(d["clipped"] / n_states, 5))
        ess_min.append(round(d["ess_min"], 3))
        ess_med.append(round(d["ess_median"], 1))
        c_prev = c
    s.close()
    return {"states": n_states, "c_sign_flip_fraction": flips, "clipped_fraction": clipped,
            "ess_min": ess_min, "ess_median": ess_med}


def time_workload(w, steps, warmup, e2e_steps, dev, stream, rank, world, group=None, sharded=False):
    """Time `steps` full solves of workload w (after `warmup` untimed ones) on this rank's
    share of the states: the step's device time with CUDA events on the launching stream
    (L2 flushed before each step), the sweep kernel's own duration from the library's events
    around its launch, and the end-to-end solve through hjg_value_grad with pinned host
    buffers."""
    import torch
    from paper_2605_18566_gb300 import Solver, sharding
    x_np = hjg_inputs.points(w) if w.M == BENCH_WORKLOADS[w.game].M else \
        hjg_inputs.points(BENCH_WORKLOADS[w.game])[:w.M]
    lo, hi = sharding.shard_bounds(w.M, world, rank) if sharded else (0, w.M)
    x = torch.from_numpy(x_np[lo:hi]).to(dev)
    Ms = hi - lo
    solver = Solver(w.game, w.nu, w.T, w.N, w.K, radius=w.radius, seed=0, point_offset=lo,
                    stream=stream, speed=list(w.speed) or None)
    l2 = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    last = {}

    def solve_parts(a, b):
        solver.set_points(x)
        r, sup = solver.picard_sweep(w.K, residuals=True)
        return solver.residual_parts(w.K), (r, sup, solver.diagnostics()["last_ms"])

    def step():
        if sharded:
            _, _, rel, _, (_, _, kms) = shard_solve(solve_parts, w.M, world, rank, group)
        else:
            _, (rel, _, kms) = solve_parts(lo, hi)
        last["resid"], last["kern_ms"] = rel, kms

    with torch.cuda.stream(stream):
        solver.set_points(x)
        tuned = solver.autotune(max_states=16 * SMS * 6)   # launch variant, outside timing
        for _ in range(warmup):
            step()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    kern_ms = []
    with ClockSampler(dev.index or 0) as clk:
        for i in range(steps):
            with torch.cuda.stream(stream):
                flush_l2(l2)
                ev[i][0].record(stream)
                step()
                ev[i][1].record(stream)
            kern_ms.append(last["kern_ms"])
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    with torch.cuda.stream(stream):
        st = solver.get_state()
        final = (st["v"].cpu().numpy(), st["p"].cpu().numpy())
    del l2

    # ---- end to end through the public API with pinned host buffers
    x_host = torch.from_numpy(x_np[lo:hi]).pin_memory()
    v_host = torch.empty(Ms, dtype=torch.float64).pin_memory()
    g_host = torch.empty(Ms, w.n, dtype=torch.float32).pin_memory()
    e2e_steps = max(1, min(steps, e2e_steps))
    with torch.cuda.stream(stream):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            solver.value_grad(x_host, v_out=v_host, grad_out=g_host)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / e2e_steps
    solver.close()
    return {"step_ms": step_ms, "kern_ms": kern_ms, "e2e_s": e2e_s, "e2e_steps": e2e_steps,
            "tuned": tuned, "resid": last["resid"], "clocks": clk.summary(), "x": x_np,
            "final": final, "lo": lo, "hi": hi, "steps": steps,
            "h2d": int(x_np[lo:hi].nbytes), "d2h": int(Ms * 8 + Ms * w.n * 4 + w.K * 8)}


def workload_line(w, m, world, dev, sharded):
    """The JSON fields of one timed workload: whole-job throughput from the slowest rank's
    time, the sweep kernel's roofline, e2e and the residual floor."""
    total_ms, e2e_s = sum(m["step_ms"]), m["e2e_s"]
    kern_s = statistics.median(m["kern_ms"]) / 1e3
    if world > 1:
        total_ms = max_over_ranks(total_ms, dev)
        e2e_s = max_over_ranks(e2e_s, dev)
        kern_s = max_over_ranks(kern_s, dev)
    samples_per_step = w.M * w.N * w.K              # the whole state set, all ranks together
    rank_samples = (m["hi"] - m["lo"]) * w.N * w.K  # this rank's share (the roofline's units)
    scale = world if sharded else 1
    return {
        "value": samples_per_step * m["steps"] / (total_ms / 1e3),
        "ms_per_step": total_ms / m["steps"],
        "step_ms": {"median": statistics.median(m["step_ms"]),
                    "iqr": float(np.subtract(*np.percentile(m["step_ms"], [75, 25])))},
        "e2e": {"value": samples_per_step / e2e_s, "unit": UNIT, "steps": m["e2e_steps"],
                "h2d_bytes_per_step": m["h2d"] * scale, "d2h_bytes_per_step": m["d2h"] * scale},
        "roofline": dict(roofline(w.game, rank_samples, kern_s,
                                  full_size=not sharded and w.M == BENCH_WORKLOADS[w.game].M,
                                  variant=m["tuned"]["variant"]),
                         kernel_ms_per_step=kern_s * 1e3),
        "launch": {"variant": m["tuned"]["variant"], "threads": m["tuned"]["threads"]},
        "residuals": [float(r) for r in m["resid"]],
        "sweeps_to_floor": sweeps_to_floor(m["resid"]),
    }


DESCRIPTIONS = {
    "rockets45_gauss": "rockets45_gauss: 45-D 15-rocket game, M=262144 states (positions N(0,2^2), "
                       "headings U[-pi,pi]), N=131072 samples/state/sweep, K=30 sweeps, nu=0.05, T=2",
    "rockets6_uniform": "rockets6_uniform: 6-D two-rocket game, M=65536 states in [-3,3]^4x[-pi,pi]^2, "
                        "N=65536 samples/state/sweep, K=20 sweeps, nu=0.05, T=2",
}


def run_ours(args, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    sharded = world > 1
    stream = torch.cuda.Stream(device=dev)
    w = BENCH_WORKLOADS[args.workload]
    if args.states:   # a prefix of the state set (profiling): same states, same draws
        import dataclasses
        w = dataclasses.replace(w, M=min(args.states, w.M))
    m = time_workload(w, args.steps, args.warmup, args.e2e_steps, dev, stream, rank, world, sharded=sharded)
    line = workload_line(w, m, world, dev, sharded)
    out = {
        "metric": METRIC, "value": line["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": line["ms_per_step"], "higher_is_better": True,
        "step_ms": line["step_ms"],
        "scaling": "strong" if sharded else "weak", "vs_baseline": None,
        "dtype": "f32 (FP64 combine/log/residual)",
        "data": "synthetic (seeded states)",
        "config": {"workload": DESCRIPTIONS[w.name], "M": w.M, "N": w.N, "K": w.K,
                   "l2": "flushed (256 MB write) between steps", "launch": line["launch"],
                   "parallelism": ("states sharded over %d GPUs (contiguous blocks, Philox point offset, "
                                   "one all-reduce of the [K,3] residual parts per solve)" % world)
                                  if sharded else "1 GPU"},
        "e2e": line["e2e"],
        "gpu_launches": 3 * args.steps,
        "roofline": line["roofline"],
        "clocks": m["clocks"],
        "hbm_peak_gbs_measured": load_peaks().get("hbm_gbs"),
        "residuals": line["residuals"],
        "sweeps_to_floor": line["sweeps_to_floor"],
        "paper_context": PAPER_CONTEXT,
    }
    if not args.no_extras and w is W:
        # the 6-D workload timed the same way, then per-sweep diagnostics of both
        st2 = min(args.steps, 10)
        m2 = time_workload(W_EXTRA, st2, 3, args.e2e_steps, dev, stream, rank, world, sharded=sharded)
        l2 = workload_line(W_EXTRA, m2, world, dev, sharded)
        out[W_EXTRA.name] = {"workload": DESCRIPTIONS[W_EXTRA.name], "steps": st2, "warmup": 3,
                             **{k: l2[k] for k in ("value", "ms_per_step", "e2e", "roofline", "launch",
                                                   "residuals", "sweeps_to_floor")}}
        if rank == 0:
            with torch.cuda.stream(stream):
                out["diagnostics"] = {
                    w.name: sweep_diagnostics(w, torch.from_numpy(m["x"]).to(dev), stream=stream),
                    W_EXTRA.name: sweep_diagnostics(W_EXTRA, torch.from_numpy(m2["x"]).to(dev),
                                                    stream=stream)}
    out["_final"] = (m["final"], w)
    return out


def run_cpu_baseline(w, seconds_target=15.0):
    """The FP64 oracle as it stands, on a bounded sample of the workload's states (full N
    and K), timed on all host threads."""
    import oracle
    x = hjg_inputs.points(w)
    P = oracle.make_problem(w.game, w.n, w.delta, w.T, radius=w.radius, seed=0,
                            speed=list(w.speed) or None)
    # calibrate: one sweep of one state per thread, then size the timed sample so that the
    # full K-sweep solve takes about seconds_target of wall time on all host threads
    threads = oracle.num_threads()
    probe = hjg_inputs.subset_indices(w.M, threads, seed=4)
    t0 = time.perf_counter()
    oracle.picard(P, x[probe].astype(np.float64), w.N, 1, idx=probe)
    wall_per_state_sweep = max(time.perf_counter() - t0, 1e-4)   # per thread
    m = int(seconds_target / (wall_per_state_sweep * w.K)) * threads
    m = int(min(w.M, max(threads, m)))
    idx = hjg_inputs.subset_indices(w.M, m, seed=5)
    t0 = time.perf_counter()
    ref = oracle.picard(P, x[idx].astype(np.float64), w.N, w.K, idx=idx)
    el = time.perf_counter() - t0
    return {"value": m * w.N * w.K / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d of %d states (seeded subset), full N=%d and K=%d, %.1f s"
                      % (m, w.M, w.N, w.K, el), "elapsed_s": el}, (idx, ref, P, x)


ORACLE_AMP = 1e-5   # relative coefficient perturbation per sweep of the sensitivity check


def oracle_error(final, sample, w, max_explain=16):
    """The benchmark solve's error against the oracle's FP64 trajectory on the oracle's
    sample of states (same global indices, same draws): per state |dv|/(1+|v|) and
    ||dDv||/(1+||Dv||), the fraction within the parity tolerance (1e-4, 1e-3), and for the
    states outside it whether the oracle's own trajectory there moves by more than a tenth
    of the tolerance under relative coefficient perturbations of ORACLE_AMP per sweep
    (explained: a state where the Picard map is not contractive)."""
    import oracle
    (v, p), (idx, ref, P, x) = final, sample
    dv = np.abs(v[idx] - ref["v"]) / (1.0 + np.abs(ref["v"]))
    dp = np.linalg.norm(p[idx].astype(np.float64) - ref["p"], axis=1) / (1.0 + np.linalg.norm(ref["p"], axis=1))
    fail = (dv > 1e-4) | (dp > 1e-3)
    out = {"states": int(len(idx)), "within_tolerance": float((~fail).mean()),
           "dv_median": float(np.median(dv)), "dv_max": float(dv.max()),
           "dgrad_median": float(np.median(dp)), "dgrad_max": float(dp.max()),
           "tolerance": "|dv| <= 1e-4 (1+|v|), ||dDv|| <= 1e-3 (1+||Dv||) after K sweeps (FP64 oracle trajectory)"}
    bad = np.nonzero(fail)[0][:max_explain]
    explained = 0
    if len(bad):
        sub = idx[bad]
        ill = oracle.ill_conditioned(P, x[sub].astype(np.float64), w.N, w.K, ORACLE_AMP,
                                     {"v": ref["v"][bad], "p": ref["p"][bad]}, idx=sub)
        explained = int(ill.sum())
    out.update({"outside_tolerance": int(fail.sum()), "explained": explained,
                "unexplained": int(fail.sum()) - explained,
                "explained_by": "oracle trajectory moves > tol/10 under %.0e relative coefficient "
                                "perturbations per sweep (non-contractive state)" % ORACLE_AMP})
    return out


def ncu_case(w, variant, M=None, N=None, K=2):
    """A small case of one workload for ncu: M states (default 12 x 152: two waves of the
    CTA-per-state kernels; the warp-per-state kernels need 48 x 152 for one full wave), a
    few MB on the device, N samples (default the workload's), K sweeps per launch, launch
    variant `variant`; one warm-up launch, then one profiled launch."""
    import torch
    from paper_2605_18566_gb300 import Solver
    M = M or 12 * SMS
    N = N or w.N
    x = torch.from_numpy(hjg_inputs.points(w)[:M] if M <= w.M else hjg_inputs.points(w, M=M)).cuda()
    s = Solver(w.game, w.nu, w.T, N, K, radius=w.radius, variant=variant, speed=list(w.speed) or None)
    for _ in range(2):
        s.set_points(x)
        r, _ = s.picard_sweep(K)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": w.name, "M": M, "N": N, "K": K, "variant": variant,
                      "sweep_ms": s.diagnostics()["last_ms"], "resid": list(r)}))
    s.close()


def ncu_case_surrogate():
    """A small case of the surrogate's training for ncu: one epoch of 8 Adam steps at batch
    8,192 on 65,536 seeded Gaussian tuples of the 45-D network (45 -> 256^3 -> 46)."""
    import torch
    from paper_2605_18566_gb300 import Surrogate
    g = torch.Generator(device="cuda").manual_seed(0)
    X = torch.randn(65536, 45, device="cuda", generator=g)
    Y = torch.randn(65536, 46, device="cuda", generator=g)
    sur = Surrogate(45, 46, 256, seed=0)
    hist = sur.fit(X, Y, epochs=1, batch=8192, lr=1e-3, lr_final=1e-4)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": "surrogate_mlp", "batch": 8192, "steps": 8, "loss": hist[-1]}))
    sur.close()


def run_mixed(args):
    """The mixed batch plus the 100,000-agent flock, all at nu = 0.02, T = 1, N = 16,384,
    K = 15 (the instances of hjg_inputs.MIXED and the flock), advanced by one CUDA-graph
    launch per step; value = total point-samples of all instances / device time."""
    import torch
    from paper_2605_18566_gb300 import Batch, Solver
    N, K, nu, T = 16384, 15, 0.02, 1.0
    inst = list(hjg_inputs.MIXED) + [(hjg_inputs.FLOCK, hjg_inputs.FLOCK.M)]
    solvers, xs = [], []
    for i, (w, M) in enumerate(inst):
        x = hjg_inputs.points(w, M=M) if w.game != "dubins3" else \
            np.tile(hjg_inputs.points(w), (max(1, M // 4096), 1))[:M]
        xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        s = Solver(w.game, nu, T, N, K, radius=w.radius, instance=i)
        s.set_points(xt)
        s.autotune(max_states=4 * SMS * 6)
        solvers.append(s); xs.append(xt)
    b = Batch(solvers)
    samples = sum(M for _, M in inst) * N * K
    for _ in range(args.warmup):
        for s, x in zip(solvers, xs):
            s.set_points(x)
        b.run(K)
    ms = []
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            for s, x in zip(solvers, xs):
                s.set_points(x)
            _, t = b.run(K)
            ms.append(t)
    out = {"metric": METRIC, "value": samples / (sum(ms) / len(ms) / 1e3), "unit": UNIT,
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": sum(ms) / len(ms), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32 (FP64 combine/log/residual)",
           "data": "synthetic (seeded states; flock of 6 Gaussian clusters on a ring)",
           "config": {"workload": "mixed batch, plain form (every instance from the plain initial "
                                  "iterate, no surrogate warm start): Dubins 1,024 + 65,536; rockets6 "
                                  "4,096 + 131,072; rockets45 16,384 + 262,144 states; + 100,000-agent "
                                  "flock, nu=0.02, T=1, N=16384, K=15, one CUDA-graph launch",
                      "instances": len(inst), "states": sum(M for _, M in inst),
                      "launch": "graph of per-instance sweep + residual kernels (batch)"},
           "clocks": clk.summary()}
    b.close()
    for s in solvers:
        s.close()
    return out


def run_games(args):
    """Every game's sweep kernel on its own workload's states: the autotuner's launch variant,
    the best of three timed launches of 2 sweeps at the workload's N (the Dubins game at
    N = 65,536), with the binding-pipe roofline where the game's per-sample work is counted
    (the flock's target reads its neighbour lists: no count, no roofline); and the 3-D Dubins
    workload as specified (4,096 states, N = 4,096, 10 sweeps) solved in FP32 and in FP64."""
    import torch
    from paper_2605_18566_gb300 import Solver
    games = {}
    with ClockSampler(0) as clk:
        for w in (hjg_inputs.DOUBLE_INT2, hjg_inputs.DUBINS3, hjg_inputs.ROCKETS_REL3, hjg_inputs.FLOCK,
                  hjg_inputs.ROCKETS6, hjg_inputs.ROCKETS45):
            x = torch.from_numpy(hjg_inputs.points(w)).cuda()
            N = 65536 if w.game == "dubins3" else w.N
            s = Solver(w.game, w.nu, w.T, N, 2, radius=w.radius, speed=list(w.speed) or None)
            s.set_points(x)
            t = s.autotune(max_states=4 * SMS * 6)
            best = float("inf")
            for _ in range(max(3, args.steps)):
                s.set_points(x)
                s.picard_sweep(2)
                best = min(best, s.diagnostics()["last_ms"])
            samples = x.shape[0] * N * 2
            games[w.name] = {"game": w.game, "M": int(x.shape[0]), "N": N, "sweeps": 2,
                             "variant": t["variant"], "threads": t["threads"], "kernel_ms": best,
                             "value": samples / (best / 1e3),
                             "roofline": roofline(w.game, samples, best / 1e3, variant=t["variant"])
                             if w.game in BLOCKS_PER_SAMPLE else None}
            s.close()
        w = hjg_inputs.DUBINS3
        x = torch.from_numpy(hjg_inputs.points(w)).cuda()
        solves = {}
        for prec in ("fp32", "fp64"):
            s = Solver(w.game, w.nu, w.T, w.N, w.K, radius=w.radius, precision=prec)
            s.set_points(x)
            if prec == "fp32":
                s.autotune()
            best = float("inf")
            for _ in range(3):
                s.set_points(x)
                s.picard_sweep(w.K)
                best = min(best, s.diagnostics()["last_ms"])
            solves[prec] = {"kernel_ms": best, "value": w.M * w.N * w.K / (best / 1e3)}
            s.close()
    return {"metric": METRIC + ", per game", "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
            "dtype": "f32 (FP64 combine/log/residual)", "data": "synthetic (seeded states)",
            "games": games, "dubins3_workload_solve": solves, "clocks": clk.summary()}


def surrogate_study(points_fn, label):
    """One study of the learned part on the 45-D game.  Tuples: the invariant-frame features
    (hjg_frame_features, 56 inputs) of 1,048,576 states drawn by points_fn and the correction
    (v - l, Dv - Dl) that 12 tilted control-variate sweeps at N = 16,384 make to the initial
    iterate, in the frame and averaged over the last four sweeps (hjg_frame_targets, 43
    outputs).  GPU training of the 56 -> 256^3 -> 43 BF16 network on them.  Then, on 1,024
    held-out states, the value error against a tilted N = 2^20, 12-sweep reference of: the
    plain form (Algorithm 1 as printed, 12 sweeps), the tilted control-variate sweep started
    from l, and the same sweep warm-started from the network (hjg_warm_start_frame, position
    rows only), for K = 1, 2, 3, 6, 12 sweeps and N = 4,096, 16,384, 65,536.
    `sweeps_to_match`: per N, the fewest sweeps after which the assisted form is at least as
    close as the sweep from l after 12, with the device time of both (sweep kernel, plus the
    network's features, forward pass and warm start for the assisted one)."""
    import torch
    from paper_2605_18566_gb300 import Solver, Surrogate
    w = hjg_inputs.ROCKETS45
    k_data, n_data, chunk, m_train = 12, 16384, 262144, 1 << 20
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X, Y = [], []
    for c in range(m_train // chunk):
        x = torch.from_numpy(points_fn(chunk, 100 + c)).cuda()
        s = Solver(w.game, w.nu, w.T, n_data, k_data, radius=w.radius, tilt=True, cv=True)
        s.set_points(x)
        X.append(s.frame_features())
        s.picard_sweep(k_data - 4, residuals=False)
        acc = None
        for _ in range(4):
            s.picard_sweep(1, residuals=False)
            t = s.frame_targets()
            acc = t if acc is None else acc + t
        Y.append(acc / 4)
        s.close()
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    X = torch.cat(X); Y = torch.cat(Y)
    perm = torch.from_numpy(np.random.default_rng(0).permutation(X.shape[0])).cuda()
    X = X[perm].contiguous(); Y = Y[perm].contiguous()
    sur = Surrogate(56, 43, 256, seed=0)
    epochs, batch = 30, 8192
    torch.cuda.synchronize(); t1 = time.perf_counter()
    hist = sur.fit(X, Y, epochs=epochs, batch=batch, lr=2e-3, lr_final=1e-4)
    torch.cuda.synchronize(); t_train = time.perf_counter() - t1
    xte = torch.from_numpy(points_fn(1024, 1)).cuda()
    probe = Solver(w.game, w.nu, w.T, 1024, 1, radius=w.radius)
    probe.set_points(xte)
    pred = sur.forward(probe.frame_features())
    probe.close()
    sur.close()

    def solve(N, K, tilt=True, cv=True, warm=False, seed=11, timed=False):
        so = Solver(w.game, w.nu, w.T, N, max(K, 1), radius=w.radius, tilt=tilt, seed=seed, cv=cv)
        so.set_points(xte)
        if warm:
            so.warm_start_frame(pred, positions_only=True)
        r = so.picard_sweep(K)[0] if K > 0 else [float("nan")]
        ms = so.diagnostics()["last_ms"] if K > 0 else 0.0
        st = so.get_state()
        so.close()
        out = (st["v"].cpu().numpy(), float(r[-1]))
        return out + (ms,) if timed else out

    # device time of the network's part of an assisted solve: frame features, forward pass,
    # warm start (CUDA events on the current stream, best of three)
    tsol = Solver(w.game, w.nu, w.T, 4096, 1, radius=w.radius, tilt=True, cv=True)
    tsol.set_points(xte)
    tnet = Surrogate(56, 43, 256, seed=0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    net_ms = float("inf")
    for _ in range(3):
        ev[0].record()
        tsol.warm_start_frame(tnet.forward(tsol.frame_features()), positions_only=True)
        ev[1].record()
        torch.cuda.synchronize()
        net_ms = min(net_ms, ev[0].elapsed_time(ev[1]))
    tsol.close(); tnet.close()

    vref, rref = solve(1 << 20, 12, cv=False, seed=7)
    rms = lambda v: float(np.sqrt(np.mean((v - vref) ** 2)))
    rows, match = [], []
    for N in (4096, 16384, 65536):
        v, r = solve(N, 12, tilt=False, cv=False)
        rows.append({"mode": "plain", "N": N, "K": 12, "rms_value_error": rms(v), "final_residual": r})
        for K in (1, 2, 3, 6, 12):
            for mode in ("tilt+cv", "surrogate+tilt+cv"):
                v, r, ms = solve(N, K, warm=mode.startswith("surrogate"), timed=True)
                rows.append({"mode": mode, "N": N, "K": K, "rms_value_error": rms(v), "final_residual": r,
                             "sweep_ms": ms})
        e12 = next(q["rms_value_error"] for q in rows if q["mode"] == "tilt+cv" and q["N"] == N and q["K"] == 12)
        ks = [q["K"] for q in rows if q["mode"] == "surrogate+tilt+cv" and q["N"] == N
              and q["rms_value_error"] <= e12]
        k_a = min(ks) if ks else None
        t12 = next(q["sweep_ms"] for q in rows if q["mode"] == "tilt+cv" and q["N"] == N and q["K"] == 12)
        ta = next((q["sweep_ms"] for q in rows if q["mode"] == "surrogate+tilt+cv" and q["N"] == N
                   and q["K"] == k_a), None)
        match.append({"N": N, "from_l_12_sweeps_error": e12, "assisted_sweeps": k_a,
                      "from_l_12_sweeps_ms": t12,
                      "assisted_ms_incl_network": ta + net_ms if ta is not None else None})
    return {"label": label, "tuple_generation_s": t_data, "train_s": t_train,
            "tuples": int(X.shape[0]), "epochs": epochs, "batch": batch,
            "loss": [hist[0], hist[-1]],
            "reference": {"N": 1 << 20, "K": 12, "tilt": True, "final_residual": rref},
            "initial_iterate_rms_value_error": rms(solve(4096, 0)[0]),
            "surrogate_alone_rms_value_error": rms(solve(4096, 0, warm=True)[0]),
            "network_ms_per_1024_states": net_ms, "study": rows, "sweeps_to_match": match}


def run_surrogate(args):
    """The learned part on the 45-D game, on two state distributions: the paper's wide one
    (positions uniform in [-100, 100]) and the workload's own (positions N(0, 2^2): most
    states start near a capture and no form converges there); the line's value is the
    training throughput of the first."""
    main = surrogate_study(lambda M, seed: hjg_inputs.rockets45_wide_points(M, seed),
                           "positions uniform in [-100, 100]")
    narrow = surrogate_study(lambda M, seed: hjg_inputs.rockets45_points(M, seed), "positions N(0, 2^2)")
    # per tuple: forward (4 layers), backward data gradients (3 products) and weight
    # gradients (4 layers) of the 56 -> 256^3 -> 43 network at its padded widths 64 and 48
    fwd = 64 * 256 + 2 * 256 * 256 + 256 * 48
    flops_per_tuple = 2 * (fwd + (48 * 256 + 2 * 256 * 256) + fwd)
    tuples = main["tuples"] * main["epochs"]
    tflops = tuples * flops_per_tuple / main["train_s"] / 1e12
    tensor_peak = load_peaks().get("bf16_tflops", 1906.5)
    return {"metric": "surrogate training tuples/s and error vs sweeps (45-D game)",
            "value": tuples / main["train_s"], "unit": "tuples/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "bf16 (FP32 accumulate)",
            "data": "synthetic (tuples from tilted control-variate sweeps)",
            "config": {"workload": "45-D game, 1,048,576 states uniform in [-100, 100], 12 sweeps at "
                                   "N = 16,384 -> 1,048,576 frame tuples; MLP 56-256-256-256-43",
                       "epochs": main["epochs"], "batch": main["batch"]},
            "mlp_tflops": tflops,
            "roofline": {"bound": "tensor", "achieved": tflops, "peak": tensor_peak, "unit": "TFLOP/s",
                         "frac": tflops / tensor_peak,
                         "note": "whole training step (products + element-wise + Adam) at batch 8192"},
            "studies": [main, narrow]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=2, help="end-to-end solves timed (at most --steps)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="time the headline workload only")
    ap.add_argument("--states", type=int, default=0,
                    help="profiling: time only the first STATES states of the workload (same draws)")
    ap.add_argument("--workload", default="rockets45", choices=list(BENCH_WORKLOADS) + ["mixed", "surrogate", "games"],
                    help="rockets45 (default, the benchmark line), rockets6, the mixed batch + flock, "
                         "the learned part on the 45-D game, or every game's sweep kernel")
    ap.add_argument("--ncu-case", default=None, choices=list(hjg_inputs.WORKLOADS) + ["surrogate_mlp"],
                    help="run one small launch of the named workload's sweep (profiling)")
    ap.add_argument("--variant", type=int, default=2, help="sweep launch variant for --ncu-case")
    ap.add_argument("--ncu-states", type=int, default=0, help="states of --ncu-case (default 12 x 152)")
    ap.add_argument("--ncu-N", type=int, default=0, help="samples of --ncu-case (default the workload's)")
    ap.add_argument("--ncu-K", type=int, default=2, help="sweeps of --ncu-case")
    args = ap.parse_args()
    rank, world, local_rank = dist_env()
    if args.ncu_case == "surrogate_mlp":
        ncu_case_surrogate()
        return
    if args.ncu_case:
        ncu_case(hjg_inputs.WORKLOADS[args.ncu_case], args.variant, args.ncu_states or None,
                 args.ncu_N or None, args.ncu_K)
        return

    if args.impl == "reference":
        if rank != 0:
            return
        w = BENCH_WORKLOADS.get(args.workload, W)
        runs = []
        for i in range(args.warmup + args.steps):
            r = run_cpu_baseline(w, seconds_target=6.0)[0]
            if i >= args.warmup:
                runs.append(r)
        val = statistics.median(r["value"] for r in runs)
        out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": 1e3 * statistics.median(r["elapsed_s"] for r in runs),
               "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded states)",
               "config": {"workload": DESCRIPTIONS[w.name] + " (bounded CPU sample per step)",
                          "M": w.M, "N": w.N, "K": w.K},
               "cpu_baseline": {"value": val, "unit": UNIT, "cores": runs[0]["cores"],
                                "kind": "oracle", "sample": runs[0]["sample"]},
               "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                       "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return

    if args.workload in ("mixed", "surrogate", "games"):
        if rank == 0:
            run = {"mixed": run_mixed, "surrogate": run_surrogate, "games": run_games}[args.workload]
            print(json.dumps(run(args)))
        return
    out = run_ours(args, rank, world, local_rank)
    final, w = out.pop("_final")
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"], sample = run_cpu_baseline(w)
            out["oracle_error"] = oracle_error(final, sample, w)
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
