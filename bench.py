"""Benchmark: point-samples per second of the frozen-coefficient Picard sweep on GB300.

One step = one full Picard solve (Algorithm 1: initial iterate + K sweeps + residuals) of
the two-rocket 6-D workload: 65,536 states uniform in [-3,3]^4 x [-pi,pi]^2, N = 65,536
samples per state and sweep, K = 20 sweeps, nu = 0.05 (delta = 0.1), T = 2.
metric value = M * N * K / (device time of the step); the inputs are resident in HBM
before the step starts.  e2e repeats the measurement through hjg_value_grad with pinned
host buffers (state upload and value/gradient download inside the timed region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the test oracle, as it stands) on a bounded
sample of the same workload on the host cores.  Multi-GPU (torchrun): every rank solves
its own independent instance of the workload (weak scaling, no collective on the data
path); rank 0 prints the max-over-ranks timing.
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
W = hjg_inputs.ROCKETS6
# The paper's own throughput on this path, for context only (its timings are CPU-only): its
# 3-D slice runs (1,600 states, N = 14,000, 12 sweeps in 13.5 s; N = 20,000, 15 sweeps in
# 23.6 s) give about 2.0e7 point-samples/s.
PAPER_CONTEXT = {"value": 2.0e7, "unit": UNIT,
                 "hardware": "one core of an Intel Core i7-14700K, JAX on the CPU backend",
                 "derived_from": "3-D slice timings (states x N x sweeps / time)"}

# Algorithmic per-point-sample work of the sweep on the two pipes that bind it (counts
# for each workload's game; the block index sits in the Philox counter words the first
# round does not multiply, so 4 of the 20 multiplies of a block depend only on the state
# and sweep and are not per-sample work):
#   Philox blocks per sample (six normals per block): n / 6 for n <= 8 (packed slots),
#   ceil(n/6) above
#   high halves of the 32x32 products (mul.hi.u32, 32 per SM and clock): 16 per block
#   (the low halves issue at twice that rate and are not the binding part)
#   MUFU (XU pipe): log2, sqrt, sin, cos per Box-Muller pair, one sqrt for the target
#   distance, one exp2 weight (exp2 issues at twice the rate of the others on GB300)
BLOCKS_PER_SAMPLE = {"dubins3": 0.5, "rockets6": 1.0, "rockets45": 8.0}
MUFU_PER_SAMPLE = {"dubins3": 2 * 3 + 2, "rockets6": 2 * 6 + 2, "rockets45": 2 * 45 + 2}
IMUL_PER_BLOCK = 16
# GB300 unit counts and clock: 152 SMs at 2070 MHz; per SM and clock 16 MUFU operations
# and 32 high-half integer multiplies.
SMS = 152
SM_MAX_MHZ = 2070.0
MUFU_PER_SM_CLK = 16
IMUL_PER_SM_CLK = 32


# DRAM bytes of one benchmark sweep launch (65,536 states, K = 20, the CTA-per-state
# pipelined variant the autotuner picks), from a one-pass ncu capture of that launch inside
# the benchmark command: dram__bytes_read.sum 5,168,896 B + dram__bytes_write.sum 0 B (the
# 11 MB of outputs and history rows stay in L2 until after the launch).
DRAM_BYTES_BENCH_LAUNCH = 5168896.0 + 0.0


def roofline(game, samples, kernel_s, states=None):
    """Binding-pipe roofline of the sweep kernel: achieved algorithmic operations per
    second over the pipe's peak at the maximum SM clock."""
    clk = SMS * SM_MAX_MHZ * 1e6
    pipes = {
        "int_mul_hi": (samples * BLOCKS_PER_SAMPLE[game] * IMUL_PER_BLOCK, IMUL_PER_SM_CLK * clk),
        "mufu": (samples * (MUFU_PER_SAMPLE[game] - 0.5), MUFU_PER_SM_CLK * clk),
    }
    fr = {k: (ops / kernel_s) / peak for k, (ops, peak) in pipes.items()}
    bind = max(fr, key=fr.get)
    ops, peak = pipes[bind]
    traffic = DRAM_BYTES_BENCH_LAUNCH if states == W.M and game == W.game else None
    return {"bound": "alu", "pipe": bind, "achieved": ops / kernel_s / 1e9, "peak": peak / 1e9,
            "unit": "Gop/s", "frac": fr[bind], "traffic": traffic,
            "hbm_gbs": traffic / kernel_s / 1e9 if traffic else None,
            "ops_per_point_sample": ops / samples,
            "other_pipes": {k: round(v, 4) for k, v in fr.items() if k != bind},
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


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2605_18566_gb300 import Solver
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    x_np = hjg_inputs.points(W, seed=W.seed + rank)
    x = torch.from_numpy(x_np).to(dev)
    stream = torch.cuda.Stream(device=dev)
    solver = Solver(W.game, W.nu, W.T, W.N, W.K, radius=W.radius, seed=0, instance=rank,
                    stream=stream)
    l2 = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2

    def step():
        solver.set_points(x)
        solver.picard_sweep(W.K, residuals=False)

    with torch.cuda.stream(stream):
        solver.set_points(x)
        tuned = solver.autotune(max_states=16 * SMS * 6)   # launch variant, outside timing
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(local_rank) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush_l2(l2)
                ev[i][0].record(stream)
                step()
                ev[i][1].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # sweep-kernel duration alone: the library brackets the sweep launch with its own CUDA
    # events on the launching stream and reports it when residuals are read back
    kern_ms = []
    with torch.cuda.stream(stream):
        for i in range(max(3, min(args.steps, 5))):
            solver.set_points(x)
            resid, _ = solver.picard_sweep(W.K, residuals=True)
            kern_ms.append(solver.diagnostics()["last_ms"])
        st = solver.get_state()
        final_v, final_p = st["v"].cpu().numpy(), st["p"].cpu().numpy()
    total_ms = sum(step_ms)
    if world > 1:
        total_ms = max_over_ranks(total_ms, dev)

    # ---- end to end through the public API with pinned host buffers
    x_host = torch.from_numpy(x_np).pin_memory()
    v_host = torch.empty(W.M, dtype=torch.float64).pin_memory()
    g_host = torch.empty(W.M, W.n, dtype=torch.float32).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    with torch.cuda.stream(stream):
        solver.value_grad(x_host, v_out=v_host, grad_out=g_host)   # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            solver.value_grad(x_host, v_out=v_host, grad_out=g_host)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / e2e_steps
    if world > 1:
        e2e_s = max_over_ranks(e2e_s, dev)
    solver.close()

    samples_per_step = W.M * W.N * W.K
    value = world * samples_per_step * args.steps / (total_ms / 1e3)
    e2e_value = world * samples_per_step / e2e_s
    clocks = clk.summary()
    peaks = load_peaks()
    kern_s = statistics.median(kern_ms) / 1e3
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "step_ms": {"median": statistics.median(step_ms),
                    "iqr": float(np.subtract(*np.percentile(step_ms, [75, 25])))},
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 combine/log/residual)",
        "data": "synthetic (seeded uniform states)",
        "config": {"workload": "rockets6_uniform: 6-D two-rocket game, M=65536 states in "
                               "[-3,3]^4x[-pi,pi]^2, N=65536 samples/state/sweep, K=20 sweeps, "
                               "nu=0.05, T=2",
                   "M": W.M, "N": W.N, "K": W.K, "l2": "flushed (256 MB write) between steps",
                   "launch": {"variant": tuned["variant"], "threads": tuned["threads"]},
                   "parallelism": "independent instance per GPU" if world > 1 else "1 GPU"},
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": int(x_np.nbytes),
                "d2h_bytes_per_step": int(W.M * 8 + W.M * W.n * 4 + W.K * 8)},
        "gpu_launches": 3 * args.steps,
        "roofline": dict(roofline(W.game, samples_per_step, kern_s, states=W.M),
                         kernel_ms_per_step=statistics.median(kern_ms)),
        "clocks": clocks,
        "hbm_peak_gbs_measured": peaks.get("hbm_gbs"),
        "residuals": [float(r) for r in resid],
        "sweeps_to_floor": sweeps_to_floor(resid),
        "paper_context": PAPER_CONTEXT,
    }
    out["_final"] = (final_v, final_p)
    return out


def sweeps_to_floor(resid):
    """Residual floor = median of the last three sweeps' residuals; sweeps to the floor =
    first sweep whose residual is within 10 % of it."""
    r = np.asarray(resid, dtype=np.float64)
    floor = float(np.median(r[-3:]))
    k = int(np.nonzero(r <= 1.1 * floor)[0][0]) + 1
    return {"floor": floor, "sweeps": k}


def run_cpu_baseline(seconds_target=12.0, rank=0):
    """The FP64 oracle as it stands, on a bounded sample of the workload's states."""
    import oracle
    x = hjg_inputs.points(W)
    P = oracle.make_problem(W.game, W.n, W.delta, W.T, radius=W.radius, seed=0)
    # calibrate: one sweep of one state per thread, then size the timed sample so that the
    # full K-sweep solve takes about seconds_target of wall time on all host threads
    threads = oracle.num_threads()
    probe = hjg_inputs.subset_indices(W.M, threads, seed=4)
    t0 = time.perf_counter()
    oracle.picard(P, x[probe].astype(np.float64), W.N, 1, idx=probe)
    wall_per_state_sweep = max(time.perf_counter() - t0, 1e-4)   # per thread
    m = int(seconds_target / (wall_per_state_sweep * W.K)) * threads
    m = int(min(W.M, max(threads, m)))
    idx = hjg_inputs.subset_indices(W.M, m, seed=5)
    t0 = time.perf_counter()
    ref = oracle.picard(P, x[idx].astype(np.float64), W.N, W.K, idx=idx)
    el = time.perf_counter() - t0
    return {"value": m * W.N * W.K / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d of %d states (seeded subset), full N=%d and K=%d, %.1f s"
                      % (m, W.M, W.N, W.K, el), "elapsed_s": el}, (idx, ref)


def oracle_error(final, sample):
    """The benchmark solve's error against the oracle's FP64 trajectory on the oracle's
    sample of states (same global indices, same draws): per state |dv|/(1+|v|) and
    ||dDv||/(1+||Dv||), and the fraction within the parity tolerance (1e-4, 1e-3)."""
    (v, p), (idx, ref) = final, sample
    dv = np.abs(v[idx] - ref["v"]) / (1.0 + np.abs(ref["v"]))
    dp = np.linalg.norm(p[idx].astype(np.float64) - ref["p"], axis=1) / (1.0 + np.linalg.norm(ref["p"], axis=1))
    ok = (dv <= 1e-4) & (dp <= 1e-3)
    return {"states": int(len(idx)), "within_tolerance": float(ok.mean()),
            "dv_median": float(np.median(dv)), "dv_max": float(dv.max()),
            "dgrad_median": float(np.median(dp)), "dgrad_max": float(dp.max()),
            "tolerance": "|dv| <= 1e-4 (1+|v|), ||dDv|| <= 1e-3 (1+||Dv||) after K sweeps (FP64 oracle trajectory)"}


def ncu_case(w, variant, M=None):
    """A small case of one workload for ncu: M states (default 12 x 152: two waves of the
    CTA-per-state kernels; the warp-per-state kernels need 48 x 152 for one full wave), a
    few MB on the device, the workload's N, two sweeps per launch, launch variant
    `variant`; one warm-up launch, then one profiled launch."""
    import torch
    from paper_2605_18566_gb300 import Solver
    M = M or 12 * SMS
    x = torch.from_numpy(hjg_inputs.points(w, M=M)).cuda()
    s = Solver(w.game, w.nu, w.T, w.N, 2, radius=w.radius, variant=variant)
    for _ in range(2):
        s.set_points(x)
        r, _ = s.picard_sweep(2)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": w.name, "M": M, "N": w.N, "K": 2, "variant": variant,
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
           "config": {"workload": "mixed batch (Dubins 1,024 + 65,536; rockets6 4,096 + "
                                  "131,072; rockets45 16,384 + 262,144 states) + 100,000-agent "
                                  "flock, nu=0.02, T=1, N=16384, K=15, one CUDA-graph launch",
                      "instances": len(inst), "states": sum(M for _, M in inst),
                      "launch": "graph of per-instance sweep + residual kernels (batch)"},
           "clocks": clk.summary()}
    b.close()
    for s in solvers:
        s.close()
    return out


def surrogate_study(points_fn, label):
    """One study of the learned part on the 45-D game: tuples (x, v, Dv) from the plain
    sweeps of 262,144 states drawn by points_fn (sweeps 23-30 of 30 at N = 131,072:
    2,097,152 tuples), GPU training of the 45 -> 256^3 -> 46 BF16 network on them, and, on
    1,024 held-out states, the value error against a tilted N = 2^20 reference for the plain
    form, the tilted form without the network, and the surrogate-assisted form (warm start +
    tilt, with and without the control variate) over N = 4,096 ... 262,144, 12 sweeps each.  `four_x` compares each plain run
    with the assisted run at a quarter of its point-samples: success when the assisted run
    reaches the plain run's residual at no larger value error."""
    import torch
    from paper_2605_18566_gb300 import Solver, Surrogate
    w = hjg_inputs.ROCKETS45
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x = torch.from_numpy(points_fn(w.M, 0)).cuda()
    s = Solver(w.game, w.nu, w.T, w.N, w.K, radius=w.radius)
    s.set_points(x)
    s.autotune(max_states=4 * SMS * 2)
    s.picard_sweep(w.K - 8, residuals=False)
    X, Y = [], []
    resid = []
    for _ in range(8):
        r, _ = s.picard_sweep(1)
        resid.append(float(r[0]))
        st = s.get_state()
        X.append(x)
        Y.append(torch.cat([st["v"][:, None].float(), st["p"]], 1))
    s.close()
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    X = torch.cat(X); Y = torch.cat(Y)
    perm = torch.from_numpy(np.random.default_rng(0).permutation(X.shape[0])).cuda()
    X = X[perm].contiguous(); Y = Y[perm].contiguous()
    sur = Surrogate(45, 46, 256, seed=0)
    epochs, batch = 8, 8192
    torch.cuda.synchronize(); t1 = time.perf_counter()
    hist = sur.fit(X, Y, epochs=epochs, batch=batch, lr=2e-3, lr_final=1e-4)
    torch.cuda.synchronize(); t_train = time.perf_counter() - t1
    xte = torch.from_numpy(points_fn(1024, 1)).cuda()

    def solve(N, K, tilt=False, warm=None, seed=11, cv=False):
        so = Solver(w.game, w.nu, w.T, N, K, radius=w.radius, tilt=tilt, seed=seed, cv=cv)
        so.set_points(xte)
        if warm is not None:
            so.warm_start(warm[1], warm[0])
        r, _ = so.picard_sweep(K)
        st = so.get_state()
        so.close()
        return st["v"].cpu().numpy(), float(r[-1])

    vref, rref = solve(1 << 20, 12, tilt=True, seed=7)
    pred = sur.forward(xte)
    vs, ps = pred[:, 0].double().contiguous(), pred[:, 1:].contiguous()
    rows = []
    K = 12
    for N in (4096, 16384, 65536, 262144):
        for mode in ("plain", "tilt", "surrogate+tilt", "surrogate+tilt+cv"):
            v, r = solve(N, K, tilt=mode != "plain", warm=(vs, ps) if mode.startswith("surrogate") else None,
                         cv=mode.endswith("+cv"))
            rows.append({"mode": mode, "N": N, "K": K, "point_samples_per_state": N * K,
                         "rms_value_error": float(np.sqrt(np.mean((v - vref) ** 2))),
                         "final_residual": r})
    sur.close()
    four_x = []
    for p in rows:
        if p["mode"] != "plain":
            continue
        for a in rows:
            if a["mode"].startswith("surrogate") and a["N"] * 4 == p["N"]:
                four_x.append({"plain_N": p["N"], "assisted": a["mode"], "assisted_N": a["N"],
                               "met": bool(a["final_residual"] <= p["final_residual"]
                                           and a["rms_value_error"] <= p["rms_value_error"])})
    return {"label": label, "tuple_generation_s": t_data, "train_s": t_train,
            "tuples": int(X.shape[0]), "epochs": epochs, "batch": batch,
            "loss": [hist[0], hist[-1]], "data_residuals": resid,
            "reference": {"N": 1 << 20, "K": 12, "tilt": True, "final_residual": rref},
            "surrogate_alone_rms_value_error": float(np.sqrt(np.mean((vs.cpu().numpy() - vref) ** 2))),
            "study": rows, "four_x": four_x}


def run_surrogate(args):
    """The learned part on the 45-D game, on two state distributions: the workload's own
    (positions N(0, 2^2): most states start near a capture) and the paper's wider one
    (positions uniform in [-100, 100]); the line's value is the training throughput of the
    first."""
    w = hjg_inputs.ROCKETS45
    main = surrogate_study(lambda M, seed: hjg_inputs.rockets45_points(M, seed), "positions N(0, 2^2)")
    wide = surrogate_study(lambda M, seed: hjg_inputs.rockets45_wide_points(M, seed),
                           "positions uniform in [-100, 100]")
    flops_per_tuple = 6 * (48 * 256 + 256 * 256 * 2 + 256 * 48)   # forward + backward GEMMs
    tuples = main["tuples"] * main["epochs"]
    tflops = tuples * flops_per_tuple / main["train_s"] / 1e12
    tensor_peak = load_peaks().get("bf16_tflops", 1906.5)
    return {"metric": "surrogate training tuples/s and error vs point-samples (45-D game)",
            "value": tuples / main["train_s"], "unit": "tuples/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "bf16 (FP32 accumulate)", "data": "synthetic (tuples from the plain sweeps)",
            "config": {"workload": "rockets45_gauss sweeps 23-30 -> 2,097,152 tuples; MLP 45-256-256-256-46",
                       "epochs": main["epochs"], "batch": main["batch"]},
            "rockets45_point_samples_per_s": w.M * w.N * w.K / main["tuple_generation_s"],
            "mlp_tflops": tflops,
            "roofline": {"bound": "tensor", "achieved": tflops, "peak": tensor_peak, "unit": "TFLOP/s",
                         "frac": tflops / tensor_peak,
                         "note": "whole training step (GEMMs + element-wise + Adam) at batch 8192"},
            "studies": [main, wide]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="rockets6", choices=["rockets6", "mixed", "surrogate"],
                    help="rockets6 (default, the benchmark line), the mixed batch + flock, or "
                         "the learned part on the 45-D game")
    ap.add_argument("--ncu-case", default=None, choices=list(hjg_inputs.WORKLOADS) + ["surrogate_mlp"],
                    help="run one small launch of the named workload's sweep (profiling)")
    ap.add_argument("--variant", type=int, default=2, help="sweep launch variant for --ncu-case")
    ap.add_argument("--ncu-states", type=int, default=0, help="states of --ncu-case (default 12 x 152)")
    args = ap.parse_args()
    rank, world, local_rank = dist_env()
    if args.ncu_case == "surrogate_mlp":
        ncu_case_surrogate()
        return
    if args.ncu_case:
        ncu_case(hjg_inputs.WORKLOADS[args.ncu_case], args.variant, args.ncu_states or None)
        return

    if args.impl == "reference":
        if rank != 0:
            return
        import oracle
        runs = []
        for i in range(args.warmup + args.steps):
            r = run_cpu_baseline(seconds_target=6.0)[0]
            if i >= args.warmup:
                runs.append(r)
        val = statistics.median(r["value"] for r in runs)
        out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": 1e3 * statistics.median(r["elapsed_s"] for r in runs),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f64", "data": "synthetic (seeded uniform states)",
               "config": {"workload": "rockets6_uniform (bounded CPU sample per step)",
                          "M": W.M, "N": W.N, "K": W.K},
               "cpu_baseline": {"value": val, "unit": UNIT, "cores": runs[0]["cores"],
                                "kind": "oracle", "sample": runs[0]["sample"]},
               "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                       "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return

    if args.workload in ("mixed", "surrogate"):
        if rank == 0:
            print(json.dumps(run_mixed(args) if args.workload == "mixed" else run_surrogate(args)))
        return
    out = run_ours(args, rank, world, local_rank)
    final = out.pop("_final")
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"], sample = run_cpu_baseline()
            out["oracle_error"] = oracle_error(final, sample)
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
