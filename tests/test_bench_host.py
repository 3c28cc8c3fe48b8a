"""Host logic of the benchmark (no GPU): the per-point-sample work constants agree with the
sampler's stream layout as the oracle defines it, the residual-floor and oracle-error
summaries behave on synthetic inputs, and the reference arm prints the contract's line."""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import bench
import hjg_inputs
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("game,n", [("dubins3", 3), ("rockets6", 6), ("rockets45", 45)])
def test_work_constants_follow_the_stream_layout(game, n):
    # Philox blocks per sample: slots per sample over the eight normals a block yields
    assert bench.BLOCKS_PER_SAMPLE[game] == pytest.approx(oracle.slot_stride(n) / 8.0)
    # MUFU: lg2 and sqrt per Box-Muller pair of the n normals used (cos and sin from the
    # angle table), one square root for the target distance, one exp2 weight at half cost
    assert bench.MUFU_PER_SAMPLE[game] == n + 1.5
    # the transcendental evaluations with cos and sin on the MUFU pipe
    assert bench.MUFU_EQUIV_PER_SAMPLE[game] == 4 * n / 2 + 1.5


def test_roofline_picks_the_binding_pipe():
    clk = bench.SMS * bench.SM_MAX_MHZ * 1e6
    samples = 1e12
    # a time at which the MUFU pipe runs exactly at its peak
    t = samples * bench.MUFU_PER_SAMPLE["rockets6"] / (bench.MUFU_PER_SM_CLK * clk)
    r = bench.roofline("rockets6", samples, t)
    assert r["pipe"] == "mufu" and r["bound"] == "alu"
    assert r["frac"] == pytest.approx(1.0)
    assert r["other_pipes"]["int_mul_hi"] < 1.0 and "issue" not in r["other_pipes"]
    assert r["mufu_equivalent_frac"] == pytest.approx(13.5 / 7.5, rel=1e-3)
    assert r["traffic"] is None                      # not a full-size launch
    r2 = bench.roofline("rockets6", hjg_inputs.ROCKETS6.M * 10, 1.0, full_size=True)
    assert r2["traffic"] == bench.DRAM_BYTES_LAUNCH.get("rockets6")
    # with a measured instruction count the issue port joins, and binds where it is closest
    v = 7
    t_issue = samples * bench.INSTR_PER_SAMPLE["rockets6"][v] / (bench.ISSUE_PER_SM_CLK * clk)
    r3 = bench.roofline("rockets6", samples, t_issue, variant=v)
    assert r3["pipe"] == "issue" and r3["frac"] == pytest.approx(1.0)
    assert r3["ops_per_point_sample"] == pytest.approx(bench.INSTR_PER_SAMPLE["rockets6"][v])
    # every launch variant of every counted game has its measured instruction count
    for game, counts in bench.INSTR_PER_SAMPLE.items():
        assert game in bench.BLOCKS_PER_SAMPLE and set(counts) == set(range(12)), game
        # the sampler alone is at least n normals of work per sample
        assert all(c > bench.GAME_N[game] for c in counts.values()), game


def test_sweeps_to_floor():
    r = [0.5, 0.2, 0.11, 0.1, 0.1, 0.1]
    out = bench.sweeps_to_floor(r)
    assert out["floor"] == pytest.approx(0.1)
    assert out["sweeps"] == 3                        # |0.11 - 0.1| <= 0.1 * 0.1
    assert bench.sweeps_to_floor([0.3, 0.3, 0.3])["sweeps"] == 1
    # a residual that dips and then rises back settles only where it enters the band for good
    rise = [0.418, 0.097, 0.103, 0.118, 0.135, 0.150, 0.159, 0.163, 0.170, 0.178, 0.176, 0.178]
    out = bench.sweeps_to_floor(rise)
    assert out["floor"] == pytest.approx(0.178)
    assert out["sweeps"] == 8                        # band [0.160, 0.196]: 0.163 onward
    assert out["min"] == pytest.approx(0.097) and out["min_sweep"] == 2
    # the last residual is outside the band: not settled (K + 1)
    out = bench.sweeps_to_floor([1.0, 0.5, 0.25, 0.125, 0.3, 0.05])
    assert out["sweeps"] == 7 and not out["settled"]


def test_oracle_error_summary():
    """One state moved far off the oracle's trajectory: counted outside the tolerance and
    classified (explained or not) by the oracle's own sensitivity there."""
    import dataclasses
    w = dataclasses.replace(hjg_inputs.DUBINS3, N=256, K=2)
    x = hjg_inputs.points(w)
    idx = hjg_inputs.subset_indices(w.M, 20, seed=3)
    P = oracle.make_problem(w.game, w.n, w.delta, w.T, radius=w.radius)
    ref = oracle.picard(P, x[idx].astype(np.float64), w.N, w.K, idx=idx)
    v = np.zeros(w.M); p = np.zeros((w.M, w.n), np.float32)
    v[idx] = ref["v"]; p[idx] = ref["p"]
    v[idx[3]] += 1.0                                 # one state far outside the tolerance
    out = bench.oracle_error((v, p), (idx, ref, P, x), w)
    assert out["states"] == 20
    assert out["within_tolerance"] == pytest.approx(19 / 20)
    assert out["dv_max"] == pytest.approx(1.0 / (1.0 + abs(ref["v"][3])))
    assert out["outside_tolerance"] == 1 and out["explained"] + out["unexplained"] == 1


@pytest.mark.timeout(600)
def test_reference_arm_prints_the_contract_line():
    proc = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                          timeout=600, cwd=ROOT)
    assert proc.returncode == 0, proc.stderr[-2000:]
    line = json.loads(proc.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and math.isfinite(line["value"])
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def _max_rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = bench.max_over_ranks(10.0 + 7.5 * rank, "cpu")   # rank 1 is the slow one
    with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
        f.write(repr(got))
    dist.barrier()
    dist.destroy_process_group()


def test_timing_is_the_maximum_over_two_gloo_ranks(tmp_path):
    """The multi-GPU bench divides the work of all ranks by the slowest rank's time: every
    rank must see the same maximum."""
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_max_rank_main, args=(2, port, str(tmp_path)), nprocs=2,
                       start_method="spawn", join=True)
    for r in range(2):
        assert float(open(tmp_path / ("rank%d.txt" % r)).read()) == 17.5


@pytest.mark.timeout(600)
def test_reference_arm_under_torchrun_prints_once():
    """Launched by torchrun on two ranks, the reference arm runs on rank 0 alone and prints
    one line; the other rank exits 0 without work."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    proc = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert proc.returncode == 0, proc.stderr[-2000:]
    lines = [l for l in proc.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, proc.stdout[-2000:]
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0


def test_paper_context_is_the_derived_rate():
    # rockets slices: 1,600 states x N = 14,000 x 12 sweeps in 13.5 s; Dubins: N = 20,000,
    # 15 sweeps in 23.6 s
    for rate in (1600 * 14000 * 12 / 13.5, 1600 * 20000 * 15 / 23.6):
        assert bench.PAPER_CONTEXT["value"] == pytest.approx(rate, rel=0.02)
    json.dumps(bench.PAPER_CONTEXT)


def test_clock_summary_parses_the_sampled_lines():
    cs = bench.ClockSampler(0)
    assert cs.summary()["reasons"] == ["unsampled"]
    cs.lines = ["0, 2070, 2070, 910.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
                "0, 1995, 2070, 1395.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
                "0, 2070, 2070, 1390.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
                "garbage", "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    cs.lines.append("0, 1500, 2070, 1400, 0x8, Active, Not Active, Active, Not Active")
    assert bench.ClockSampler.summary(cs)["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def _shard_rank_main(rank, world, port, out_dir):
    """One gloo rank of the benchmark's sharded solve, its block computed by the oracle."""
    import dataclasses
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = dataclasses.replace(hjg_inputs.ROCKETS6, M=203, N=512, K=3)
    x = hjg_inputs.points(w, M=w.M).astype(np.float64)
    P = oracle.make_problem(w.game, w.n, w.delta, w.T, radius=w.radius)

    def solve_parts(lo, hi):
        out = oracle.picard(P, x[lo:hi], w.N, w.K, idx=np.arange(lo, hi))
        vh = out["v_hist"]
        dv = np.diff(vh, axis=0)
        parts = np.stack([(dv ** 2).sum(1), (vh[:-1] ** 2).sum(1), np.abs(dv).max(1)], 1)
        return parts, out["v"]
    lo, hi, rel, sup, v = bench.shard_solve(solve_parts, w.M, world, rank)
    np.savez(os.path.join(out_dir, "rank%d.npz" % rank), rel=rel, sup=sup, v=v, lo=lo, hi=hi)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_bench_solve_equals_unsharded(tmp_path, world):
    """The benchmark's multi-GPU path (contiguous blocks, Philox point offset, one
    all-reduce of the residual parts) on gloo ranks whose blocks the oracle solves: every
    rank holds the unsharded solve's residuals and its block's values bit for bit."""
    import dataclasses
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_shard_rank_main, args=(world, port, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    w = dataclasses.replace(hjg_inputs.ROCKETS6, M=203, N=512, K=3)
    x = hjg_inputs.points(w, M=w.M).astype(np.float64)
    P = oracle.make_problem(w.game, w.n, w.delta, w.T, radius=w.radius)
    full = oracle.picard(P, x, w.N, w.K)
    covered = 0
    for r in range(world):
        d = np.load(tmp_path / ("rank%d.npz" % r))
        np.testing.assert_allclose(d["rel"], full["resid"], rtol=1e-12)
        np.testing.assert_allclose(d["sup"], full["sup"], rtol=1e-12)
        np.testing.assert_array_equal(d["v"], full["v"][int(d["lo"]):int(d["hi"])])
        covered += int(d["hi"]) - int(d["lo"])
    assert covered == w.M
