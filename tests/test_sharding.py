"""Sharding one state set over ranks: contiguous blocks, Philox counters offset by the
block's first global index, and one all-reduce of the residual parts per solve.  Run with
two gloo ranks on the CPU; each rank's share is computed by the FP64 oracle, and the
combined residuals and per-state values must equal the unsharded solve."""
import os
import socket

import numpy as np
import pytest

import hjg_inputs
from paper_2605_18566_gb300 import sharding


def test_shard_bounds_cover_exactly():
    for M in (0, 1, 7, 100, 4097):
        for world in (1, 2, 3, 8):
            blocks = [sharding.shard_bounds(M, world, r) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == M
            assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
            sizes = [h - l for l, h in blocks]
            assert max(sizes) - min(sizes) <= 1


def _parts(v_hist):
    dv = np.diff(v_hist, axis=0)
    return np.stack([(dv ** 2).sum(1), (v_hist[:-1] ** 2).sum(1), np.abs(dv).max(1)], 1)


def _rank_main(rank, world, port, M, N, K, out_dir):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = hjg_inputs.DUBINS3
    x = hjg_inputs.points(w)[:M].astype(np.float64)
    lo, hi = sharding.shard_bounds(M, world, rank)
    P = oracle.make_problem(w.game, w.n, w.delta, w.T, radius=w.radius)
    out = oracle.picard(P, x[lo:hi], N, K, idx=np.arange(lo, hi))
    rel, sup = sharding.combine_residual_parts(_parts(out["v_hist"]))
    np.savez(os.path.join(out_dir, "rank%d.npz" % rank), rel=rel, sup=sup, v=out["v"], lo=lo, hi=hi)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_solve_equals_unsharded(tmp_path):
    import torch.multiprocessing as mp
    import oracle
    M, N, K, world = 301, 512, 3, 2
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_rank_main, args=(world, port, M, N, K, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    w = hjg_inputs.DUBINS3
    x = hjg_inputs.points(w)[:M].astype(np.float64)
    P = oracle.make_problem(w.game, w.n, w.delta, w.T, radius=w.radius)
    full = oracle.picard(P, x, N, K)
    rs = [np.load(tmp_path / ("rank%d.npz" % r)) for r in range(world)]
    for r in rs:
        np.testing.assert_allclose(r["rel"], full["resid"], rtol=1e-12)
        np.testing.assert_allclose(r["sup"], full["sup"], rtol=0, atol=0)
    v = np.concatenate([r["v"] for r in rs])
    np.testing.assert_array_equal(v, full["v"])


def _combine_main(rank, world, port, parts_all, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rel, sup = sharding.combine_residual_parts(parts_all[rank])
    np.savez(os.path.join(out_dir, "c%d.npz" % rank), rel=rel, sup=sup)
    dist.barrier()
    dist.destroy_process_group()


def test_three_ranks_one_empty_shard():
    """More ranks than a shard has states: an empty rank contributes zero sums and a zero
    maximum (what hjg_get_residual_parts leaves after a sweep over no states), and every
    rank ends with the residual of the states that exist."""
    import tempfile
    import torch.multiprocessing as mp
    M, world = 2, 3
    assert [sharding.shard_bounds(M, world, r) for r in range(world)] == [(0, 1), (1, 2), (2, 2)]
    rng = np.random.default_rng(3)
    K = 4
    v_hist = rng.normal(size=(K + 1, M)) + 2.0
    parts_all = [_parts(v_hist[:, r:r + 1]) for r in range(2)] + [np.zeros((K, 3))]
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_combine_main, args=(world, port, parts_all, d), nprocs=world,
                           start_method="spawn", join=True)
        want = _parts(v_hist)
        for r in range(world):
            got = np.load(os.path.join(d, "c%d.npz" % r))
            np.testing.assert_allclose(got["rel"], np.sqrt(want[:, 0] / want[:, 1]), rtol=1e-14)
            np.testing.assert_array_equal(got["sup"], want[:, 2])


@pytest.mark.gpu
@pytest.mark.parametrize("world", [2, 3])
def test_gpu_shards_reproduce_unsharded_solve(world):
    """Each shard, solved alone with its point offset, draws the unsharded solve's samples:
    the per-state values and gradients agree bit for bit, and the all-reduced residual
    parts give the unsharded residual (up to the order of the FP64 sums)."""
    torch = pytest.importorskip("torch")
    from helpers import solver_for
    w = hjg_inputs.ROCKETS6
    M, N, K = 3001, 4096, 4
    x = torch.from_numpy(hjg_inputs.points(w, M=M)).cuda()
    full = solver_for(w, N=N, K=K)
    full.set_points(x)
    r_full, sup_full = full.picard_sweep(K)
    ref = {k: t.cpu().numpy() for k, t in full.get_state().items()}
    full.close()
    parts, vs, ps = [], [], []
    for rank in range(world):
        lo, hi = sharding.shard_bounds(M, world, rank)
        s = solver_for(w, N=N, K=K, point_offset=lo)
        s.set_points(x[lo:hi].contiguous())
        s.picard_sweep(K)
        parts.append(s.residual_parts(K))
        st = s.get_state()
        vs.append(st["v"].cpu().numpy()); ps.append(st["p"].cpu().numpy())
        s.close()
    np.testing.assert_array_equal(np.concatenate(vs), ref["v"])
    np.testing.assert_array_equal(np.concatenate(ps), ref["p"])
    P = np.stack(parts)
    rel = np.sqrt(P[:, :, 0].sum(0)) / np.sqrt(P[:, :, 1].sum(0))
    np.testing.assert_allclose(rel, r_full, rtol=1e-12)
    np.testing.assert_array_equal(P[:, :, 2].max(0), sup_full)
