"""The murmuration game on the GPU: exact 7-nearest-neighbour search and mean headings
against the oracle's k-d tree, and the per-agent Picard sweep against the oracle."""
import numpy as np
import pytest

import hjg_inputs
import oracle
from helpers import check_trajectory

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W = hjg_inputs.FLOCK


@pytest.mark.parametrize("M", [8, 1000, 20000])
def test_neighbours_match_kdtree(M):
    from paper_2605_18566_gb300 import flock_neighbours
    x = hjg_inputs.flock_states(M, seed=3)
    idx, psibar = flock_neighbours(torch.from_numpy(x).cuda())
    idx = idx.cpu().numpy(); psibar = psibar.cpu().numpy()
    ref_idx, _, ref_pb = oracle.flock_neighbours(x)
    pos = x[:, :3].astype(np.float64)
    same = np.all(np.sort(idx, 1) == np.sort(ref_idx, 1), axis=1)
    for i in np.nonzero(~same)[0]:      # only near-ties at the 7th neighbour may differ
        dg = np.sort(np.linalg.norm(pos[idx[i]] - pos[i], axis=1))
        dr = np.sort(np.linalg.norm(pos[ref_idx[i]] - pos[i], axis=1))
        np.testing.assert_allclose(dg, dr, rtol=1e-5)
    assert same.mean() > 0.999
    ok = same
    dpsi = np.angle(np.exp(1j * (psibar[ok].astype(np.float64) - ref_pb[ok])))
    assert np.abs(dpsi).max() < 1e-5
    # each agent's list is ordered by distance and excludes the agent
    assert np.all(idx != np.arange(M)[:, None])
    d = np.linalg.norm(pos[idx] - pos[:, None, :], axis=2)
    assert np.all(np.diff(d, axis=1) >= -1e-6)


def test_flock_trajectory_parity():
    x = hjg_inputs.flock_states(2000, seed=5)
    check_trajectory(W, x, 4096, 4)


def test_flock_full_size_sampled():
    """100,000 agents (neighbours among all of them), the workload's N and all its sweeps;
    a seeded subset of agents is recomputed by the oracle."""
    x = hjg_inputs.points(W)
    idx = hjg_inputs.subset_indices(W.M, 24, seed=8)
    check_trajectory(W, x, W.N, W.K, idx=idx, min_pass=0.9, rows_only=True)


def test_neighbours_and_solve_with_non_finite_agents():
    """A NaN position never qualifies as a neighbour: other agents' lists skip it, its own
    list is empty (-1, psibar NaN), and where fewer than 7 finite agents remain the empty
    slots are -1.  A solve reports such agents as non-finite and leaves the rest finite."""
    from paper_2605_18566_gb300 import _lib, flock_neighbours
    from helpers import solver_for
    x = hjg_inputs.flock_states(100, seed=4)
    x[5, 0] = np.nan
    idx, pb = flock_neighbours(torch.from_numpy(x).cuda())
    idx = idx.cpu().numpy(); pb = pb.cpu().numpy()
    assert np.all(idx[5] == -1) and np.isnan(pb[5])
    pos = x[:, :3].astype(np.float64)
    for i in range(100):
        if i == 5:
            continue
        d = np.linalg.norm(pos - pos[i], axis=1)
        d[i] = np.inf; d[5] = np.inf
        assert 5 not in idx[i] and np.all(idx[i] >= 0)
        np.testing.assert_allclose(np.sort(d[idx[i]]), np.sort(d)[:7], rtol=1e-5)
        assert np.isfinite(pb[i])
    y = hjg_inputs.flock_states(12, seed=6)
    y[:6, 1] = np.nan
    idx2, pb2 = flock_neighbours(torch.from_numpy(y).cuda())
    idx2 = idx2.cpu().numpy(); pb2 = pb2.cpu().numpy()
    assert np.all(idx2[:6] == -1)
    for i in range(6, 12):   # five finite others, then two empty slots
        assert sorted(idx2[i][:5]) == sorted(j for j in range(6, 12) if j != i)
        assert np.all(idx2[i][5:] == -1) and np.isnan(pb2[i])
    s = solver_for(W, N=1024, K=2)
    s.set_points(torch.from_numpy(x).cuda())
    s.picard_sweep(2)
    st = {k: t.cpu().numpy() for k, t in s.get_state().items()}
    status = s.last_status
    s.close()
    assert status == _lib.HJG_ENONFINITE
    assert not np.isfinite(st["v"][5])
    keep = np.arange(100) != 5
    assert np.all(np.isfinite(st["v"][keep])) and np.all(np.isfinite(st["p"][keep]))
