"""Mixed-game batches advanced by one CUDA-graph launch: every instance must come out
bit-identical to the same instance run on its own (same kernels, same draws), across two
consecutive runs (the second run updates the instantiated graph)."""
import numpy as np
import pytest

import hjg_inputs
import oracle
from helpers import assert_parity, problem_for, solver_for

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [(hjg_inputs.DUBINS3, 1000, 4096), (hjg_inputs.ROCKETS6, 700, 8192),
         (hjg_inputs.ROCKETS45, 50, 4096)]


def test_batch_matches_individual_runs():
    from paper_2605_18566_gb300 import Batch
    xs = [torch.from_numpy(hjg_inputs.points(w, M=M)).cuda() for w, M, _ in CASES]
    solo = []
    for (w, M, N), x in zip(CASES, xs):
        s = solver_for(w, N=N, K=3, instance=7)
        s.set_points(x)
        r1, _ = s.picard_sweep(3)
        r2, _ = s.picard_sweep(3)
        solo.append(({k: t.cpu() for k, t in s.get_state().items()}, np.concatenate([r1, r2])))
        s.close()
    solvers = []
    for (w, M, N), x in zip(CASES, xs):
        s = solver_for(w, N=N, K=3, instance=7)
        s.set_points(x)
        solvers.append(s)
    b = Batch(solvers)
    ra, ms_a = b.run(3)
    rb, ms_b = b.run(3)
    assert ms_a > 0 and ms_b > 0
    for i, s in enumerate(solvers):
        st = {k: t.cpu() for k, t in s.get_state().items()}
        for key in ("v", "p", "c"):
            assert torch.equal(st[key], solo[i][0][key]), (i, key)
        np.testing.assert_array_equal(np.concatenate([ra[i], rb[i]]), solo[i][1])
    b.close()
    for s in solvers:
        s.close()


def test_batch_instances_against_oracle():
    from paper_2605_18566_gb300 import Batch
    solvers, xs = [], []
    for w, M, N in CASES:
        x = hjg_inputs.points(w, M=min(M, 64))
        s = solver_for(w, N=N, K=2)
        s.set_points(torch.from_numpy(x).cuda())
        solvers.append(s); xs.append(x)
    b = Batch(solvers)
    r, _ = b.run(2)
    for (w, M, N), s, x, ri in zip(CASES, solvers, xs, r):
        st = {k: t.cpu().numpy() for k, t in s.get_state().items()}
        ref = oracle.picard(problem_for(w), x.astype(np.float64), N, 2)
        assert_parity(st["v"], st["p"], ref["v"], ref["p"], frac=0.95, what="batch %s" % w.game)
        np.testing.assert_allclose(ri, ref["resid"], rtol=1e-2)
    b.close()
    for s in solvers:
        s.close()
