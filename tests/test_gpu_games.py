"""The appendix's relative two-rocket game and double integrator on the GPU against the FP64
oracle (same P1 / Gamma / P2 protocol as the other games), and the double integrator at its
three horizons in one solve."""
import numpy as np
import pytest

import hjg_inputs
import oracle
from helpers import check_trajectory, problem_for, rel_errors, solver_for

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WR, WD = hjg_inputs.ROCKETS_REL3, hjg_inputs.DOUBLE_INT2


@pytest.mark.parametrize("w,step,N,K", [(WR, 97, 14000, 4), (WD, 8, 8000, 5)],
                         ids=["rockets_rel3", "double_int2"])
def test_trajectory_parity(w, step, N, K):
    x = hjg_inputs.points(w)[::step].copy()
    out = check_trajectory(w, x, N, K, min_pass=0.97 if len(x) > 200 else 0.9)
    assert np.isfinite(out["resid"]).all()


def test_double_integrator_horizons():
    w = WD
    x = hjg_inputs.points(w)[::16].copy()
    M, N, K = len(x), w.N, 6
    times = list(hjg_inputs.DOUBLE_INT2_HORIZONS)
    s = solver_for(w, N=N, K=K)
    s.set_horizons(times)
    s.set_points(torch.from_numpy(x).cuda())
    r, sup = s.picard_sweep(K)
    st = {k: t.cpu().numpy() for k, t in s.get_state().items()}
    s.close()
    ref = oracle.picard_horizons(problem_for(w), x.astype(np.float64), N, K, times)
    dv, dp = rel_errors(st["v"], st["p"], ref["v"], ref["p"])
    assert ((dv <= 1e-4) & (dp <= 1e-3)).mean() >= 0.97
    np.testing.assert_allclose(r, ref["resid"], rtol=5e-3, atol=1e-7)
