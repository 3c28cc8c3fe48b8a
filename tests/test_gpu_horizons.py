"""Several horizons in one solve on the GPU (hjg_set_horizons).

* Item h M + m equals, bit for bit, a single-horizon solve at T = t_h whose states carry
  the point offset h M (same draws, same arithmetic), for the CTA, warp and 45-D kernels.
* The first sweep at every horizon agrees with the oracle handed the same coefficient (P1),
  and the K-sweep result with the oracle's several-horizon run (P2, same protocol as the
  single-horizon tests: most states within tolerance).
* The flock keeps one neighbour structure for all horizons."""
import numpy as np
import pytest

import hjg_inputs
import oracle
from helpers import assert_parity, problem_for, rel_errors, solver_for

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W1, W2, W3, WF = hjg_inputs.DUBINS3, hjg_inputs.ROCKETS6, hjg_inputs.ROCKETS45, hjg_inputs.FLOCK
TIMES = [0.25, 0.6, 1.0, 1.7]


def _state(s):
    return {k: t.cpu().numpy() for k, t in s.get_state().items()}


@pytest.mark.parametrize("w,M,N,variant", [(W1, 300, 2048, 0), (W1, 300, 2048, 5), (W2, 97, 4096, 2),
                                           (W3, 9, 2048, 0), (WF, 400, 1024, 2)],
                         ids=["dubins3-cta", "dubins3-warp", "rockets6", "rockets45", "flock"])
def test_horizons_equal_offset_single_solves(w, M, N, variant):
    x = torch.from_numpy(hjg_inputs.points(w, M=M)).cuda()
    K = 3
    s = solver_for(w, N=N, K=K, variant=variant)
    s.set_horizons(TIMES)
    s.set_points(x)
    s.picard_sweep(K)
    multi = _state(s)
    s.close()
    assert multi["v"].shape[0] == len(TIMES) * M
    for h, t in enumerate(TIMES):
        from paper_2605_18566_gb300 import Solver
        one = Solver(w.game, w.nu, t, N, K, radius=w.radius, variant=variant, point_offset=h * M)
        one.set_points(x)
        one.picard_sweep(K)
        st = _state(one)
        one.close()
        sl = slice(h * M, (h + 1) * M)
        for key in ("v", "p", "c", "ess"):
            np.testing.assert_array_equal(multi[key][sl], st[key], err_msg="%s horizon %d" % (key, h))


def test_horizons_parity_with_oracle():
    w, M, N, K = W1, 512, 4096, 4
    xn = hjg_inputs.points(w, M=M)
    s = solver_for(w, N=N, K=K)
    s.set_horizons(TIMES)
    s.set_points(torch.from_numpy(xn).cuda())
    st0 = _state(s)
    s.picard_sweep(1)
    st1 = _state(s)
    P = problem_for(w)
    xd = xn.astype(np.float64)
    T0 = P.T
    for h, t in enumerate(TIMES):   # P1 at every horizon
        sl = slice(h * M, (h + 1) * M)
        P.T = t
        v, p, _ = oracle.sweep(P, xd, st0["c"][sl].astype(np.float64), N, 0, idx=h * M + np.arange(M))
        assert_parity(st1["v"][sl], st1["p"][sl], v, p, what="P1 horizon %g" % t)
    P.T = T0
    s.set_points(torch.from_numpy(xn).cuda())
    r, sup = s.picard_sweep(K)
    st = _state(s)
    s.close()
    ref = oracle.picard_horizons(P, xd, N, K, TIMES)
    dv, dp = rel_errors(st["v"], st["p"], ref["v"], ref["p"])
    ok = (dv <= 1e-4) & (dp <= 1e-3)
    assert ok.mean() >= 0.97, ok.mean()
    np.testing.assert_allclose(r, ref["resid"], rtol=5e-3, atol=1e-7)
