"""The reach-avoid obstacle on the GPU against the oracle (same P1 / Gamma / P2 protocol as
the other games): the avoid disc enters the datum of every sweep as max{l, o} and bounds
the value from below after every sweep.  The value never
falls below the obstacle's constraint function, every launch variant agrees with the
oracle, and games without a position plane refuse the option."""
import numpy as np
import pytest

import hjg_inputs
from helpers import check_trajectory, solver_for

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W1, WR, WD = hjg_inputs.DUBINS3, hjg_inputs.ROCKETS_REL3, hjg_inputs.DOUBLE_INT2
OBST = {"dubins3": (0.8, 0.3, 0.6), "rockets_rel3": (20.0, -10.0, 15.0), "double_int2": (0.6, -0.4, 0.35)}


@pytest.mark.parametrize("w,step,N,K,tilt", [(W1, 9, 4096, 5, False), (W1, 9, 4096, 5, True),
                                             (WR, 97, 14000, 4, False), (WD, 8, 8000, 5, False)],
                         ids=["dubins3", "dubins3-tilt", "rockets_rel3", "double_int2"])
def test_obstacle_trajectory_parity(w, step, N, K, tilt):
    x = hjg_inputs.points(w)[::step].copy()
    out = check_trajectory(w, x, N, K, tilt=tilt, obstacle=OBST[w.game],
                           min_pass=0.97 if len(x) > 200 else 0.9)
    cx, cy, r = OBST[w.game]
    o = r - np.hypot(x[:, 0] - cx, x[:, 1] - cy)
    for st in out["states"]:
        assert np.all(st["v"] >= o - 1e-6 * (1 + np.abs(o)))
    inside = o > 0
    assert inside.any() and np.all(out["states"][-1]["v"][inside] > 0)


def test_obstacle_every_variant_matches_the_oracle():
    """CTA- and warp-per-state kernels, plain, pipelined and two-group samplers: one sweep
    with the obstacle agrees with the oracle's sweep from the same coefficients."""
    import oracle
    from helpers import assert_parity, problem_for
    xs = hjg_inputs.points(W1)[::5].copy()
    x = torch.from_numpy(xs).cuda()
    for v in (0, 3, 5, 9):
        s = solver_for(W1, N=2048, K=1, variant=v, obstacle=OBST["dubins3"])
        s.set_points(x)
        c0 = s.get_state()["c"].cpu().numpy().astype(np.float64)
        s.picard_sweep(1)
        st = {k: t.cpu().numpy() for k, t in s.get_state().items()}
        s.close()
        vr, pr, _ = oracle.sweep(problem_for(W1, obstacle=OBST["dubins3"]), xs.astype(np.float64), c0, 2048, 0)
        assert_parity(st["v"], st["p"], vr, pr, what="obstacle, variant %d" % v)


def test_obstacle_refused_without_a_position_plane():
    from paper_2605_18566_gb300 import HJGError
    with pytest.raises(HJGError):
        solver_for(hjg_inputs.ROCKETS6, N=1024, K=1, obstacle=(0.0, 0.0, 1.0))
