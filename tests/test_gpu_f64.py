"""The FP64-throughout sweep (precision="fp64": normals, samples, target, log-weights and
sums in double precision; the "FP64 samples" of the 3-D workload) against the oracle:
one sweep agrees to rounding (~1e-12, far inside the FP32 path's tolerance), whole
trajectories pass the usual protocol, the FP32 path stays within its tolerance of it, and
the options it does not support are refused."""
import numpy as np
import pytest

import hjg_inputs
import oracle
from helpers import check_trajectory, problem_for, rel_errors, solver_for

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W1, W2, WF = hjg_inputs.DUBINS3, hjg_inputs.ROCKETS6, hjg_inputs.FLOCK


def _one_sweep(w, xs, N, precision, tilt=False, **kw):
    s = solver_for(w, N=N, K=1, precision=precision, tilt=tilt, **kw)
    s.set_points(torch.from_numpy(xs).cuda())
    st0 = {k: t.cpu().numpy() for k, t in s.get_state().items()}
    s.picard_sweep(1)
    st = {k: t.cpu().numpy() for k, t in s.get_state().items()}
    s.close()
    return st0, st


@pytest.mark.parametrize("w,step,N,tilt,kw", [(W1, 4, 4096, False, {}), (W1, 4, 4096, True, {}),
                                              (W2, 512, 65536, False, {}),
                                              (W1, 4, 4096, False, {"obstacle": (0.8, 0.3, 0.6)})],
                         ids=["dubins3", "dubins3-tilt", "rockets6", "dubins3-obstacle"])
def test_one_sweep_matches_the_oracle_to_rounding(w, step, N, tilt, kw):
    xs = hjg_inputs.points(w)[::step].copy()
    st0, st = _one_sweep(w, xs, N, "fp64", tilt=tilt, **kw)
    c0 = st0["c"].astype(np.float64)
    theta = -w.sigma2 * c0[:, None] * st0["p"].astype(np.float64) if tilt else None
    v, p, ess = oracle.sweep(problem_for(w, **kw), xs.astype(np.float64), c0, N, 0, theta=theta)
    dv, dp = rel_errors(st["v"], st["p"], v, p)
    assert dv.max() < 1e-10, dv.max()
    assert dp.max() < 1e-6, dp.max()            # Dv is stored in FP32
    np.testing.assert_allclose(st["ess"], ess, rtol=1e-6)


def test_flock_one_sweep_fp64():
    x = hjg_inputs.flock_states(600, seed=9)
    _, nb, pb = oracle.flock_neighbours(x)
    st0, st = _one_sweep(WF, x, 4096, "fp64")
    c0 = st0["c"].astype(np.float64)
    v, p, _ = oracle.sweep(problem_for(WF), x.astype(np.float64), c0, 4096, 0, nbr=nb)
    dv, dp = rel_errors(st["v"], st["p"], v, p)
    assert dv.max() < 1e-10 and dp.max() < 1e-6, (dv.max(), dp.max())


def test_dubins_workload_trajectory_fp64():
    """The 3-D workload as specified (4,096 grid states, N = 4,096 FP64 samples, 10 sweeps)."""
    x = hjg_inputs.points(W1)
    out = check_trajectory(W1, x, W1.N, W1.K, precision="fp64")
    assert out["pass_fraction"] > 0.99


def test_fp32_path_within_tolerance_of_fp64():
    xs = hjg_inputs.points(W2, M=512)
    _, a = _one_sweep(W2, xs, 65536, "fp64")
    _, b = _one_sweep(W2, xs, 65536, "fp32")
    dv, dp = rel_errors(b["v"], b["p"], a["v"], a["p"].astype(np.float64))
    assert dv.max() <= 1e-4 and dp.max() <= 1e-3, (dv.max(), dp.max())
    assert np.median(dv) < 1e-6


def test_unsupported_combinations_are_refused():
    from paper_2605_18566_gb300 import HJGError
    with pytest.raises(HJGError):
        solver_for(hjg_inputs.ROCKETS45, N=1024, K=1, precision="fp64")
    s = solver_for(W1, N=1024, K=1, precision="fp64", cv=True)
    with pytest.raises(HJGError):   # refused when the sweep is launched
        s.set_points(torch.from_numpy(hjg_inputs.points(W1, M=8)).cuda())
        s.picard_sweep(1)
    s.close()
