"""Degenerate and edge cases of the sweep against the oracle: one sample per state (ESS = 1),
a single state, states far from the target (weights spanning hundreds of orders of
magnitude, handled by the running log-sum-exp shift), coefficients pinned at the clip
bounds, and a non-finite state that is reported (HJG_ENONFINITE) without disturbing the
others."""
import numpy as np
import pytest

import hjg_inputs
import oracle
from helpers import assert_parity, check_trajectory, problem_for, solver_for

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W1, W2 = hjg_inputs.DUBINS3, hjg_inputs.ROCKETS6


def _run(w, x, N, K, **kw):
    s = solver_for(w, N=N, K=K, **kw)
    s.set_points(torch.from_numpy(np.ascontiguousarray(x)).cuda())
    r, sup = s.picard_sweep(K)
    st = {k: t.cpu().numpy() for k, t in s.get_state().items()}
    d = s.diagnostics()
    status = s.last_status
    s.close()
    return st, r, d, status


@pytest.mark.parametrize("N", [1, 2, 5])
def test_tiny_sample_counts(N):
    x = hjg_inputs.points(W1, M=200)
    out = check_trajectory(W1, x, N, 3, min_pass=0.9)
    if N == 1:
        np.testing.assert_allclose(out["states"][-1]["ess"], 1.0, rtol=1e-6)


def test_single_state_many_sweeps():
    x = hjg_inputs.points(W2, M=1)
    st, r, d, _ = _run(W2, x, 65536, 8)
    ref = oracle.picard(problem_for(W2), x.astype(np.float64), 65536, 8)
    assert_parity(st["v"], st["p"], ref["v"], ref["p"], what="M=1")
    np.testing.assert_allclose(r, ref["resid"], rtol=1e-3)


def test_far_states_and_clipped_coefficients():
    """States 50-5000 units from the capture disc: c is at its clip bound (|c| = 1e2/delta)
    and c l(y) reaches ~1e5, so the weights span far beyond FP32 range before the shift."""
    rng = np.random.default_rng(5)
    M = 64
    rad = np.exp(rng.uniform(np.log(50.0), np.log(5000.0), M))
    ang = rng.uniform(-np.pi, np.pi, M)
    x = np.stack([rad * np.cos(ang), rad * np.sin(ang), rng.uniform(-np.pi, np.pi, M)], 1).astype(np.float32)
    st, r, d, _ = _run(W1, x, 4096, 3)
    ref = oracle.picard(problem_for(W1), x.astype(np.float64), 4096, 3)
    assert np.all(np.isfinite(st["v"])) and np.all(np.isfinite(st["p"]))
    assert_parity(st["v"], st["p"], ref["v"], ref["p"], what="far states")
    c_max = 1e2 / W1.delta
    assert d["clipped"] > 0 and np.any(np.isclose(np.abs(st["c"]), c_max, rtol=1e-6))


def test_nonfinite_state_is_reported_and_isolated():
    x = hjg_inputs.points(W1, M=300)
    bad = x.copy()
    bad[17, 0] = np.nan
    st_bad, _, d, status = _run(W1, bad, 1024, 2)
    st_ok, _, _, status_ok = _run(W1, x, 1024, 2)
    from paper_2605_18566_gb300 import _lib
    assert status == _lib.HJG_ENONFINITE and status_ok == _lib.HJG_OK
    assert d["nonfinite"] >= 1
    assert not np.isfinite(st_bad["v"][17])
    keep = np.arange(300) != 17
    np.testing.assert_array_equal(st_bad["v"][keep], st_ok["v"][keep])
    np.testing.assert_array_equal(st_bad["p"][keep], st_ok["p"][keep])


def test_point_offset_range():
    """The state's global index is one 32-bit Philox counter word: a shard whose offset plus
    its states would pass 2^32 is refused, the largest one that fits is accepted."""
    from paper_2605_18566_gb300 import HJGError
    x = torch.from_numpy(hjg_inputs.points(W1, M=11)).cuda()
    s = solver_for(W1, N=64, K=1, point_offset=2**32 - 10)
    s.set_points(x[:10])
    s.picard_sweep(1)
    assert np.all(np.isfinite(s.get_state()["v"].cpu().numpy()))
    with pytest.raises(HJGError):
        s.set_points(x)
    s.close()


def test_failed_growth_leaves_the_context_usable():
    """A load the device cannot hold (2^31 states of the 45-D game: 412 GB of padded state
    rows, refused by the first allocation, before any state is read) returns HJG_ENOMEM and
    leaves the context with no states; the failed allocation is not reported again by the
    next sweep, and a later load solves exactly as a fresh context does."""
    import ctypes as C
    from paper_2605_18566_gb300 import _lib
    w = hjg_inputs.ROCKETS45
    x = torch.from_numpy(hjg_inputs.points(w, M=64)).cuda()
    s = solver_for(w, N=256, K=2)
    s.set_points(x)
    s.picard_sweep(2)
    huge = 1 << 31
    assert huge * 48 * 4 > 300e9   # more than the device holds: the first cudaMalloc fails
    st = s.lib.hjg_set_points(s.ctx, C.c_void_p(x.data_ptr()), huge, x.stride(0), 1, None)
    assert st == _lib.HJG_ENOMEM
    r = np.full(2, -1.0)
    assert s.lib.hjg_picard_sweep(s.ctx, 1, r.ctypes.data_as(C.c_void_p), None) == _lib.HJG_OK
    assert r[0] == -1.0            # no states loaded: nothing ran
    s.set_points(x)
    r1, _ = s.picard_sweep(2)
    got = {k: t.cpu().numpy() for k, t in s.get_state().items()}
    s.close()
    f = solver_for(w, N=256, K=2)
    f.set_points(x)
    r2, _ = f.picard_sweep(2)
    ref = {k: t.cpu().numpy() for k, t in f.get_state().items()}
    f.close()
    for key in ("v", "p", "c"):
        np.testing.assert_array_equal(got[key], ref[key])
    np.testing.assert_array_equal(r1, r2)
