"""The invariant frame of the 45-D game (hjg_frame_features, hjg_frame_targets,
hjg_warm_start_frame) against a numpy restatement.

Section 3.2's game is unchanged by a common translation of all positions, by a common
rotation of the positions together with the same turn of every heading, and (equal pursuer
speeds) by a relabelling of the pursuers.  The frame puts the evader at the origin heading
along the first axis and lists the pursuers by distance.  Checked here:
  * the features equal the numpy frame of the same states, and do not change when the
    states are translated, rotated or their pursuers relabelled;
  * for a correction h(x) that is a function of the frame coordinates only, loaded in state
    coordinates (value and a finite-difference gradient, hjg_warm_start_delta), the frame
    targets equal dh/dr_k and dh/dphi_k in the frame, and warm-starting a second solver from
    those targets (hjg_warm_start_frame) gives back the same v, Dv and c = Gamma(Dv): the
    chain rule that maps the frame back to state coordinates, including the evader's
    position and heading rows that the frame does not list, is the one a finite difference
    sees.
"""
import math

import numpy as np
import pytest

import hjg_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W = hjg_inputs.ROCKETS45
P = 14


def _split(x):
    x = np.asarray(x, np.float64)
    pos = x[:, :42].reshape(-1, P, 3)
    return pos[:, :, :2], pos[:, :, 2], x[:, 42:44], x[:, 44]


def _frame(x):
    """Numpy frame: (order, r [M, 14, 2] in the evader's frame, phi [M, 14]) in that order."""
    pp, th, pe, te = _split(x)
    d = pp - pe[:, None, :]
    ce, se = np.cos(te)[:, None], np.sin(te)[:, None]
    r = np.stack([d[..., 0] * ce + d[..., 1] * se, -d[..., 0] * se + d[..., 1] * ce], -1)
    order = np.argsort((d ** 2).sum(-1), axis=1, kind="stable")
    take = lambda a: np.take_along_axis(a, order[..., None] if a.ndim == 3 else order, 1)
    return order, take(r), take(th - te[:, None])


def _features(x):
    _, r, phi = _frame(x)
    return np.concatenate([r, np.cos(phi)[..., None], np.sin(phi)[..., None]], -1).reshape(len(x), -1)


A = np.linspace(-0.02, 0.03, P)
B = np.linspace(0.5, 1.5, P) * 1e-4
C = np.linspace(0.2, -0.1, P)


def _h(x):
    """A correction that depends on the frame coordinates only (per pursuer index, so no
    relabelling symmetry is assumed): sum_i a_i r_i,x + b_i r_i,z^2 + c_i sin(phi_i)."""
    pp, th, pe, te = _split(x)
    d = pp - pe[:, None, :]
    ce, se = np.cos(te)[:, None], np.sin(te)[:, None]
    rx = d[..., 0] * ce + d[..., 1] * se
    rz = -d[..., 0] * se + d[..., 1] * ce
    return (A * rx + B * rz ** 2 + C * np.sin(th - te[:, None])).sum(1)


def _grad_fd(x, eps=1e-5):
    x = np.asarray(x, np.float64)
    g = np.zeros_like(x)
    for j in range(x.shape[1]):
        e = np.zeros(x.shape[1]); e[j] = eps
        g[:, j] = (_h(x + e) - _h(x - e)) / (2 * eps)
    return g


def _close(got, want, rel, what):
    """|got - want| <= rel (1 + |want|) everywhere, else report the worst element."""
    err = np.abs(got - want) / (1 + np.abs(want))
    i = np.unravel_index(np.argmax(err), err.shape)
    assert err[i] <= rel, "%s: worst at %s: got %r, want %r (row got %s, want %s)" % (
        what, i, got[i], want[i], np.round(got[i[0]][:8], 4), np.round(want[i[0]][:8], 4))


def _solver(x):
    from paper_2605_18566_gb300 import Solver
    s = Solver(W.game, W.nu, W.T, 1024, 1, radius=W.radius)
    s.set_points(torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda())
    return s


def _transform(x, shift, turn, perm):
    pp, th, pe, te = _split(x)
    c, s = math.cos(turn), math.sin(turn)
    rot = lambda q: np.stack([c * q[..., 0] - s * q[..., 1], s * q[..., 0] + c * q[..., 1]], -1)
    pp, pe = rot(pp) + shift, rot(pe) + shift
    th, te = th + turn, te + turn
    pp, th = pp[:, perm], th[:, perm]
    out = np.concatenate([np.concatenate([pp, th[..., None]], -1).reshape(len(x), -1), pe, te[:, None]], 1)
    return out.astype(np.float32)


def test_features_match_numpy_and_are_invariant():
    x = hjg_inputs.rockets45_wide_points(2000, 5)
    s = _solver(x)
    f = s.frame_features().cpu().numpy()
    s.close()
    ref = _features(x.astype(np.float32))
    _close(f, ref, 1e-6, "features")
    perm = np.random.default_rng(3).permutation(P)
    xt = _transform(x, np.array([12.5, -40.25]), 0.75, perm)
    s = _solver(xt)
    ft = s.frame_features().cpu().numpy()
    s.close()
    # the transformed states are rounded to FP32, which can reorder two pursuers whose
    # squared distances lie within that rounding: compare the states without such near ties
    pp, _, pe, _ = _split(x.astype(np.float32))
    d2 = np.sort(((pp - pe[:, None, :]) ** 2).sum(-1), 1)
    clear = np.diff(d2, axis=1).min(1) > 1.0
    assert clear.mean() > 0.9
    scale = 1 + np.abs(ref[clear])
    assert np.max(np.abs(ft[clear] - ref[clear]) / scale) < 1e-3


def test_targets_and_warm_start_round_trip():
    x = hjg_inputs.rockets45_wide_points(768, 6).astype(np.float32)
    xd = x.astype(np.float64)
    h, g = _h(xd), _grad_fd(xd)
    d = torch.from_numpy(np.concatenate([h[:, None], g], 1).astype(np.float32)).cuda()
    s1 = _solver(x)
    s1.warm_start_delta(d)
    st1 = {k: v.cpu().numpy() for k, v in s1.get_state().items()}
    t = s1.frame_targets()
    s1.close()
    tn = t.cpu().numpy()

    order, r, phi = _frame(xd)
    Ao, Bo, Co = A[order], B[order], C[order]
    ref = np.zeros((len(x), 1 + 3 * P))
    ref[:, 0] = h
    ref[:, 1::3] = Ao
    ref[:, 2::3] = 2 * Bo * r[..., 1]
    ref[:, 3::3] = Co * np.cos(phi)
    _close(tn, ref, 2e-6, "targets")

    s2 = _solver(x)
    s2.warm_start_frame(t, positions_only=False)
    st2 = {k: v.cpu().numpy() for k, v in s2.get_state().items()}
    s2.close()
    _close(st2["v"][:, None], st1["v"][:, None], 1e-6, "v")
    # pursuer rows come back through one rotation; the evader's heading row sums
    # u x r over the pursuers (|r| up to ~300), so its FP32 rounding is larger
    np.testing.assert_allclose(st2["p"][:, :44], st1["p"][:, :44], rtol=0, atol=1e-5)
    np.testing.assert_allclose(st2["p"][:, 44], st1["p"][:, 44], rtol=0, atol=2e-4)
    np.testing.assert_allclose(st2["c"], st1["c"], rtol=1e-3, atol=0)


def test_frame_rejects_other_games():
    from paper_2605_18566_gb300 import Solver
    w = hjg_inputs.DUBINS3
    s = Solver(w.game, w.nu, w.T, 1024, 1, radius=w.radius)
    s.set_points(torch.zeros((4, 3), device="cuda"))
    with pytest.raises(RuntimeError):
        s.frame_features()
    s.close()


def test_positions_only_warm_start_keeps_heading_rows_of_l():
    """positions_only: the position rows of Dv are those of the full mapping, the 15 heading
    rows keep Dl's (zero), the value is the same, and c is Gamma of that Dv (recomputed here
    through hjg_warm_start_delta with the same state-coordinate correction)."""
    x = hjg_inputs.rockets45_wide_points(512, 7).astype(np.float32)
    xd = x.astype(np.float64)
    h, g = _h(xd), _grad_fd(xd)
    d = torch.from_numpy(np.concatenate([h[:, None], g], 1).astype(np.float32)).cuda()
    s1 = _solver(x)
    s1.warm_start_delta(d)
    t = s1.frame_targets()
    s1.close()
    s2 = _solver(x)
    s2.warm_start_frame(t, positions_only=True)
    st2 = {k: v.cpu().numpy() for k, v in s2.get_state().items()}
    d2 = s2.state_delta().cpu().numpy()
    s2.close()
    heading = np.arange(2, 45, 3)
    position = np.setdiff1d(np.arange(45), heading)
    assert np.all(d2[:, 1 + heading] == 0.0)
    np.testing.assert_allclose(d2[:, 1 + position], g[:, position], rtol=0, atol=1e-5)
    gp = g.copy(); gp[:, heading] = 0.0
    s3 = _solver(x)
    s3.warm_start_delta(torch.from_numpy(np.concatenate([h[:, None], gp], 1).astype(np.float32)).cuda())
    st3 = {k: v.cpu().numpy() for k, v in s3.get_state().items()}
    s3.close()
    _close(st2["v"][:, None], st3["v"][:, None], 1e-6, "v")
    np.testing.assert_allclose(st2["c"], st3["c"], rtol=1e-3, atol=0)
