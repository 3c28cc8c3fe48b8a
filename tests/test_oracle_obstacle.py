"""Pins for the reach-avoid obstacle of the oracle (the reading of Eq. HJI-RCBRAT-Visc: an
avoid disc o(y) = r_O - |y_{0,1} - c_O| > 0 inside, datum max{l, o} in every sweep, and
after every sweep v <- max{v, o(x)} with Dv <- Do(x) where the obstacle binds).

* One sweep at a given coefficient equals a numpy restatement of that definition on the
  oracle's own normals (datum, log-sum-exp, gradient, projection).
* An obstacle that no sample can reach changes nothing, bit for bit.
* The value never falls below the obstacle's constraint function, at any sweep.
* With the same positive coefficient the value is monotone in the datum: the obstacle can
  only raise it."""
import numpy as np
import pytest

import hjg_inputs
import oracle

W = hjg_inputs.DUBINS3


def _problem(obstacle=None, game=W.game, n=W.n):
    return oracle.make_problem(game, n, W.delta, W.T, radius=W.radius, obstacle=obstacle)


def _restated_sweep(x, c, N, sweep, obstacle, radius):
    """v, Dv of one frozen-coefficient sweep, written out from the definition."""
    cx, cy, r = obstacle
    sigma = np.sqrt(W.delta * W.T)
    out_v, out_p = [], []
    for m in range(len(x)):
        z = np.array([oracle.normals(W.n, 0, 0, i, m, sweep) for i in range(N)])
        y = x[m] + sigma * z
        ell = np.hypot(y[:, 0], y[:, 1]) - radius
        obs = r - np.hypot(y[:, 0] - cx, y[:, 1] - cy)
        lw = -c[m] * np.maximum(ell, obs)
        mx = lw.max()
        w = np.exp(lw - mx)
        v = -(mx + np.log(w.mean())) / c[m]
        p = (x[m] - (w[:, None] * y).sum(0) / w.sum()) / (W.T * W.delta * c[m])
        ox, oy = x[m, 0] - cx, x[m, 1] - cy
        o_x = r - np.hypot(ox, oy)
        if o_x > v:
            v = o_x
            rho = np.hypot(ox, oy)
            p = np.zeros(W.n)
            p[0], p[1] = -ox / rho, -oy / rho
        out_v.append(v); out_p.append(p)
    return np.array(out_v), np.array(out_p)


def test_one_sweep_matches_the_definition():
    obstacle = (0.8, 0.1, 0.6)
    x = np.array([[0.9, 0.2, 0.3], [0.8, 0.05, -1.0], [1.6, -0.4, 2.0], [-0.3, 0.7, 0.1],
                  [0.0, 0.0, 0.5], [1.3, 0.6, -2.5]])
    c = np.array([2.5, 4.0, 1.0, 5.0, 3.0, 0.7])
    N = 3000
    v, p, _ = oracle.sweep(_problem(obstacle), x, c, N, 1)
    v_ref, p_ref = _restated_sweep(x, c, N, 1, obstacle, W.radius)
    np.testing.assert_allclose(v, v_ref, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(p, p_ref, rtol=1e-9, atol=1e-11)
    o_x = obstacle[2] - np.hypot(x[:, 0] - obstacle[0], x[:, 1] - obstacle[1])
    assert np.any(v == o_x) and np.any(v > o_x)   # both branches are exercised


def test_unreachable_obstacle_changes_nothing():
    x = hjg_inputs.points(W)[::16].astype(np.float64)
    a = oracle.picard(_problem(), x, 2048, 4)
    b = oracle.picard(_problem((1e3, 1e3, 1.0)), x, 2048, 4)
    for k in ("v", "p", "c", "resid"):
        np.testing.assert_array_equal(a[k], b[k])


@pytest.mark.parametrize("game,n", [("dubins3", 3), ("rockets_rel3", 3), ("double_int2", 2)])
def test_value_never_below_the_obstacle(game, n):
    rng = np.random.default_rng(3)
    x = rng.uniform(-1.5, 1.5, size=(300, n))
    if game == "dubins3":
        x[:, 2] = rng.uniform(-np.pi, np.pi, 300)
    obstacle = (0.6, -0.3, 0.5)
    P = oracle.make_problem(game, n, W.delta, W.T, radius=0.4, obstacle=obstacle,
                            speed=[1.0, 0.5] if game == "rockets_rel3" else None)
    res = oracle.picard(P, x, 1024, 5)
    o_x = obstacle[2] - np.hypot(x[:, 0] - obstacle[0], x[:, 1] - obstacle[1])
    for k in range(6):
        assert np.all(res["v_hist"][k] >= o_x - 1e-15), k
    inside = o_x > 0
    assert inside.sum() > 10 and np.all(res["v"][inside] > 0)   # avoid states are not captured


def test_obstacle_only_raises_the_value_at_a_fixed_coefficient():
    x = hjg_inputs.points(W)[::8].astype(np.float64)
    c = np.full(len(x), 3.0)
    v0, _, _ = oracle.sweep(_problem(), x, c, 2048, 0)
    v1, _, _ = oracle.sweep(_problem((0.5, 0.5, 0.7)), x, c, 2048, 0)
    assert np.all(v1 >= v0 - 1e-12)
    assert np.mean(v1 > v0 + 1e-9) > 0.05
