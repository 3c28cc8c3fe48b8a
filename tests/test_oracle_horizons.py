"""Pins for the oracle's several-horizon solve: each horizon t_h is the heat kernel of width
sqrt(delta t_h) (Lemma 2.2).

* Exact Cole-Hopf case (H = |p|^2/2, c = 1/delta): one sweep at every horizon matches the
  closed-form viscous solution at sigma^2 = delta t_h within Monte-Carlo error.
* One horizon reproduces the single-horizon run bit for bit; horizon h draws the samples
  of global index h M + m (a single-horizon run with those indices agrees bit for bit).
* The residual is the relative L2 change over all items together.
"""
import numpy as np

import hjg_inputs
import oracle
from test_oracle_estimator import check_against, quad_closed_form


def _problem(delta=0.2, T=1.0):
    n = 3
    A = hjg_inputs.spd_matrix(n, 0.5, 1.5, seed=12)
    return oracle.make_problem("quadratic", n, delta, T, A=A, x0=np.zeros(n), d=0.1, eta=0.0), A


def test_each_horizon_is_the_closed_form_at_its_width():
    P, A = _problem()
    x = hjg_inputs.random_states(3, 3, 1.0, seed=13).astype(np.float64)
    times = [0.1, 0.5, 2.0]
    R = 24   # replicas: the mean's standard error estimated from R - 1 degrees of freedom
    vs, ps = [], []
    for r in range(R):
        P.seed = 700 + r
        out = oracle.picard_horizons(P, x, 1 << 13, 1, times)
        vs.append(out["v"]); ps.append(out["p"])
    vs, ps = np.array(vs), np.array(ps)
    M = len(x)
    for h, t in enumerate(times):
        for m in range(M):
            v_ref, p_ref = quad_closed_form(A, np.zeros(3), 0.1, x[m], 1.0 / P.delta, P.delta * t)
            check_against(vs[:, h * M + m], ps[:, h * M + m], v_ref, p_ref)
    # the horizons are distinguishable: their closed forms differ by far more than the error
    v_a = quad_closed_form(A, np.zeros(3), 0.1, x[0], 1.0 / P.delta, P.delta * times[0])[0]
    v_b = quad_closed_form(A, np.zeros(3), 0.1, x[0], 1.0 / P.delta, P.delta * times[-1])[0]
    assert abs(v_a - v_b) > 50 * vs[:, 0].std()


def test_horizon_indices_and_single_horizon():
    P, _ = _problem()
    x = hjg_inputs.random_states(20, 3, 1.0, seed=14).astype(np.float64)
    one = oracle.picard_horizons(P, x, 256, 2, [P.T])
    ref = oracle.picard(P, x, 256, 2)
    for key in ("v", "p", "c"):
        np.testing.assert_array_equal(one[key], ref[key])
    for key in ("resid", "sup"):   # same norms, summed in another order
        np.testing.assert_allclose(one[key], ref[key], rtol=1e-12)
    multi = oracle.picard_horizons(P, x, 256, 2, [0.3, 0.7])
    T0 = P.T
    P.T = 0.7
    h1 = oracle.picard(P, x, 256, 2, idx=20 + np.arange(20))
    P.T = T0
    np.testing.assert_array_equal(multi["v"][20:], h1["v"])
    np.testing.assert_array_equal(multi["p"][20:], h1["p"])
    vh = multi["v_hist"]
    np.testing.assert_allclose(multi["resid"][1], np.linalg.norm(vh[2] - vh[1]) / np.linalg.norm(vh[1]),
                               rtol=1e-12)
