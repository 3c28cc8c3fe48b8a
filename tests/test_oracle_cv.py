"""Pins for the oracle's Stein control variate (surrogate-assisted sweep, zero-mean
polynomials of the normals with coefficients from a guess of the value and gradient).

* Unbiased for any guess: with a deliberately wrong guess the replica mean still matches
  the closed-form Gaussian expectation of a quadratic target (value and gradient), in the
  plain and in the tilted frame.
* With a good guess (the closed form itself) the replica spread of the gradient shrinks
  several-fold against the plain estimator.
* Structure: a zero gradient guess leaves the value untouched; a guess that would make the
  corrected weight sum non-positive falls back to the plain sums bit for bit.
"""
import numpy as np
import pytest

import hjg_inputs
import oracle
from test_oracle_estimator import check_against, quad_closed_form

n = 3
A = hjg_inputs.spd_matrix(n, 0.5, 1.5, seed=21)
X0 = np.zeros(n)
D = 0.2
DELTA, T = 0.2, 1.0
SIG2 = DELTA * T


def _problem(cv, tilt=False):
    return oracle.make_problem("quadratic", n, DELTA, T, A=A, x0=X0, d=D, cv=cv, tilt=tilt)


def _replicas(P, x, c, N, R, theta=None, cv_v=None, cv_p=None):
    vs, ps = [], []
    for r in range(R):
        P.seed = 9000 + r
        v, p, _ = oracle.sweep(P, x, c, N, 0, theta=theta, cv_v=cv_v, cv_p=cv_p)
        vs.append(v); ps.append(p)
    return np.array(vs), np.array(ps)


@pytest.mark.parametrize("tilt", [False, True])
def test_unbiased_for_a_wrong_guess(tilt):
    x = hjg_inputs.random_states(3, n, 0.8, seed=22).astype(np.float64)
    c = np.array([1.5, 0.8, 2.5])
    ref = [quad_closed_form(A, X0, D, x[m], c[m], SIG2) for m in range(len(x))]
    g_guess = np.array([0.7 * r[1] + 0.1 for r in ref])
    v_guess = np.array([r[0] + 0.15 for r in ref])
    theta = -SIG2 * c[:, None] * g_guess if tilt else None
    vs, ps = _replicas(_problem(True, tilt), x, c, 1 << 12, 12, theta, v_guess, g_guess)
    for m in range(len(x)):
        check_against(vs[:, m], ps[:, m], ref[m][0], ref[m][1])


@pytest.mark.parametrize("tilt", [False, True])
def test_good_guess_reduces_gradient_spread(tilt):
    x = hjg_inputs.random_states(3, n, 0.8, seed=23).astype(np.float64)
    c = np.array([1.0, 0.6, 1.4])
    ref = [quad_closed_form(A, X0, D, x[m], c[m], SIG2) for m in range(len(x))]
    g = np.array([r[1] for r in ref]); v = np.array([r[0] for r in ref])
    theta = -SIG2 * c[:, None] * g if tilt else None
    _, p_plain = _replicas(_problem(False, tilt), x, c, 2048, 40, theta)
    _, p_cv = _replicas(_problem(True, tilt), x, c, 2048, 40, theta, v, g)
    ratio = p_plain.std(0).mean(1) / p_cv.std(0).mean(1)
    assert np.all(ratio > 2.0), ratio


def test_zero_gradient_guess_keeps_the_value_and_fallback_is_exact():
    x = hjg_inputs.random_states(5, n, 0.8, seed=24).astype(np.float64)
    c = np.full(5, 1.2)
    P0, P1 = _problem(False), _problem(True)
    v0, p0, e0 = oracle.sweep(P0, x, c, 512, 0)
    # the plain value as the guess: mu equals the sample mean weight exactly
    v1, p1, e1 = oracle.sweep(P1, x, c, 512, 0, cv_v=v0, cv_p=np.zeros((5, n)))
    np.testing.assert_array_equal(v1, v0)           # b = 0: the weight sum is unchanged
    np.testing.assert_array_equal(e1, e0)
    assert np.all(np.any(p1 != p0, axis=1))         # the gradient sum is corrected
    # a large gradient guess: -mu b.(sum z) has the sign of +-(u . sum z), so of the guesses
    # +g and -g exactly one makes the weight sum negative (mu = mean weight, so that needs
    # c sigma |g| |u . sum z| > N: with |g| = 1e4 every stream but one whose |u . sum z| is
    # below 0.1, against a typical sqrt(N) = 23), and that one falls back to the plain sums
    # bit for bit
    for m in range(5):
        res = []
        for sgn in (1.0, -1.0):
            g = np.zeros((5, n)); g[m] = sgn * 1e4 * np.array([0.6, -0.64, 0.48])
            v2, p2, _ = oracle.sweep(P1, x, c, 512, 0, cv_v=v0, cv_p=g)
            res.append(bool(v2[m] == v0[m] and np.all(p2[m] == p0[m])))
        assert res.count(True) == 1, (m, res)
    # a value guess far from the sample mean weight (factor > 4) is not used at all
    v3, p3, _ = oracle.sweep(P1, x, c, 512, 0, cv_v=v0 - 2.0, cv_p=np.ones((5, n)))
    np.testing.assert_array_equal(v3, v0)
    np.testing.assert_array_equal(p3, p0)
