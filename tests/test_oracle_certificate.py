"""Pins for the oracle's conservative certificate (Cor. 2.9) and the per-state Monte-Carlo
standard error it uses.

* The delta-method standard error sqrt(1/ESS - 1/N)/|c| matches the spread of v over
  independent replicas of one sweep (quadratic target, fixed c).
* In the exact Cole-Hopf case (H = |p|^2/2, c = 1/delta, no quasi-linearisation defect)
  one sweep is the viscous solution up to Monte-Carlo error, whose closed form is known:
  the certificate with e0 = 0 never labels a state SAFE whose exact value is <= 0 or UNSAFE
  whose exact value is >= 0, and it does certify the states far from the boundary.
* The band and labels follow their definitions on hand-made inputs.
"""
import math

import numpy as np

import hjg_inputs
import oracle
from test_oracle_estimator import quad_closed_form


def test_band_and_labels_by_hand():
    v = np.array([1.0, -1.0, 0.1, -0.1, 0.0])
    se = np.full(5, 0.1)
    lab, band = oracle.certify(v, se, sup_last=0.02, e0=0.05, q=0.5, delta_p=0.05)
    z = math.sqrt(2 * math.log(40.0))
    np.testing.assert_allclose(band, 0.05 + 0.02 + z * 0.1)
    np.testing.assert_array_equal(lab, [1, -1, 0, 0, 0])
    lab0, _ = oracle.certify(v, np.zeros(5), 0.0, 0.0, 0.0, 0.05)
    np.testing.assert_array_equal(lab0, [1, -1, 1, -1, 0])   # zero band: the sign, 0 undetermined
    # a collapsed ESS leaves the state undetermined whatever its value
    lab1, _ = oracle.certify(v, se, 0.0, 0.0, 0.0, 0.05, ess=np.array([5, 500, 500, 500, 500.0]),
                             ess_min=10.0)
    np.testing.assert_array_equal(lab1, [0, -1, 0, 0, 0])


def test_standard_error_matches_replica_spread():
    n = 3
    A = hjg_inputs.spd_matrix(n, 0.5, 1.5, seed=8)
    x0 = np.zeros(n)
    P = oracle.make_problem("quadratic", n, 0.2, 1.0, A=A, x0=x0, d=0.0)
    x = hjg_inputs.random_states(4, n, 1.2, seed=9).astype(np.float64)
    c = np.array([2.0, 0.7, -0.8, 0.5])
    N, R = 2048, 160
    vs, ses, esss = [], [], []
    for r in range(R):
        P.seed = 5000 + r
        v, _, ess = oracle.sweep(P, x, c, N, 0)
        vs.append(v)
        ses.append(oracle.mc_std_error(ess, c, N))
        esss.append(ess)
    vs, ses = np.array(vs), np.array(ses)
    # weights not collapsed, so the delta method applies: the typical replica keeps a large
    # ESS (with c < 0 the weights are heavy-tailed and a single replica may not)
    assert np.all(np.median(esss, 0) > 0.15 * N)
    ratio = vs.std(0, ddof=1) / ses.mean(0)
    assert np.all(np.abs(ratio - 1.0) < 0.2), ratio


def test_certificate_never_misclassifies_in_the_exact_case():
    n = 3
    delta, T = 0.2, 1.0
    A = hjg_inputs.spd_matrix(n, 0.5, 1.5, seed=10)
    x0 = np.zeros(n); d = -0.6                     # zero level set: an ellipsoid
    P = oracle.make_problem("quadratic", n, delta, T, A=A, x0=x0, d=d, eta=0.0)
    x = hjg_inputs.random_states(600, n, 1.0, seed=11).astype(np.float64)
    v0, p0, c0 = oracle.init(P, x)
    np.testing.assert_allclose(c0, 1.0 / delta, rtol=1e-12)
    N = 1024
    v, _, ess = oracle.sweep(P, x, c0, N, 0)
    se = oracle.mc_std_error(ess, c0, N)
    lab, band = oracle.certify(v, se, 0.0, 0.0, 0.0, 0.01)
    v_exact = np.array([quad_closed_form(A, x0, d, xm, 1.0 / delta, delta * T)[0] for xm in x])
    assert not np.any((lab == 1) & (v_exact <= 0.0))
    assert not np.any((lab == -1) & (v_exact >= 0.0))
    # the undetermined band is narrow: states far from the boundary are certified
    far = np.abs(v_exact) > 3 * band
    assert far.sum() > 300 and np.all(lab[far] == np.sign(v_exact[far]))
    assert (lab == 1).sum() > 50 and (lab == -1).sum() > 50
