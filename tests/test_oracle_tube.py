"""Pins for the oracle's tube form (Eq. HJ-RCBRT-Visc): v_t + min{0, H} = (delta/2) Lap v.

Only the coefficient map changes: Gamma is built from min{0, H}.  Checked against
  * a brute-force max_u min_d of <p, f> for the Dubins game (Appendix D.2 dynamics),
    clipped to zero from above;
  * a game whose Hamiltonian is never positive (H = -|p|^2/2), where the tube and the
    plain iteration coincide bit for bit;
  * a game whose Hamiltonian is never negative (H = +|p|^2/2), where min{0, H} = 0, the
    coefficient stays at +c_min and every sweep is the Gaussian expectation of the
    quadratic target at c = c_min (closed form), i.e. the heat equation up to O(c_min).
"""
import math

import numpy as np

import hjg_inputs
import oracle
from test_oracle_estimator import check_against, quad_closed_form, replicate_sweep

GRID = np.linspace(-1.0, 1.0, 41)


def brute_dubins_h(x, p):
    def f(u, d):
        return np.array([-1.0 + math.cos(x[2]) + u * x[1], math.sin(x[2]) - u * x[0], d - u])
    return max(min(float(p @ f(u, d)) for d in GRID) for u in GRID)


def test_tube_coefficient_map_brute_force():
    delta = 0.2
    P = oracle.make_problem("dubins3", 3, delta, 1.0, radius=0.5, tube=True)
    r = np.random.default_rng(7)
    seen_pos = seen_neg = 0
    for _ in range(60):
        x = r.normal(size=3) * 2
        p = r.normal(size=3) * r.uniform(0.05, 5)
        h = brute_dubins_h(x, p)
        c = oracle.coef(P, x, p)
        if h > 1e-9:
            seen_pos += 1
            assert c == P.c_min
        elif h < -1e-9:
            seen_neg += 1
            raw = (2.0 / delta) * h / (p @ p + P.eta)
            expect = -min(max(abs(raw), P.c_min), P.c_max)
            np.testing.assert_allclose(c, expect, rtol=1e-9)
    assert seen_pos > 5 and seen_neg > 5


def test_tube_equals_plain_when_hamiltonian_nonpositive():
    n = 3
    A = hjg_inputs.spd_matrix(n, 0.5, 1.0, seed=3)
    kw = dict(A=A, x0=np.zeros(n), d=0.1, h_sign=-1.0)
    P = oracle.make_problem("quadratic", n, 0.2, 1.0, **kw)
    Pt = oracle.make_problem("quadratic", n, 0.2, 1.0, tube=True, **kw)
    x = hjg_inputs.random_states(50, n, 1.0, seed=5).astype(np.float64)
    a = oracle.picard(P, x, 512, 3)
    b = oracle.picard(Pt, x, 512, 3)
    for key in ("v", "p", "c", "resid"):
        np.testing.assert_array_equal(a[key], b[key])
    assert np.all(a["c"] < 0)


def test_tube_with_nonnegative_hamiltonian_is_heat_equation():
    n = 3
    A = hjg_inputs.spd_matrix(n, 0.5, 1.0, seed=2)
    x0 = np.zeros(n); d = 0.2
    delta, T = 0.2, 1.0
    P = oracle.make_problem("quadratic", n, delta, T, A=A, x0=x0, d=d, h_sign=1.0, tube=True)
    x = hjg_inputs.random_states(3, n, 1.0, seed=4).astype(np.float64)
    v0, p0, c0 = oracle.init(P, x)
    np.testing.assert_array_equal(c0, P.c_min)
    out = oracle.picard(P, x, 1 << 12, 3)
    np.testing.assert_array_equal(out["c"], P.c_min)
    vs, ps = replicate_sweep(P, x, c0, 1 << 14, 8)
    for m in range(len(x)):
        v_ref, p_ref = quad_closed_form(A, x0, d, x[m], P.c_min, delta * T)
        check_against(vs[:, m], ps[:, m], v_ref, p_ref)
    # the plain form of the same game has c = 1/delta (Cole-Hopf), not c_min
    Pp = oracle.make_problem("quadratic", n, delta, T, A=A, x0=x0, d=d, h_sign=1.0, eta=0.0)
    _, _, cp = oracle.init(Pp, x)
    np.testing.assert_allclose(cp, 1.0 / delta, rtol=1e-9)
