"""Pins for the oracle's games, coefficient map, residual and Picard bookkeeping.

* Closed-form Hamiltonians vs a brute-force max_u min_d of <p, f(x,u,d)> over a control
  grid that includes the bang-bang corners, with the dynamics written out here from the
  game definitions (Appendix D.2 Dubins relative dynamics, Section 3.2 per-agent rocket
  dynamics).
* Target gradients vs central finite differences.
* The 45-D target equals the union (pointwise min, Eq. sdf_union) of the 14 two-rocket
  pursuer/evader targets.
* The coefficient map keeps the sign of H, clips |c| and reduces to 1/delta when
  H = |p|^2/2 (Corollary B.2).
* The residual is the relative L2 change of Algorithm 1; resuming at sweep k reproduces
  the uninterrupted run bit for bit.
"""
import math

import numpy as np
import pytest

import hjg_inputs
import oracle

GRID = np.linspace(-1.0, 1.0, 41)


def dubins_f(x, u, d):
    return np.array([-1.0 + math.cos(x[2]) + u * x[1], math.sin(x[2]) - u * x[0], d - u])


def brute_maxmin(p, f, x):
    best = -np.inf
    for u in GRID:
        worst = min(float(p @ f(x, u, d)) for d in GRID)
        best = max(best, worst)
    return best


def test_dubins_hamiltonian_brute_force():
    P = oracle.make_problem("dubins3", 3, 0.2, 1.0, radius=0.5)
    r = np.random.default_rng(0)
    for _ in range(25):
        x = r.normal(size=3) * np.array([2, 2, 2])
        p = r.normal(size=3)
        assert abs(oracle.hamiltonian(P, x, p) - brute_maxmin(p, dubins_f, x)) < 1e-9


def test_rockets6_hamiltonian_brute_force():
    P = oracle.make_problem("rockets6", 6, 0.1, 2.0, radius=0.3, speed=[1.3, 0.7])

    def f(x, u, d):
        return np.array([1.3 * math.cos(x[4]), 1.3 * math.sin(x[4]),
                         0.7 * math.cos(x[5]), 0.7 * math.sin(x[5]), u, d])

    r = np.random.default_rng(1)
    for _ in range(25):
        x = r.normal(size=6) * 2
        p = r.normal(size=6)
        assert abs(oracle.hamiltonian(P, x, p) - brute_maxmin(p, f, x)) < 1e-9


def test_rockets45_hamiltonian_brute_force():
    """15 agents, controls enter <p,f> separably, so max over the evader's turn rate and
    min over each pursuer's are taken one control at a time on the grid."""
    speeds = list(np.linspace(0.8, 1.6, 15))
    P = oracle.make_problem("rockets45", 45, 0.1, 2.0, radius=0.3, speed=speeds)
    r = np.random.default_rng(2)
    for _ in range(10):
        x = r.normal(size=45) * 2
        p = r.normal(size=45)
        drift = 0.0
        for i in range(15):
            th = x[3 * i + 2]
            drift += p[3 * i] * speeds[i] * math.cos(th) + p[3 * i + 1] * speeds[i] * math.sin(th)
        ctrl = max(u * p[44] for u in GRID)
        for i in range(14):
            ctrl += min(u * p[3 * i + 2] for u in GRID)
        assert abs(oracle.hamiltonian(P, x, p) - (drift + ctrl)) < 1e-9


def test_flock_hamiltonian_brute_force():
    P = oracle.make_problem("flock4", 4, 0.04, 1.0, radius=0.2)

    def wrap(a):
        return (a + math.pi) % (2 * math.pi) - math.pi

    r = np.random.default_rng(3)
    for _ in range(20):
        x = r.normal(size=4) * 2
        p = r.normal(size=4)
        psibar = r.uniform(-math.pi, math.pi)

        def f(x_, u, d):
            return np.array([math.cos(x_[3]), math.sin(x_[3]), u, wrap(psibar - x_[3]) + d])

        assert abs(oracle.hamiltonian(P, x, p, psibar) - brute_maxmin(p, f, x)) < 1e-9


def fd_grad(fun, x, h=1e-6):
    g = np.zeros_like(x)
    for a in range(len(x)):
        e = np.zeros_like(x); e[a] = h
        g[a] = (fun(x + e) - fun(x - e)) / (2 * h)
    return g


@pytest.mark.parametrize("game,n", [("dubins3", 3), ("rockets6", 6), ("rockets45", 45)])
def test_target_gradient_finite_differences(game, n):
    P = oracle.make_problem(game, n, 0.1, 1.0, radius=0.4)
    r = np.random.default_rng(4)
    for _ in range(10):
        x = r.normal(size=n) * 2
        g = oracle.grad_ell(P, x)
        np.testing.assert_allclose(g, fd_grad(lambda y: oracle.ell(P, y), x), atol=1e-6)


def test_quadratic_target_and_gradient():
    n = 3
    A = hjg_inputs.spd_matrix(n, seed=6); x0 = np.array([0.1, -0.2, 0.3])
    P = oracle.make_problem("quadratic", n, 0.2, 1.0, A=A, x0=x0, d=0.7)
    x = np.array([0.5, 0.4, -1.0])
    np.testing.assert_allclose(oracle.grad_ell(P, x), fd_grad(lambda y: oracle.ell(P, y), x),
                               atol=1e-6)
    assert abs(oracle.ell(P, x0) - 0.7) < 1e-15


def test_dubins_target_is_signed_distance_to_disc():
    P = oracle.make_problem("dubins3", 3, 0.2, 1.0, radius=0.5)
    assert oracle.ell(P, [0.0, 0.0, 1.0]) == -0.5
    assert abs(oracle.ell(P, [0.3, 0.4, -2.0])) < 1e-15
    assert abs(oracle.ell(P, [3.0, 4.0, 0.0]) - 4.5) < 1e-15
    np.testing.assert_array_equal(oracle.grad_ell(P, [0.0, 0.0, 0.0]), np.zeros(3))


def test_rockets45_target_is_union_of_pairs():
    P45 = oracle.make_problem("rockets45", 45, 0.1, 2.0, radius=0.3)
    P6 = oracle.make_problem("rockets6", 6, 0.1, 2.0, radius=0.3)
    X = hjg_inputs.rockets45_points(50, seed=3).astype(np.float64)
    for x in X:
        ag = x.reshape(15, 3)
        pairs = [oracle.ell(P6, [ag[i, 0], ag[i, 1], ag[14, 0], ag[14, 1], 0, 0])
                 for i in range(14)]
        assert oracle.ell(P45, x) == min(pairs)


def test_coefficient_map_sign_clip_and_exact_case():
    delta = 0.2
    P = oracle.make_problem("dubins3", 3, delta, 1.0)
    r = np.random.default_rng(5)
    for _ in range(50):
        x = r.normal(size=3); p = r.normal(size=3) * r.uniform(0.01, 10)
        h = oracle.hamiltonian(P, x, p)
        c = oracle.coef(P, x, p)
        assert P.c_min <= abs(c) <= P.c_max
        assert (c > 0) == (h > 0) or h == 0
        if P.c_min < abs(c) < P.c_max:
            np.testing.assert_allclose(c * delta * (p @ p + P.eta) / 2, h, rtol=1e-12)
    # p = 0 => H = 0 => c = +c_min
    assert oracle.coef(P, np.ones(3), np.zeros(3)) == P.c_min
    Q = oracle.make_problem("quadratic", 2, delta, 1.0, eta=0.0, A=np.eye(2))
    assert abs(oracle.coef(Q, [0, 0], [0.3, -2.0]) - 1 / delta) < 1e-12
    # regularised map is the perturbed Hamiltonian of Lemma 2.7: |H_eta - H| <= C_H sqrt(eta)/2
    R = oracle.make_problem("dubins3", 3, delta, 1.0, eta=1e-2, c_max=1e12, c_min=1e-12)
    x = np.array([0.3, -0.4, 0.9])
    CH = max(abs(oracle.hamiltonian(R, x, q / np.linalg.norm(q)))
             for q in r.normal(size=(2000, 3)))
    for s in np.logspace(-3, 1, 30):
        p = s * np.array([0.6, -0.3, 0.2])
        h_eta = oracle.coef(R, x, p) * delta * (p @ p) / 2
        assert abs(h_eta - oracle.hamiltonian(R, x, p)) <= CH * math.sqrt(R.eta) / 2 * 1.01 + 1e-12


def test_residual_matches_norms():
    r = np.random.default_rng(6)
    a, b = r.normal(size=1000), r.normal(size=1000)
    rel, sup = oracle.residual(a, b)
    assert abs(rel - np.linalg.norm(b - a) / np.linalg.norm(a)) < 1e-12
    assert sup == np.max(np.abs(b - a))


def test_picard_resume_is_bit_exact_and_residual_settles():
    w = hjg_inputs.DUBINS3
    P = oracle.make_problem("dubins3", 3, w.delta, w.T, radius=w.radius)
    x = hjg_inputs.points(w)[::64].astype(np.float64)
    full = oracle.picard(P, x, 1024, 6)
    half = oracle.picard(P, x, 1024, 3)
    rest = oracle.picard(P, x, 1024, 3, k0=3, state=(half["v"], half["p"], half["c"]))
    np.testing.assert_array_equal(full["v"], rest["v"])
    np.testing.assert_array_equal(full["p"], rest["p"])
    np.testing.assert_array_equal(full["resid"][3:], rest["resid"])
    # the residual of the first sweep (leaving the target data) dominates later ones
    assert full["resid"][0] > full["resid"][-1]
    assert np.all(np.isfinite(full["v"])) and np.all(full["ess"] >= 1.0)


def test_flock_neighbours_brute_force_and_target():
    """k-d-tree neighbours equal a brute-force search; the flock target is the distance to
    the nearest neighbour minus the radius; psibar is the circular mean."""
    x = hjg_inputs.flock_states(600, seed=2).astype(np.float64)
    idx, nbr, psibar = oracle.flock_neighbours(x)
    pos = x[:, :3]
    d2 = ((pos[:, None, :] - pos[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    brute = np.argsort(d2, axis=1, kind="stable")[:, :7]
    np.testing.assert_array_equal(np.sort(idx, 1), np.sort(brute, 1))
    P = oracle.make_problem("flock4", 4, 0.04, 1.0, radius=0.2)
    for i in (0, 17, 333):
        expect = np.sqrt(d2[i][brute[i]].min()) - 0.2
        assert abs(oracle.ell(P, x[i], nbr[i]) - expect) < 1e-12
        ang = x[idx[i], 3]
        assert abs(np.angle(np.exp(1j * (psibar[i] - np.angle(np.exp(1j * ang).sum()))))) < 1e-12
    # identical headings average to themselves; opposite pairs around a direction to it
    y = x[:40].copy(); y[:, 3] = 0.7
    _, _, pb = oracle.flock_neighbours(y)
    np.testing.assert_allclose(pb, 0.7, atol=1e-12)


def test_flock_workload_shape():
    x = hjg_inputs.flock_states(20000, seed=0)
    idx, nbr, _ = oracle.flock_neighbours(x[:, :4])
    dnn = np.linalg.norm(x[:, :3] - x[idx[:, 0], :3], axis=1)
    assert 0.1 < np.median(dnn) < 0.6        # 20k of the 100k birds: sparser than full size
    assert np.all(np.abs(x[:, 3]) <= np.pi)


def test_relative_rockets_hamiltonian_brute_force():
    """Eq. ham_def with the vector field as printed there: H = -max_{u_e} min_{u_p} <p, f>."""
    a, g = 64.0, 32.0
    P = oracle.make_problem("rockets_rel3", 3, 0.08, 1.0, radius=1.5, speed=[a, g])

    def f(x, ue, up):
        return np.array([a * math.cos(x[2]) + ue * x[0], a * math.sin(x[2]) + a + up * x[0] - g, up - ue])

    r = np.random.default_rng(7)
    for _ in range(25):
        x = r.normal(size=3) * np.array([5, 5, 1])
        p = r.normal(size=3)
        brute = -max(min(float(p @ f(x, ue, up)) for up in GRID) for ue in GRID)
        assert abs(oracle.hamiltonian(P, x, p) - brute) < 1e-9 * (1 + abs(brute))


def test_double_integrator_hamiltonian_brute_force():
    """Eq. dint_ham with the minimising control: H = min_u (p1 x2 + p2 u)."""
    P = oracle.make_problem("double_int2", 2, 0.08, 0.8, radius=0.25)
    r = np.random.default_rng(8)
    for _ in range(25):
        x = r.normal(size=2) * 2
        p = r.normal(size=2)
        brute = min(p[0] * x[1] + p[1] * u for u in GRID)
        assert abs(oracle.hamiltonian(P, x, p) - brute) < 1e-12


@pytest.mark.parametrize("game,n", [("rockets_rel3", 3), ("double_int2", 2)])
def test_extra_game_targets(game, n):
    P = oracle.make_problem(game, n, 0.08, 1.0, radius=1.5)
    r = np.random.default_rng(9)
    for _ in range(10):
        x = r.normal(size=n) * 3
        assert abs(oracle.ell(P, x) - (math.hypot(x[0], x[1]) - 1.5)) < 1e-12
        np.testing.assert_allclose(oracle.grad_ell(P, x), fd_grad(lambda y: oracle.ell(P, y), x), atol=1e-6)
