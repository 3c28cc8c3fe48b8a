"""Pins for the oracle's heat-kernel estimator and Picard loop.

Each test compares the oracle with something fixed by mathematics rather than by the
oracle itself:
  * the closed-form Gaussian expectation for a quadratic target at any fixed c
    (value and gradient of the frozen-coefficient map Phi, Lemma 2.2 / Cor. 2.3);
  * the exact Cole-Hopf case H = |p|^2/2, where c = 1/delta and one sweep gives the
    viscous solution (Corollary B.2), and its negative-c mirror H = -|p|^2/2;
  * the zero-Hamiltonian limit (Remark 2.8: c -> 0 recovers the Gaussian mean);
  * unbiasedness of the tilted proposal for every shift (Corollary B.6);
  * the O(N^-1/2) Monte-Carlo error law (Theorem 2.4);
  * robustness to terminal-cost perturbations (Theorem thm:robustness-g), exact on fixed
    draws for one frozen-coefficient solve;
  * the effective sample size against its closed form (Section 2.4);
  * dense 2-D quadrature of the heat integral for the non-quadratic Dubins and
    two-rocket targets (Eq. heat_kernel), and a whole quadrature Picard loop on the 2-D
    double integrator against the Monte-Carlo Picard loop (a stale coefficient or a
    wrong sample variance in the loop moves the values by 20 to 10^4 standard errors).
"""
import math

import numpy as np
import pytest

import hjg_inputs
import oracle


# ----------------------------------------------------------------- closed forms
def quad_closed_form(A, x0, d, x, c, sigma2):
    """E_{y~N(x, sigma2 I)} exp(-c l(y)) for l = (y-x0)^T A (y-x0)/2 + d, returned as
    (v, Dv) with v = -(1/c) log E.  Derived by Gaussian integration:
    v = d + mu^T M A mu / 2 + log det(I + c sigma2 A) / (2c),  Dv = M A mu,
    M = (I + c sigma2 A)^-1, mu = x - x0."""
    n = len(x0)
    mu = np.asarray(x, dtype=np.float64) - x0
    B = np.eye(n) + c * sigma2 * A
    Minv = np.linalg.inv(B)
    sign, logdet = np.linalg.slogdet(B)
    assert sign > 0
    v = d + 0.5 * mu @ Minv @ A @ mu + logdet / (2.0 * c)
    g = Minv @ A @ mu
    return v, g


def replicate_sweep(P, x, c, N, R, theta=None, sweep_index=0):
    vs, ps = [], []
    for r in range(R):
        P.seed = 1000 + r
        v, p, ess = oracle.sweep(P, x, c, N, sweep_index, theta=theta)
        vs.append(v); ps.append(p)
    return np.array(vs), np.array(ps)


def check_against(vs, ps, v_ref, p_ref, k=5.0, floor_v=1e-6, floor_p=1e-6):
    """Replica mean within k standard errors (plus a tiny floor) of the reference."""
    R = vs.shape[0]
    v_se = vs.std(0, ddof=1) / math.sqrt(R) + floor_v
    p_se = ps.std(0, ddof=1) / math.sqrt(R) + floor_p
    assert np.all(np.abs(vs.mean(0) - v_ref) < k * v_se), (vs.mean(0), v_ref, v_se)
    assert np.all(np.abs(ps.mean(0) - p_ref) < k * p_se), (ps.mean(0), p_ref, p_se)


@pytest.mark.parametrize("c", [0.7, 3.0, -0.4])
def test_fixed_c_quadratic_closed_form(c):
    n = 3
    A = hjg_inputs.spd_matrix(n, 0.3, 1.2, seed=3)
    x0 = np.array([0.2, -0.1, 0.4]); d = -0.3
    delta, T = 0.2, 1.0
    P = oracle.make_problem("quadratic", n, delta, T, A=A, x0=x0, d=d)
    x = hjg_inputs.random_states(4, n, 1.0, seed=5).astype(np.float64)
    cc = np.full(len(x), c)
    vs, ps = replicate_sweep(P, x, cc, 1 << 15, 8)
    for m in range(len(x)):
        v_ref, p_ref = quad_closed_form(A, x0, d, x[m], c, delta * T)
        check_against(vs[:, m], ps[:, m], v_ref, p_ref)
    # a wrong sample variance (sigma instead of sigma^2) would move v by far more
    v_bad, _ = quad_closed_form(A, x0, d, x[0], c, math.sqrt(delta * T))
    assert abs(vs[:, 0].mean() - v_bad) > 10 * vs[:, 0].std(ddof=1) / math.sqrt(len(vs))


def test_exact_cole_hopf_case_one_sweep():
    """H = |p|^2/2 with eta = 0: c = 1/delta, one sweep is the exact viscous solution,
    and the Picard loop stays there (every sweep, every replica seed)."""
    n = 2
    A = np.array([[1.0, 0.3], [0.3, 0.6]]); x0 = np.array([0.5, -0.5]); d = 0.1
    delta, T = 0.2, 1.5
    P = oracle.make_problem("quadratic", n, delta, T, A=A, x0=x0, d=d, eta=0.0)
    x = hjg_inputs.random_states(5, n, 1.0, seed=11).astype(np.float64)
    outs = []
    for r in range(8):
        P.seed = 500 + r
        outs.append(oracle.picard(P, x, 1 << 14, 3))
        np.testing.assert_allclose(outs[-1]["c"], 1.0 / delta, rtol=1e-12)
    for m in range(len(x)):
        v_ref, p_ref = quad_closed_form(A, x0, d, x[m], 1.0 / delta, delta * T)
        for k in (1, 2, 3):
            vs = np.array([o["v_hist"][k, m] for o in outs])
            ps = np.array([o["p"][m] for o in outs])
            check_against(vs, ps, v_ref, p_ref)
    # initial iterate: v0 = g, c0 = 1/delta
    v0, p0, c0 = oracle.init(P, x)
    np.testing.assert_allclose(c0, 1.0 / delta, rtol=1e-12)


def test_negative_coefficient_case():
    """H = -|p|^2/2: c = -1/delta, estimator still the closed form (I - T A > 0)."""
    n = 2
    A = np.array([[0.5, 0.1], [0.1, 0.3]]); x0 = np.zeros(2); d = 0.0
    delta, T = 0.2, 1.0
    P = oracle.make_problem("quadratic", n, delta, T, A=A, x0=x0, d=d, eta=0.0, h_sign=-1.0)
    x = np.array([[0.5, 0.2], [-1.0, 0.7]])
    v0, p0, c0 = oracle.init(P, x)
    np.testing.assert_allclose(c0, -1.0 / delta, rtol=1e-12)
    vs, ps = replicate_sweep(P, x, c0, 1 << 15, 8)
    for m in range(len(x)):
        v_ref, p_ref = quad_closed_form(A, x0, d, x[m], -1.0 / delta, delta * T)
        check_against(vs[:, m], ps[:, m], v_ref, p_ref)


def test_zero_hamiltonian_limit():
    """H = 0: c is clipped to +c_min and v approaches the Gaussian mean E[l] (Remark 2.8)."""
    n = 3
    A = hjg_inputs.spd_matrix(n, 0.5, 1.0, seed=2); x0 = np.zeros(n); d = 0.2
    delta, T = 0.2, 1.0
    P = oracle.make_problem("zero_h", n, delta, T, A=A, x0=x0, d=d)
    x = hjg_inputs.random_states(3, n, 1.0, seed=4).astype(np.float64)
    v0, p0, c0 = oracle.init(P, x)
    np.testing.assert_allclose(c0, P.c_min)
    vs, ps = replicate_sweep(P, x, c0, 1 << 14, 8)
    sigma2 = delta * T
    for m in range(len(x)):
        v_ref, p_ref = quad_closed_form(A, x0, d, x[m], P.c_min, sigma2)
        check_against(vs[:, m], ps[:, m], v_ref, p_ref)
        # heat-equation mean E[l] = l(x) + sigma^2 tr(A)/2 within O(c) of v
        mean_l = 0.5 * x[m] @ A @ x[m] + d + 0.5 * sigma2 * np.trace(A)
        assert abs(v_ref - mean_l) < 5 * P.c_min * sigma2 * (1 + np.sum(A * A))


@pytest.mark.parametrize("scale", [0.3, 1.0])
def test_tilted_proposal_unbiased(scale):
    n = 3
    A = hjg_inputs.spd_matrix(n, 0.4, 1.0, seed=8); x0 = np.array([0.1, 0.2, -0.3]); d = 0.0
    delta, T = 0.2, 1.0
    P = oracle.make_problem("quadratic", n, delta, T, A=A, x0=x0, d=d)
    x = hjg_inputs.random_states(3, n, 1.0, seed=9).astype(np.float64)
    # shifts of a fraction of / one sampling standard deviation per axis
    theta = scale * math.sqrt(delta * T) * hjg_inputs.random_states(3, n, 1.0, seed=10)
    theta = theta.astype(np.float64)
    c = np.array([2.0, 0.5, 4.0])
    vs, ps = replicate_sweep(P, x, c, 1 << 15, 8, theta=theta)
    for m in range(len(x)):
        v_ref, p_ref = quad_closed_form(A, x0, d, x[m], c[m], delta * T)
        check_against(vs[:, m], ps[:, m], v_ref, p_ref)


def test_laplace_tilt_reduces_variance():
    """With theta = -sigma^2 c Dv (Eq. tilt_shift) the ESS rises for a strongly weighted case."""
    n = 3
    A = np.eye(n); x0 = np.zeros(n)
    delta, T = 0.2, 1.0
    P = oracle.make_problem("quadratic", n, delta, T, A=A, x0=x0)
    x = np.array([[2.0, -1.5, 1.0]])
    c = np.array([8.0])
    _, p_ref = quad_closed_form(A, x0, 0.0, x[0], c[0], delta * T)
    theta = -delta * T * c[0] * p_ref[None, :]
    _, _, ess0 = oracle.sweep(P, x, c, 4096, 0)
    _, _, ess1 = oracle.sweep(P, x, c, 4096, 0, theta=theta)
    assert ess1[0] > 3 * ess0[0]


@pytest.mark.parametrize("c", [0.7, 3.0])
def test_ess_closed_form(c):
    """Effective sample size (Section 2.4), ESS = (sum w)^2 / sum w^2: ESS / N converges to
    (E w)^2 / E w^2, and for a quadratic target both moments are Gaussian integrals,
    E exp(-c l) = exp(-c v_c) and E exp(-2c l) = exp(-2c v_2c) with v_c of the closed form
    above, so ESS / N -> exp(2c (v_2c - v_c)).  A constant target (A = 0) gives equal
    weights and ESS = N exactly.  The replica means land within ~1e-4 to 7e-4 of the
    closed form, so a wrong power or shift in either sum fails."""
    n = 3
    A = hjg_inputs.spd_matrix(n, 0.4, 1.1, seed=21); x0 = np.array([0.3, -0.2, 0.1]); d = 0.4
    delta, T = 0.2, 1.0
    sigma2 = delta * T
    P = oracle.make_problem("quadratic", n, delta, T, A=A, x0=x0, d=d)
    x = hjg_inputs.random_states(3, n, 1.0, seed=22).astype(np.float64)
    cc = np.full(len(x), c)
    N, R = 1 << 15, 6
    ratios = []
    for r in range(R):
        P.seed = 2000 + r
        _, _, ess = oracle.sweep(P, x, cc, N, 0)
        ratios.append(ess / N)
    ratios = np.array(ratios)
    for m in range(len(x)):
        v_c, _ = quad_closed_form(A, x0, d, x[m], c, sigma2)
        v_2c, _ = quad_closed_form(A, x0, d, x[m], 2.0 * c, sigma2)
        ref = math.exp(2.0 * c * (v_2c - v_c))
        assert 0.0 < ref < 1.0
        se = ratios[:, m].std(ddof=1) / math.sqrt(R) + 1e-4
        assert abs(ratios[:, m].mean() - ref) < 5 * se, (m, ratios[:, m].mean(), ref)
    P0 = oracle.make_problem("quadratic", n, delta, T, A=np.zeros((n, n)), x0=x0, d=d)
    _, _, ess0 = oracle.sweep(P0, x, cc, 4096, 0)
    np.testing.assert_allclose(ess0, 4096.0, rtol=1e-12)


def test_terminal_cost_perturbation_moves_the_value_by_at_most_its_size():
    """Theorem thm:robustness-g (a terminal cost moved by at most eps moves the value by at
    most eps), at the level of one frozen-coefficient solve on fixed draws, where it holds
    exactly: v = -(1/c) log mean exp(-c l(y_i)) is monotone in l and 1-Lipschitz in the
    sup-norm for either sign of c.  A constant shift of the target (a larger capture radius)
    lowers v by exactly the shift and leaves Dv unchanged; the flock target with every
    neighbour moved by at most eps (so l moves by at most eps) moves v by at most eps."""
    eps = 0.05
    w = hjg_inputs.DUBINS3
    x = hjg_inputs.points(w, M=48).astype(np.float64)
    P1 = oracle.make_problem(w.game, w.n, w.delta, w.T, radius=w.radius)
    P2 = oracle.make_problem(w.game, w.n, w.delta, w.T, radius=w.radius + eps)
    _, _, c0 = oracle.init(P1, x)
    v1, p1, _ = oracle.sweep(P1, x, c0, 2048, 0)
    v2, p2, _ = oracle.sweep(P2, x, c0, 2048, 0)
    np.testing.assert_allclose(v2, v1 - eps, rtol=0, atol=1e-11 * (1 + np.abs(v1).max()))
    np.testing.assert_allclose(p2, p1, rtol=1e-9, atol=1e-12)

    xf = hjg_inputs.flock_states(300, seed=4).astype(np.float64)
    _, nbr, psibar = oracle.flock_neighbours(xf)
    rng = np.random.default_rng(6)
    d = rng.normal(size=(len(xf), 7, 3))
    d *= (eps * rng.uniform(0.0, 1.0, size=(len(xf), 7, 1))) / np.linalg.norm(d, axis=2, keepdims=True)
    nbr2 = nbr + d.reshape(len(xf), 21)
    P = oracle.make_problem("flock4", 4, 0.04, 1.0, radius=0.2)
    _, _, cf = oracle.init(P, xf, nbr, psibar)
    for c in (np.abs(cf), -np.abs(cf)):
        va, _, _ = oracle.sweep(P, xf, c, 1024, 0, nbr=nbr)
        vb, _, _ = oracle.sweep(P, xf, c, 1024, 0, nbr=nbr2)
        dv = np.abs(vb - va)
        assert np.all(dv <= eps * (1 + 1e-9) + 1e-12), dv.max()
        assert dv.max() > 0.1 * eps     # the perturbation does move the values


def test_mc_error_law():
    """RMS error of the value estimator falls as N^-1/2 (Theorem 2.4)."""
    n = 2
    A = np.array([[1.0, 0.0], [0.0, 0.5]]); x0 = np.zeros(2)
    delta, T = 0.2, 1.0
    P = oracle.make_problem("quadratic", n, delta, T, A=A, x0=x0)
    x = np.array([[0.8, -0.6]])
    c = np.array([2.0])
    v_ref, _ = quad_closed_form(A, x0, 0.0, x[0], c[0], delta * T)
    Ns = [256, 1024, 4096, 16384]
    rms = []
    for N in Ns:
        vs, _ = replicate_sweep(P, x, c, N, 48)
        rms.append(math.sqrt(np.mean((vs[:, 0] - v_ref) ** 2)))
    slope = np.polyfit(np.log(Ns), np.log(rms), 1)[0]
    assert -0.65 < slope < -0.35, (slope, rms)


# ----------------------------------------------------------------- quadrature
def heat_quadrature_2d(f, center, sigma2, c, half_width=8.0, n=1201):
    """E_{u ~ N(center, sigma2 I_2)}[exp(-c f(u))] and E[u exp(-c f(u))] by a dense
    trapezoid rule over +-half_width standard deviations."""
    s = math.sqrt(sigma2)
    t = np.linspace(-half_width, half_width, n)
    U1, U2 = np.meshgrid(center[0] + s * t, center[1] + s * t, indexing="ij")
    dens = np.exp(-0.5 * (t[:, None] ** 2 + t[None, :] ** 2)) / (2 * math.pi)
    h = t[1] - t[0]
    wts = np.ones(n); wts[0] = wts[-1] = 0.5
    W = wts[:, None] * wts[None, :] * h * h
    F = np.exp(-c * f(U1, U2)) * dens * W
    E = F.sum()
    return E, np.array([(U1 * F).sum() / E, (U2 * F).sum() / E])


def test_dubins_quadrature():
    """Non-quadratic target |(y1,y2)| - r: MC oracle vs 2-D quadrature of Eq. heat_kernel."""
    w = hjg_inputs.DUBINS3
    P = oracle.make_problem("dubins3", 3, w.delta, w.T, radius=w.radius)
    x = np.array([[0.3, -0.2, 1.0], [1.5, 0.5, -2.0], [-0.6, 1.1, 0.3]])
    c = np.array([3.0, 0.8, -1.5])
    vs, ps = replicate_sweep(P, x, c, 1 << 15, 8)
    sigma2 = w.sigma2
    for m in range(len(x)):
        E, ybar = heat_quadrature_2d(lambda a, b: np.sqrt(a * a + b * b) - w.radius,
                                     x[m, :2], sigma2, c[m])
        v_ref = -math.log(E) / c[m]
        g_ref = np.array([*(x[m, :2] - ybar) / (sigma2 * c[m]), 0.0])
        check_against(vs[:, m], ps[:, m], v_ref, g_ref, floor_v=1e-5, floor_p=1e-5)


def heat_log_quadrature_2d(f, x, sigma2, c, center, half_width=8.0, n=641):
    """log E_{y ~ N(x, sigma2 I_2)}[exp(-c f(y))] and E[y exp(-c f)] / E[exp(-c f)] by a
    dense trapezoid rule over +-half_width standard deviations about `center` (where the
    integrand's mass sits when |c| is large), with the exponent shifted by its maximum."""
    s = math.sqrt(sigma2)
    t = np.linspace(-half_width, half_width, n)
    h = t[1] - t[0]
    wts = np.ones(n); wts[0] = wts[-1] = 0.5
    Y1, Y2 = np.meshgrid(center[0] + s * t, center[1] + s * t, indexing="ij")
    Z1, Z2 = (Y1 - x[0]) / s, (Y2 - x[1]) / s
    a = -0.5 * (Z1 ** 2 + Z2 ** 2) - c * f(Y1, Y2)
    mx = a.max()
    F = np.exp(a - mx) * (wts[:, None] * wts[None, :] * h * h)
    S = F.sum()
    return mx + math.log(S / (2 * math.pi)), np.array([(Y1 * F).sum() / S, (Y2 * F).sum() / S])


def test_quadrature_picard_matches_mc_picard():
    """Algorithm 1 run twice on the 2-D double integrator: once with every heat integral
    done by dense quadrature (each sweep's grid centred at the Laplace point
    x - sigma^2 c Dv of the current iterate) and the coefficient map applied to the
    quadrature gradient, once by the oracle's Monte-Carlo Picard loop with the tilted
    proposal.  After every sweep the Monte-Carlo values (replicas over seeds) agree with
    the quadrature iterate, and so do the final gradients, on every state whose coefficient
    keeps its sign along the quadrature trajectory (where H crosses 0 the coefficient map
    jumps and the two iterations may legitimately part)."""
    w = hjg_inputs.DOUBLE_INT2
    t_h, K, N, R = 0.8, 4, 1 << 16, 8
    sigma2 = w.delta * t_h
    P = oracle.make_problem(w.game, w.n, w.delta, t_h, radius=w.radius)
    Pt = oracle.make_problem(w.game, w.n, w.delta, t_h, radius=w.radius, tilt=True)
    f = lambda a, b: np.sqrt(a * a + b * b) - w.radius
    rng = np.random.default_rng(1)
    x = rng.uniform(-1.6, 1.6, size=(40, 2)).astype(np.float32).astype(np.float64)
    for m in range(3):
        assert abs(oracle.ell(P, x[m]) - f(*x[m])) < 1e-12
    v, p, c = oracle.init(P, x)
    vq_hist, cs = [v.copy()], [c.copy()]
    for k in range(K):
        v = np.zeros(len(x)); pn = np.zeros_like(p)
        for m in range(len(x)):
            logE, ybar = heat_log_quadrature_2d(f, x[m], sigma2, c[m], x[m] - sigma2 * c[m] * p[m])
            v[m] = -logE / c[m]
            pn[m] = (x[m] - ybar) / (sigma2 * c[m])
        p = pn
        c = oracle.coef_batch(P, x, p)
        vq_hist.append(v.copy()); cs.append(c.copy())
    cs = np.array(cs)
    keep = np.all(np.sign(cs) == np.sign(cs[0]), axis=0)
    assert keep.mean() >= 0.8
    runs = []
    for r in range(R):
        Pt.seed = 700 + r
        runs.append(oracle.picard(Pt, x, N, K))
    for k in range(1, K + 1):
        vs = np.array([o["v_hist"][k] for o in runs])
        se = vs.std(0, ddof=1) / math.sqrt(R) + 1e-7 * (1 + np.abs(vq_hist[k]))
        z = np.abs(vs.mean(0) - vq_hist[k]) / se
        assert np.all(z[keep] < 6.0), (k, z[keep].max())
    ps = np.array([o["p"] for o in runs])
    se = ps.std(0, ddof=1) / math.sqrt(R) + 1e-7 * (1 + np.abs(p))
    z = (np.abs(ps.mean(0) - p) / se).max(1)
    assert np.all(z[keep] < 6.0), z[keep].max()


def test_rockets6_quadrature():
    """Two-rocket target depends on the position difference, which is N(dx, 2 sigma^2 I)."""
    w = hjg_inputs.ROCKETS6
    P = oracle.make_problem("rockets6", 6, w.delta, w.T, radius=w.radius)
    x = np.array([[0.4, 0.1, -0.3, 0.5, 0.2, 1.0], [2.0, -1.0, 0.5, 0.5, -2.0, 0.1]])
    c = np.array([2.0, 0.6])
    vs, ps = replicate_sweep(P, x, c, 1 << 15, 8)
    sigma2 = w.sigma2
    for m in range(len(x)):
        dx = x[m, 0:2] - x[m, 2:4]
        E, dbar = heat_quadrature_2d(lambda a, b: np.sqrt(a * a + b * b) - w.radius,
                                     dx, 2 * sigma2, c[m])
        v_ref = -math.log(E) / c[m]
        # E[y_A w]/E[w] = x_A + (E[D w]/E[w] - dx)/2 and y_B symmetrically
        shift = (dbar - dx) / 2.0
        gA = -shift / (sigma2 * c[m])
        g_ref = np.array([gA[0], gA[1], -gA[0], -gA[1], 0.0, 0.0])
        check_against(vs[:, m], ps[:, m], v_ref, g_ref, floor_v=1e-5, floor_p=1e-5)
