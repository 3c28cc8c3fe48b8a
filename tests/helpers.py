"""Shared helpers for the GPU parity tests (solver/oracle set-up and the tolerance)."""
import numpy as np

import hjg_inputs
import oracle

# Per-state tolerance: |dv| <= 1e-4 (1 + |v|), ||dDv|| <= 1e-3 (1 + ||Dv||).
TOL_V = 1e-4
TOL_P = 1e-3


def rel_errors(v_gpu, p_gpu, v_ref, p_ref):
    dv = np.abs(np.asarray(v_gpu, np.float64) - v_ref) / (1.0 + np.abs(v_ref))
    dp = np.linalg.norm(np.asarray(p_gpu, np.float64) - p_ref, axis=1) / \
        (1.0 + np.linalg.norm(p_ref, axis=1))
    return dv, dp


def assert_parity(v_gpu, p_gpu, v_ref, p_ref, frac=1.0, what=""):
    dv, dp = rel_errors(v_gpu, p_gpu, v_ref, p_ref)
    ok = (dv <= TOL_V) & (dp <= TOL_P)
    assert np.all(np.isfinite(v_gpu)) and np.all(np.isfinite(p_gpu)), what
    assert ok.mean() >= frac, "%s: %d/%d states outside tolerance (max dv %.3e, max dp %.3e)" % (
        what, (~ok).sum(), ok.size, dv.max(), dp.max())
    return dv, dp


def problem_for(w, **kw):
    if w.speed:
        kw.setdefault("speed", list(w.speed))
    return oracle.make_problem(w.game, w.n, w.delta, w.T, radius=w.radius, **kw)


def solver_for(w, N=None, K=None, **kw):
    from paper_2605_18566_gb300 import Solver
    if w.speed:
        kw.setdefault("speed", list(w.speed))
    return Solver(w.game, w.nu, w.T, N or w.N, K if K is not None else w.K, radius=w.radius, **kw)


def gpu_trajectory(w, x, N, K, keep=None, **kw):
    """Run K sweeps one launch at a time and record the iterate before and after each
    sweep (identical, bit for bit, to one K-sweep launch; checked by the tests).  With
    ``keep`` (state indices) only those rows are recorded; the iterate arrays are indexed
    by position in ``keep`` then."""
    import torch
    s = solver_for(w, N=N, K=K, **kw)
    s.set_points(torch.from_numpy(x).cuda())
    rows = None if keep is None else torch.from_numpy(np.asarray(keep, np.int64)).cuda()

    def snap():
        return {k: (t if rows is None else t[rows]).cpu().numpy() for k, t in s.get_state().items()}
    states = [snap()]
    resid = []
    for _ in range(K):
        r, _ = s.picard_sweep(1)
        resid.append(r[0])
        states.append(snap())
    s.set_points(torch.from_numpy(x).cuda())
    r_all, sup_all = s.picard_sweep(K)
    one = snap()
    s.close()
    return states, np.array(resid), one, r_all


def check_trajectory(w, x, N, K, idx=None, tilt=False, min_pass=0.97, tube=False, obstacle=None,
                     precision="fp32", solver_kw=None, rows_only=False):
    """Verify a GPU Picard trajectory step by step, then compare it with the FP64 one.

    Per sweep k (on every state, or on the subset idx of global state indices):
      Phi:   the oracle, handed the GPU's frozen coefficient c^(k) (and tilt), reproduces
             the GPU's v^(k+1), Dv^(k+1) within tolerance (P1);
      Gamma: the oracle's coefficient map applied to the GPU's Dv^(k+1) reproduces the
             GPU's c^(k+1) to 1e-5 relative (where |c| is not at a clip bound).
    After K sweeps (P2) the GPU iterate is compared with the oracle's own FP64 trajectory.
    Where the Picard map is not contractive (c changing sign between sweeps, ESS near 1)
    the FP32 sweep's local error (~1e-6) is amplified from sweep to sweep; such states
    may leave the tolerance only if the oracle itself moves there by more than a tenth of
    the tolerance when its coefficient is perturbed, each sweep, by twice the GPU's
    largest local coefficient error at that state (three random perturbations).  At least
    ``min_pass`` of the states must pass P2 outright.

    ``solver_kw`` passes further Solver options (a launch variant, an instance); with
    ``rows_only`` only the rows idx of the GPU iterate are copied back (full-size states),
    and the returned states are indexed by position in idx."""
    extra = {} if obstacle is None else {"obstacle": obstacle}
    keep = np.asarray(idx) if (rows_only and idx is not None) else None
    states, resid, one, r_all = gpu_trajectory(w, x, N, K, keep=keep, tilt=tilt, tube=tube, precision=precision,
                                               **extra, **(solver_kw or {}))
    nb_all = pb_all = None
    if w.game == "flock4":   # neighbours among all loaded agents, as the GPU found them
        _, nb_all, pb_all = oracle.flock_neighbours(x)
    # one K-sweep launch == K one-sweep launches
    for key in ("v", "p", "c"):
        np.testing.assert_array_equal(one[key], states[-1][key])
    np.testing.assert_array_equal(r_all, resid)
    sel = np.arange(len(x)) if idx is None else np.asarray(idx)
    rsel = np.arange(len(sel)) if keep is not None else sel
    xs = x[sel].astype(np.float64)
    nb = nb_all[sel] if nb_all is not None else None
    pb = pb_all[sel] if pb_all is not None else None
    P = problem_for(w, tilt=tilt, tube=tube, **extra)
    P1 = problem_for(w, tube=tube, **extra)
    local_c = np.zeros(len(sel))
    for k in range(K):
        c_k = states[k]["c"][rsel].astype(np.float64)
        theta = None
        if tilt:
            theta = -w.sigma2 * c_k[:, None] * states[k]["p"][rsel].astype(np.float64)
        v, p, _ = oracle.sweep(P1, xs, c_k, N, k, theta=theta, nbr=nb, idx=sel)
        g_v, g_p = states[k + 1]["v"][rsel], states[k + 1]["p"][rsel]
        assert_parity(g_v, g_p, v, p, what="P1 %s sweep %d" % (w.game, k))
        g_c = states[k + 1]["c"][rsel].astype(np.float64)
        gp64 = g_p.astype(np.float64)
        c_ref = oracle.coef_batch(P, xs, gp64, pb)
        # the GPU applied Gamma to its FP64 Dv, which the stored FP32 Dv rounds by half an
        # ulp: bound the effect with one-sided difference quotients of the oracle's Gamma
        slack = 1e-6 * np.abs(c_ref)
        for j in range(w.n):
            h = np.maximum(np.abs(gp64[:, j]), 1e-30) * 2.0**-24
            up = gp64.copy(); up[:, j] += h
            dn = gp64.copy(); dn[:, j] -= h
            slack += 2.0 * np.maximum(np.abs(oracle.coef_batch(P, xs, up, pb) - c_ref),
                                      np.abs(oracle.coef_batch(P, xs, dn, pb) - c_ref))
        err = np.abs(g_c - c_ref)
        assert np.all(err <= slack + 2.0**-23 * np.abs(c_ref)), ("Gamma", k, (err - slack).max())
        c_from_p1 = oracle.coef_batch(P, xs, p, pb)
        local_c = np.maximum(local_c, np.abs(g_c - c_from_p1) / np.abs(c_from_p1))
    ref = oracle.picard(P, xs, N, K, idx=sel, nbr=nb, psibar=pb)
    dv, dp = rel_errors(states[-1]["v"][rsel], states[-1]["p"][rsel], ref["v"], ref["p"])
    fail = (dv > TOL_V) | (dp > TOL_P)
    ill = np.zeros(len(sel), bool)
    if fail.any():
        amp = np.maximum(2.0 * local_c, 3e-6)
        ill = oracle.ill_conditioned(P, xs, N, K, amp, ref, idx=sel, nbr=nb, psibar=pb,
                                     tol_v=TOL_V, tol_p=TOL_P)
    unexplained = fail & ~ill
    assert not unexplained.any(), "P2 %s: states %s outside tolerance but well-conditioned" % (
        w.game, sel[np.nonzero(unexplained)[0][:10]])
    assert (~fail).mean() >= min_pass, "P2 %s: pass fraction %.4f" % (w.game, (~fail).mean())
    return {"pass_fraction": float((~fail).mean()), "failing": int(fail.sum()),
            "ill_conditioned": int(ill.sum()), "resid": resid, "ref_resid": ref["resid"],
            "states": states, "ref": ref, "local_c": local_c}
