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
    return oracle.make_problem(w.game, w.n, w.delta, w.T, radius=w.radius, **kw)


def solver_for(w, N=None, K=None, **kw):
    from paper_2605_18566_gb300 import Solver
    return Solver(w.game, w.nu, w.T, N or w.N, K if K is not None else w.K, radius=w.radius, **kw)
