"""FP64 CPU oracle for the HJ-Gauss frozen-coefficient Picard sweep.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package; the library under
``paper_2605_18566_gb300/`` never does, and shares no code with it.

The arithmetic lives in ``hjg_oracle.c`` (plain C, double precision, OpenMP over
evaluation states) and in ``mlp.py`` (surrogate network, numpy FP64).  This module
compiles the C file with gcc on first use and exposes thin ctypes wrappers.

Paper sections restated here: Algorithm 1 (Picard loop), Eq. coeff_frozen and
Lemma 2.7 (coefficient map), Remark 2.8 (sign and clip), Corollaries B.4-B.6 (value,
gradient and tilted estimators), Section 2.4 (ESS), Appendix D.2 and Section 3.2 (games).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hjg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

GAMES = {"dubins3": 1, "rockets6": 2, "rockets45": 3, "flock4": 4, "rockets_rel3": 5,
         "double_int2": 6, "quadratic": 100, "zero_h": 101}


class Problem(C.Structure):
    """Mirror of ``orc_problem`` in hjg_oracle.c."""
    _fields_ = [
        ("game", C.c_int32), ("n", C.c_int32),
        ("delta", C.c_double), ("T", C.c_double), ("eta", C.c_double),
        ("c_min", C.c_double), ("c_max", C.c_double), ("radius", C.c_double),
        ("speed", C.c_double * 16), ("h_sign", C.c_double),
        ("A", C.c_double * 64), ("x0", C.c_double * 8), ("d", C.c_double),
        ("seed", C.c_uint64), ("instance", C.c_uint32), ("tilt", C.c_int32),
        ("flock_k", C.c_int32), ("tube", C.c_int32), ("cv", C.c_int32), ("obstacle", C.c_int32),
        ("obs_c", C.c_double * 2), ("obs_r", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile hjg_oracle.c into liboracle.so (gcc, -O2, OpenMP)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        P = C.POINTER
        d, i64, u32, i32 = C.c_double, C.c_int64, C.c_uint32, C.c_int
        pd = P(C.c_double)
        L.orc_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
        L.orc_philox_batch.argtypes = [i64, P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
        L.orc_u01.argtypes = [u32]; L.orc_u01.restype = d
        L.orc_slot_stride.argtypes = [i32]; L.orc_slot_stride.restype = i32
        L.orc_normals.argtypes = [i32, C.c_uint64, u32, u32, u32, u32, pd]
        L.orc_block_words_normals.argtypes = [P(C.c_uint32), pd]
        L.orc_ell.argtypes = [P(Problem), pd, pd]; L.orc_ell.restype = d
        L.orc_grad_ell.argtypes = [P(Problem), pd, pd, pd]
        L.orc_hamiltonian.argtypes = [P(Problem), pd, pd, d]; L.orc_hamiltonian.restype = d
        L.orc_coef.argtypes = [P(Problem), pd, pd, d]; L.orc_coef.restype = d
        L.orc_coef_batch.argtypes = [P(Problem), i64, pd, pd, pd, pd]
        pi64 = P(C.c_int64)
        L.orc_sweep.argtypes = [P(Problem), i64, pd, pd, pd, pd, pi64, i64, u32, pd, pd, pd, pd, pd]
        L.orc_sweep.restype = i32
        L.orc_init.argtypes = [P(Problem), i64, pd, pd, pd, pd, pd, pd]
        L.orc_residual.argtypes = [i64, pd, pd, pd, pd]
        L.orc_picard.argtypes = [P(Problem), i64, pd, pd, pd, pi64, i64, i32, u32,
                                 pd, pd, pd, pd, pd, pd]
        L.orc_picard.restype = i32
        L.orc_num_threads.restype = i32
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _idx(a):
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(C.POINTER(C.c_int64))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


OBSTACLE_GAMES = ("dubins3", "rockets_rel3", "double_int2")


def make_problem(game: str, n: int, delta: float, T: float, *, eta=1e-6, c_min=None,
                 c_max=None, radius=0.5, speed=None, h_sign=1.0, A=None, x0=None,
                 d=0.0, seed=0, instance=0, tilt=False, flock_k=7, tube=False, cv=False,
                 obstacle=None) -> Problem:
    """Build an oracle problem.  Defaults follow the readings used throughout:
    eta = 1e-6, c_min = 1e-2/delta, c_max = 1e2/delta.  tube=True selects the tube form
    (Eq. HJ-RCBRT-Visc): the coefficient map uses min{0, H}.  obstacle = (cx, cy, r) adds the
    reach-avoid obstacle (a disc in the plane of state dims 0, 1; games dubins3, rockets_rel3,
    double_int2)."""
    P = Problem()
    P.game = GAMES[game]
    P.n = n
    P.delta = delta
    P.T = T
    P.eta = eta
    P.c_min = (1e-2 / delta) if c_min is None else c_min
    P.c_max = (1e2 / delta) if c_max is None else c_max
    P.radius = radius
    sp = [1.0] * 16 if speed is None else list(speed) + [1.0] * (16 - len(speed))
    for k in range(16):
        P.speed[k] = sp[k]
    P.h_sign = h_sign
    if A is not None:
        A = np.asarray(A, dtype=np.float64).reshape(n, n)
        for k, val in enumerate(A.ravel()):
            P.A[k] = val
    if x0 is not None:
        for k, val in enumerate(np.asarray(x0, dtype=np.float64).ravel()):
            P.x0[k] = val
    P.d = d
    P.seed = seed
    P.instance = instance
    P.tilt = 1 if tilt else 0
    P.flock_k = flock_k
    P.tube = 1 if tube else 0
    P.cv = 1 if cv else 0
    if obstacle is not None:
        if game not in OBSTACLE_GAMES:
            raise ValueError("the reach-avoid obstacle is defined for %s only" % (OBSTACLE_GAMES,))
        cx, cy, r = (float(v) for v in obstacle)
        P.obstacle = 1
        P.obs_c[0], P.obs_c[1], P.obs_r = cx, cy, r
    return P


# ---------------------------------------------------------------- primitives
def philox4x32_10(ctr, key):
    """Philox4x32-10 blocks: ctr uint32 [K,4], key uint32 [K,2] -> uint32 [K,4]."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    out = np.zeros_like(ctr)
    P = C.POINTER(C.c_uint32)
    lib().orc_philox_batch(ctr.shape[0], ctr.ctypes.data_as(P), key.ctypes.data_as(P),
                           out.ctypes.data_as(P))
    return out


def u01(x: int) -> float:
    return lib().orc_u01(int(x))


def slot_stride(n: int) -> int:
    return int(lib().orc_slot_stride(n))


def normals(n, seed, instance, sample, point, sweep):
    z = np.zeros(n, dtype=np.float64)
    lib().orc_normals(n, seed, instance, sample, point, sweep, _dp(z))
    return z


def block_words_normals(words):
    """The eight normals of one Philox output block (four uint32 words)."""
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint32).reshape(4))
    z = np.zeros(8, dtype=np.float64)
    lib().orc_block_words_normals(w.ctypes.data_as(C.POINTER(C.c_uint32)), _dp(z))
    return z


def ell(P, y, nbr=None):
    y = _f64(y)
    nb = _f64(nbr) if nbr is not None else None
    return lib().orc_ell(C.byref(P), _dp(y), _dp(nb))


def grad_ell(P, x, nbr=None):
    x = _f64(x)
    g = np.zeros(P.n)
    nb = _f64(nbr) if nbr is not None else None
    lib().orc_grad_ell(C.byref(P), _dp(x), _dp(nb), _dp(g))
    return g


def hamiltonian(P, x, p, psibar=0.0):
    return lib().orc_hamiltonian(C.byref(P), _dp(_f64(x)), _dp(_f64(p)), float(psibar))


def coef(P, x, p, psibar=0.0):
    return lib().orc_coef(C.byref(P), _dp(_f64(x)), _dp(_f64(p)), float(psibar))


def coef_batch(P, x, p, psibar=None):
    """Gamma at M states: x, p [M, n] -> c [M]."""
    x = _f64(x).reshape(-1, P.n)
    p = _f64(p).reshape(-1, P.n)
    c = np.zeros(x.shape[0])
    pb = _f64(psibar) if psibar is not None else None
    lib().orc_coef_batch(C.byref(P), x.shape[0], _dp(x), _dp(p), _dp(pb), _dp(c))
    return c


# ---------------------------------------------------------------- method
def init(P, x, nbr=None, psibar=None):
    """Algorithm 1 initial iterate: (v0, p0, c0) at states x [M,n]."""
    x = _f64(x).reshape(-1, P.n)
    M = x.shape[0]
    v0 = np.zeros(M); p0 = np.zeros((M, P.n)); c0 = np.zeros(M)
    nb = _f64(nbr) if nbr is not None else None
    pb = _f64(psibar) if psibar is not None else None
    lib().orc_init(C.byref(P), M, _dp(x), _dp(nb), _dp(pb), _dp(v0), _dp(p0), _dp(c0))
    return v0, p0, c0


def sweep(P, x, c, N, sweep_index, theta=None, nbr=None, idx=None, cv_v=None, cv_p=None):
    """One frozen-coefficient heat-kernel solve Phi(c) at states x: (v, p, ess).
    idx: global state indices of the rows (default 0..M-1).  With P.cv, (cv_v, cv_p) is the
    control variate's guess of the value and gradient (the iterate entering the sweep)."""
    x = _f64(x).reshape(-1, P.n)
    M = x.shape[0]
    c = _f64(c).reshape(M)
    th = _f64(theta).reshape(M, P.n) if theta is not None else None
    nb = _f64(nbr) if nbr is not None else None
    cvv = _f64(cv_v).reshape(M) if cv_v is not None else None
    cvp = _f64(cv_p).reshape(M, P.n) if cv_p is not None else None
    v = np.zeros(M); p = np.zeros((M, P.n)); ess = np.zeros(M)
    ia, ip = _idx(idx)
    rc = lib().orc_sweep(C.byref(P), M, _dp(x), _dp(c), _dp(th), _dp(nb), ip, int(N),
                         int(sweep_index), _dp(cvv), _dp(cvp), _dp(v), _dp(p), _dp(ess))
    if rc:
        raise RuntimeError("orc_sweep failed (%d)" % rc)
    return v, p, ess


def picard(P, x, N, K, k0=0, state=None, nbr=None, psibar=None, idx=None):
    """Algorithm 1 for K sweeps.  Returns dict with v_hist [K+1,M], p, c, resid, sup, ess.
    ``state`` = (v, p, c) to resume from; default is the initial iterate."""
    x = _f64(x).reshape(-1, P.n)
    M = x.shape[0]
    if state is None:
        v0, p, c = init(P, x, nbr, psibar)
    else:
        v0, p, c = (_f64(s).copy() for s in state)
        p = p.reshape(M, P.n)
    v_hist = np.zeros((K + 1, M)); v_hist[0] = v0
    resid = np.zeros(K); sup = np.zeros(K); ess = np.zeros(M)
    p = np.ascontiguousarray(p); c = np.ascontiguousarray(c)
    nb = _f64(nbr) if nbr is not None else None
    pb = _f64(psibar) if psibar is not None else None
    ia, ip = _idx(idx)
    rc = lib().orc_picard(C.byref(P), M, _dp(x), _dp(nb), _dp(pb), ip, int(N), int(K), int(k0),
                          _dp(v_hist), _dp(p), _dp(c), _dp(resid), _dp(sup), _dp(ess))
    if rc:
        raise RuntimeError("orc_picard failed (%d)" % rc)
    return {"v_hist": v_hist, "v": v_hist[-1].copy(), "p": p, "c": c,
            "resid": resid, "sup": sup, "ess": ess}


def ill_conditioned(P, x, N, K, amp, ref, idx=None, nbr=None, psibar=None, tol_v=1e-4, tol_p=1e-3,
                    reps=3):
    """Which states of a K-sweep trajectory are too sensitive to be compared to FP32
    rounding: the oracle's own run is repeated with its coefficient perturbed in every
    sweep by relative Gaussian noise of size ``amp`` (per state, or one scalar), ``reps``
    times; a state is ill-conditioned where any repeat ends more than a tenth of the
    tolerance (|dv| / (1 + |v|) > tol_v / 10 or ||dDv|| / (1 + ||Dv||) > tol_p / 10) away
    from the unperturbed run ``ref`` (a dict with v and p, as picard returns).  Where the
    Picard map of Algorithm 1 is not contractive (c changing sign between sweeps, ESS near
    1: outside Assumption 2.6) such a perturbation grows from sweep to sweep, and so does
    an FP32 sweep's local rounding error."""
    x = _f64(x).reshape(-1, P.n)
    M = x.shape[0]
    amp = np.broadcast_to(np.asarray(amp, dtype=np.float64), (M,))
    v0, p0, c0 = init(P, x, nbr, psibar)
    v_ref = np.asarray(ref["v"], np.float64); p_ref = np.asarray(ref["p"], np.float64)
    ill = np.zeros(M, bool)
    for rep in range(reps):
        rng = np.random.default_rng(100 + rep)
        st = (v0, p0, c0)
        for k in range(K):
            c_pert = st[2] * (1.0 + amp * rng.standard_normal(M))
            out = picard(P, x, N, 1, k0=k, state=(st[0], st[1], c_pert), idx=idx, nbr=nbr, psibar=psibar)
            st = (out["v"], out["p"], out["c"])
        sv = np.abs(st[0] - v_ref) / (1.0 + np.abs(v_ref))
        sp = np.linalg.norm(st[1] - p_ref, axis=1) / (1.0 + np.linalg.norm(p_ref, axis=1))
        ill |= (sv > 0.1 * tol_v) | (sp > 0.1 * tol_p)
    return ill


def picard_horizons(P, x, N, K, times, nbr=None, psibar=None):
    """The value at several horizons t_h: for each h an independent run of Algorithm 1 at
    T = t_h (kernel width sqrt(delta t_h), Lemma 2.2) whose state m carries the global
    index h M + m; the residual of each sweep is the relative L2 change over all items.
    Returns v [H*M], p [H*M, n], c, resid [K], sup [K], ess (horizon-major)."""
    x = _f64(x).reshape(-1, P.n)
    M = x.shape[0]
    T0 = P.T
    outs = []
    try:
        for h, t in enumerate(times):
            P.T = float(t)
            outs.append(picard(P, x, N, K, nbr=nbr, psibar=psibar, idx=h * M + np.arange(M)))
    finally:
        P.T = T0
    vh = np.concatenate([o["v_hist"] for o in outs], axis=1)
    dv = np.diff(vh, axis=0)
    resid = np.sqrt((dv ** 2).sum(1)) / np.sqrt((vh[:-1] ** 2).sum(1))
    sup = np.abs(dv).max(1) if K > 0 else np.zeros(0)
    return {"v": vh[-1].copy(), "v_hist": vh, "p": np.concatenate([o["p"] for o in outs]),
            "c": np.concatenate([o["c"] for o in outs]), "ess": np.concatenate([o["ess"] for o in outs]),
            "resid": resid, "sup": sup}


def residual(v_old, v_new):
    v_old = _f64(v_old); v_new = _f64(v_new)
    rel = C.c_double(); sup = C.c_double()
    lib().orc_residual(v_old.size, _dp(v_old), _dp(v_new), C.byref(rel), C.byref(sup))
    return rel.value, sup.value


def mc_std_error(ess, c, N):
    """Delta-method Monte-Carlo standard error of v = -(1/c) log((1/N) sum w_i) from one
    sweep: sd(w) / (sqrt(N) mean(w) |c|) = sqrt(1/ESS - 1/N) / |c| with ESS = (sum w)^2 /
    sum w^2 (Section 2.4) and c the coefficient that sweep used (Theorem 2.4 gives the
    O(N^-1/2) rate this estimates per state)."""
    ess = np.asarray(ess, dtype=np.float64)
    return np.sqrt(np.maximum(0.0, 1.0 / ess - 1.0 / N)) / np.abs(np.asarray(c, dtype=np.float64))


def certify(v, se, sup_last, e0, q, delta_p, ess=None, ess_min=0.0):
    """Conservative certificate of Cor. 2.9: band E = e0 + q/(1-q) sup_last + z se with
    z = sqrt(2 log(2/delta_p)) (the Monte-Carlo term at failure probability delta_p; the
    iteration term is the a-posteriori bound of Theorem 2.8 from the last sweep's
    sup-norm change; e0 bounds the remaining defect and viscosity terms).  Returns labels
    (+1 SAFE where v > E, -1 UNSAFE where v < -E, 0 UNDETERMINED) and E.  States whose
    ESS is below ess_min are UNDETERMINED: with collapsed weights (Section 2.4) the
    standard error itself is not trustworthy."""
    v = np.asarray(v, dtype=np.float64)
    z = math.sqrt(2.0 * math.log(2.0 / delta_p))
    band = e0 + (q / (1.0 - q)) * sup_last + z * np.asarray(se, dtype=np.float64)
    labels = np.where(v > band, 1, np.where(v < -band, -1, 0)).astype(np.int8)
    if ess is not None:
        labels[np.asarray(ess, dtype=np.float64) < ess_min] = 0
    return labels, band


def flock_neighbours(states, k=7):
    """Each agent's k nearest other agents (positions = state components 0..2, FP64
    distances, library k-d tree), their positions [M, 3k] and the circular mean of their
    headings psibar = atan2(sum sin psi_j, sum cos psi_j) (Appendix D.5, per-agent
    reading of the heading average)."""
    from scipy.spatial import cKDTree
    st = np.asarray(states, dtype=np.float64)
    pos = st[:, :3]
    M = len(st)
    d, idx = cKDTree(pos).query(pos, k=k + 1)
    out = np.empty((M, k), dtype=np.int64)
    for i in range(M):
        row = [j for j in idx[i] if j != i][:k]
        out[i] = row
    nbr = pos[out].reshape(M, 3 * k)
    psi = st[:, 3]
    psibar = np.arctan2(np.sin(psi[out]).sum(1), np.cos(psi[out]).sum(1))
    return out, nbr, psibar


def num_threads() -> int:
    return int(lib().orc_num_threads())
