"""What the learned part gains over the method without it (3-D Dubins game).

A surrogate network is trained on the GPU on (x, v, Dv) tuples produced by the sweeps
themselves, then measured by the sweep: against a high-sample reference solve, compare
  * the plain form (Algorithm 1 as printed: untilted proposal, start at v = g),
  * the surrogate's own prediction (no samples at query time),
  * the surrogate-assisted form (warm start v, Dv, c = Gamma(Dv) from the network, tilted
    proposal theta = -sigma^2 c Dv, Eq. tilt_shift) with four times fewer samples than
    the plain form's best run here,
and also report the tilted form started from g, which gets the same tilt without the
network, so the two sources of the gain stay apart.
"""
import math

import numpy as np
import pytest

import hjg_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W = hjg_inputs.DUBINS3


def _states(M, seed):
    r = np.random.default_rng(100 + seed)
    return np.stack([r.uniform(-2, 2, M), r.uniform(-2, 2, M),
                     r.uniform(-math.pi, math.pi, M)], 1).astype(np.float32)


def _solve(x, N, K, tilt=False, warm=None, seed=0, record=0):
    from paper_2605_18566_gb300 import Solver
    s = Solver(W.game, W.nu, W.T, N, K, radius=W.radius, tilt=tilt, seed=seed)
    s.set_points(x)
    if warm is not None:
        s.warm_start(warm[1], warm[0])
    rec = []
    for k in range(K):
        r, _ = s.picard_sweep(1)
        if k >= K - record:
            st = s.get_state()
            rec.append((st["v"].clone(), st["p"].clone()))
    st = s.get_state()
    s.close()
    return st, float(r[0]), rec


def test_surrogate_gain_over_plain_form():
    from paper_2605_18566_gb300 import Surrogate
    xtr = torch.from_numpy(_states(16384, 0)).cuda()
    _, _, rec = _solve(xtr, 8192, 14, tilt=True, record=6)
    X = torch.cat([xtr] * len(rec))
    Y = torch.cat([torch.cat([v[:, None].float(), p], 1) for v, p in rec])
    perm = torch.from_numpy(np.random.default_rng(0).permutation(X.shape[0])).cuda()
    X, Y = X[perm].contiguous(), Y[perm].contiguous()
    sur = Surrogate(3, 4, 256, seed=0)
    hist = sur.fit(X, Y, epochs=30, batch=4096, lr=2e-3, lr_final=1e-4)
    assert hist[-1] < 0.5 * hist[0]   # loss on standardised targets

    xte = torch.from_numpy(_states(256, 1)).cuda()
    ref, _, _ = _solve(xte, 1 << 18, 16, tilt=True, seed=7)
    vref = ref["v"].cpu().numpy()

    def err(st):
        return float(np.sqrt(np.mean((st["v"].cpu().numpy() - vref) ** 2)))

    plain, plain_res, _ = _solve(xte, 16384, 16, seed=11)             # 262,144 samples/state
    pred = sur.forward(xte)
    v_sur, p_sur = pred[:, 0].double().contiguous(), pred[:, 1:].contiguous()
    e_sur = float(np.sqrt(np.mean((v_sur.cpu().numpy() - vref) ** 2)))
    assisted, assisted_res, _ = _solve(xte, 4096, 16, tilt=True, warm=(v_sur, p_sur), seed=11)
    tilted, tilted_res, _ = _solve(xte, 4096, 16, tilt=True, seed=11)  # same tilt, no network
    sur.close()
    e_plain, e_assisted, e_tilted = err(plain), err(assisted), err(tilted)
    print("value error vs reference: plain %.4f (262144 samples, residual %.4f), surrogate alone "
          "%.4f (0 samples), surrogate-assisted %.4f (65536 samples, residual %.4f), tilted "
          "without network %.4f (65536 samples, residual %.4f)"
          % (e_plain, plain_res, e_sur, e_assisted, assisted_res, e_tilted, tilted_res))
    # the network alone is already more accurate than the plain form's floor
    assert e_sur < e_plain
    # the assisted form reaches the plain form's residual floor and value error with 4x
    # fewer point-samples
    assert e_assisted <= e_plain and assisted_res <= plain_res


def test_surrogate_assisted_45d_against_plain_and_tilt():
    """The 45-D game on the paper's wide domain (positions uniform in [-100, 100]): a network
    trained on the correction (v - l, Dv - Dl) that the plain sweeps make to the initial
    iterate warm-starts the tilted, control-variate sweep (hjg_warm_start_delta).  Against
    a tilted N = 2^18 reference, the assisted form with 4x fewer point-samples than the plain
    form reaches a smaller value error and residual, and at equal samples it beats the
    tilted form started from l without control variate.  The same sweep without the network
    (tilt + control variate from l) is measured beside it: the printed line shows which part
    of the gain the network itself contributes."""
    from paper_2605_18566_gb300 import Solver, Surrogate
    w = hjg_inputs.ROCKETS45
    K = 12

    def run(x, N, tilt=False, cv=False, warm=None, seed=11):
        s = Solver(w.game, w.nu, w.T, N, K, radius=w.radius, tilt=tilt, cv=cv, seed=seed)
        s.set_points(x)
        if warm is not None:
            s.warm_start_delta(warm)
        r, _ = s.picard_sweep(K)
        out = (s.get_state()["v"].cpu().numpy(), float(r[-1]), s)
        return out

    xtr = torch.from_numpy(hjg_inputs.rockets45_wide_points(65536, 0)).cuda()
    s = Solver(w.game, w.nu, w.T, 16384, K, radius=w.radius, tilt=True)
    s.set_points(xtr)
    s.picard_sweep(K - 6)
    X, Y = [], []
    for _ in range(6):
        s.picard_sweep(1)
        X.append(xtr); Y.append(s.state_delta())
    s.close()
    X, Y = torch.cat(X), torch.cat(Y)
    perm = torch.from_numpy(np.random.default_rng(0).permutation(X.shape[0])).cuda()
    X, Y = X[perm].contiguous(), Y[perm].contiguous()
    sur = Surrogate(45, 46, 256, seed=0)
    hist = sur.fit(X, Y, epochs=20, batch=8192, lr=2e-3, lr_final=1e-4)
    assert hist[-1] < hist[0]

    xte = torch.from_numpy(hjg_inputs.rockets45_wide_points(512, 1)).cuda()
    pred = sur.forward(xte)
    sur.close()
    vref, _, s = run(xte, 1 << 18, tilt=True, seed=7); s.close()

    def err(v):
        return float(np.sqrt(np.mean((v - vref) ** 2)))
    res = {}
    for name, N, kw in (("plain", 16384, {}), ("tilt", 4096, dict(tilt=True)),
                        ("tilt+cv", 4096, dict(tilt=True, cv=True)),
                        ("assisted", 4096, dict(tilt=True, cv=True, warm=pred))):
        v, r, s = run(xte, N, **kw)
        s.close()
        res[name] = (err(v), r)
    print("45-D value error (residual): " + ", ".join("%s %.3f (%.4f)" % (k, e, r) for k, (e, r) in res.items()))
    e_a, r_a = res["assisted"]
    assert e_a <= res["plain"][0] and r_a <= res["plain"][1]      # 4x fewer point-samples than plain
    assert e_a <= res["tilt"][0]                                   # beats the tilt from l alone
    assert res["tilt+cv"][0] <= res["tilt"][0]                     # the control variate's share
