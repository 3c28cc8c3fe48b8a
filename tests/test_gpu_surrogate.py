"""What the learned part gains over the method without it (3-D Dubins game; the 45-D game
in its own test below).

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


def test_surrogate_assisted_45d_needs_fewer_sweeps():
    """The 45-D game on the paper's wide domain (positions uniform in [-100, 100]).  A network
    on the game's invariant frame (hjg_frame_features: the evader at the origin, pursuers by
    distance; 56 inputs) is trained on the correction (v - l, Dv - Dl) that 12 tilted
    control-variate sweeps make to the initial iterate (hjg_frame_targets, averaged over the
    last four sweeps), and warm-starts the same sweep with the position rows of its gradient
    (hjg_warm_start_frame, positions only).  Against a tilted N = 2^20 reference on 1,024
    held-out states, the assisted form after 3 sweeps
      * is clearly closer than the same sweep started from l after 3 sweeps,
      * is as close as the sweep from l after 12 (4x fewer point-samples), and
      * at N = 4,096 is closer than the plain form (Algorithm 1 as printed: untilted, from l,
        no control variate) at N = 16,384 and 12 sweeps (16x fewer point-samples)."""
    from paper_2605_18566_gb300 import Solver, Surrogate
    w = hjg_inputs.ROCKETS45
    X, Y = [], []
    for chunk in range(4):
        x = torch.from_numpy(hjg_inputs.rockets45_wide_points(262144, 100 + chunk)).cuda()
        s = Solver(w.game, w.nu, w.T, 16384, 12, radius=w.radius, tilt=True, cv=True)
        s.set_points(x)
        X.append(s.frame_features())
        s.picard_sweep(8, residuals=False)
        acc = None
        for _ in range(4):
            s.picard_sweep(1, residuals=False)
            t = s.frame_targets()
            acc = t if acc is None else acc + t
        Y.append(acc / 4)
        s.close()
    X, Y = torch.cat(X), torch.cat(Y)
    perm = torch.from_numpy(np.random.default_rng(0).permutation(X.shape[0])).cuda()
    X, Y = X[perm].contiguous(), Y[perm].contiguous()
    sur = Surrogate(56, 43, 256, seed=0)
    hist = sur.fit(X, Y, epochs=30, batch=8192, lr=2e-3, lr_final=1e-4)
    assert hist[-1] < hist[0]

    xte = torch.from_numpy(hjg_inputs.rockets45_wide_points(1024, 1)).cuda()
    probe = Solver(w.game, w.nu, w.T, 1024, 1, radius=w.radius)
    probe.set_points(xte)
    pred = sur.forward(probe.frame_features())
    probe.close()
    sur.close()

    def run(N, K, tilt=True, cv=True, warm=False, seed=11):
        s = Solver(w.game, w.nu, w.T, N, K, radius=w.radius, tilt=tilt, cv=cv, seed=seed)
        s.set_points(xte)
        if warm:
            s.warm_start_frame(pred, positions_only=True)
        s.picard_sweep(K)
        v = s.get_state()["v"].cpu().numpy()
        s.close()
        return v

    vref = run(1 << 20, 12, cv=False, seed=7)   # its own error is well below the compared ones
    err = lambda v: float(np.sqrt(np.mean((v - vref) ** 2)))
    e_net3 = err(run(16384, 3, warm=True))
    e_l3 = err(run(16384, 3))
    e_l12 = err(run(16384, 12))
    e_net3_small = err(run(4096, 3, warm=True))
    e_plain = err(run(16384, 12, tilt=False, cv=False))
    print("45-D value error: network + tilt + cv, 3 sweeps %.3f (N = 4,096: %.3f); from l, 3 sweeps %.3f, "
          "12 sweeps %.3f; plain, 12 sweeps %.3f" % (e_net3, e_net3_small, e_l3, e_l12, e_plain))
    assert e_net3 <= 0.75 * e_l3
    assert e_net3 <= 1.1 * e_l12
    assert e_net3_small <= e_plain
