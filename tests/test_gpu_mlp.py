"""The surrogate network's tensor-core kernels against the FP64 reference (oracle/mlp.py):
forward outputs and every parameter gradient, at a ragged batch size; training lowers the
loss; the warm start sets c = Gamma(Dv) like the oracle's coefficient map."""
import numpy as np
import pytest

import hjg_inputs
import oracle
from oracle import mlp as omlp
from helpers import problem_for, solver_for

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_IN, N_OUT, WIDTH = 45, 46, 256


def _sur(seed=1, n_in=N_IN, n_out=N_OUT):
    from paper_2605_18566_gb300 import Surrogate
    return Surrogate(n_in, n_out, WIDTH, seed=seed)


def test_forward_matches_reference():
    s = _sur()
    x = hjg_inputs.random_states(300, N_IN, 1.5, seed=3)
    out = s.forward(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    p = s.params()
    ref_bf, _ = omlp.forward(p, x.astype(np.float64), N_IN, N_OUT, WIDTH, bf16=True)
    ref64, _ = omlp.forward(p, x.astype(np.float64), N_IN, N_OUT, WIDTH, bf16=False)
    scale = np.abs(ref64).max()
    assert np.abs(out - ref_bf).max() <= 1e-2 * scale
    assert np.median(np.abs(out - ref_bf)) <= 1e-3 * scale
    assert np.abs(out - ref64).max() <= 5e-2 * scale
    s.close()


# (45, 46): the state-coordinate network of the 45-D game (input pad 48); (56, 43): its
# invariant-frame network (input pad 64, the largest the fused step takes; output pad 48)
@pytest.mark.parametrize("n_in,n_out", [(N_IN, N_OUT), (56, 43)])
def test_gradients_match_reference(n_in, n_out):
    s = _sur(seed=2, n_in=n_in, n_out=n_out)
    rng = np.random.default_rng(4)
    x = hjg_inputs.random_states(300, n_in, 1.5, seed=5)
    y = rng.normal(size=(300, n_out)).astype(np.float32)
    loss, g = s.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    p = s.params()
    rloss, rg = omlp.loss_and_grads(p, x.astype(np.float64), y.astype(np.float64), n_in, n_out,
                                    WIDTH, bf16=True)
    assert abs(loss - rloss) <= 1e-3 * rloss
    lay, _ = omlp.layout(n_in, n_out, WIDTH)
    for (w, o, i, b) in lay:
        for a, z in ((w, w + o * i), (b, b + o)):
            gg, rr = g[a:z].astype(np.float64), rg[a:z]
            assert np.linalg.norm(gg - rr) <= 2e-2 * np.linalg.norm(rr) + 1e-12, (a, z)
    # padded outputs/inputs receive no gradient
    w4, o4, i4, b4 = lay[3]
    assert np.all(g[w4:w4 + o4 * i4].reshape(o4, i4)[n_out:] == 0)
    w1, o1, i1, b1 = lay[0]
    assert np.all(g[w1:w1 + o1 * i1].reshape(o1, i1)[:, n_in:] == 0)
    s.close()


def test_training_lowers_loss():
    s = _sur(seed=3)
    rng = np.random.default_rng(5)
    x = rng.uniform(-2, 2, size=(16384, N_IN)).astype(np.float32)
    y = np.concatenate([np.sin(x).sum(1, keepdims=True) / 10, np.cos(x) / 10], 1).astype(np.float32)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    hist = s.fit(xt, yt, epochs=40, batch=2048, lr=2e-3, lr_final=1e-4, standardize=False)
    assert hist[-1] < 0.35 * hist[0], hist
    assert all(b <= a * 1.05 for a, b in zip(hist, hist[1:])), hist   # steady descent
    out = s.forward(xt).cpu().numpy()
    r2 = 1.0 - np.mean((out[:, 0] - y[:, 0]) ** 2) / np.var(y[:, 0])
    assert r2 > 0.8, r2
    s.close()


def test_warm_start_sets_gamma():
    w = hjg_inputs.ROCKETS45
    x = hjg_inputs.points(w, M=200)
    rng = np.random.default_rng(6)
    p0 = (0.3 * rng.normal(size=(200, 45))).astype(np.float32)
    v0 = rng.normal(size=200)
    s = solver_for(w, N=1024, K=1)
    s.set_points(torch.from_numpy(x).cuda())
    s.warm_start(torch.from_numpy(p0).cuda(), torch.from_numpy(v0).cuda())
    st = {k: t.cpu().numpy() for k, t in s.get_state().items()}
    s.close()
    np.testing.assert_array_equal(st["p"], p0)
    np.testing.assert_array_equal(st["v"], v0)
    c_ref = oracle.coef_batch(problem_for(w), x.astype(np.float64), p0.astype(np.float64))
    np.testing.assert_allclose(st["c"], c_ref, rtol=1e-6)


def test_input_gradient_matches_reference():
    s = _sur(seed=4)
    x = hjg_inputs.random_states(130, N_IN, 1.0, seed=9).astype(np.float64)
    gx = s.input_grad(torch.from_numpy(x.astype(np.float32)).cuda(), 0).cpu().numpy()
    p = s.params()
    h = 1e-5
    fd = np.zeros_like(x)
    for a in range(N_IN):          # central differences of the FP64 reference's output 0
        e = np.zeros(N_IN); e[a] = h
        up, _ = omlp.forward(p, x + e, N_IN, N_OUT, WIDTH)
        dn, _ = omlp.forward(p, x - e, N_IN, N_OUT, WIDTH)
        fd[:, a] = (up[:, 0] - dn[:, 0]) / (2 * h)
    assert np.linalg.norm(gx - fd) <= 3e-2 * np.linalg.norm(fd)
    s.close()


def test_scaling_forward_gradients_and_input_grad():
    """Standardisation fitted on the device equals numpy's mean / std; forward outputs,
    parameter gradients and input gradients with it match the FP64 reference."""
    s = _sur(seed=5)
    rng = np.random.default_rng(8)
    x = (rng.normal(size=(400, N_IN)) * rng.uniform(0.5, 80, N_IN) + rng.normal(size=N_IN) * 20).astype(np.float32)
    y = (rng.normal(size=(400, N_OUT)) * rng.uniform(0.1, 50, N_OUT) + 5).astype(np.float32)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    s.fit_scaling(xt, yt)
    sc = s.scaling().astype(np.float64)
    a, m_in = sc[:N_IN], sc[N_IN:2 * N_IN]
    b, m_out = sc[2 * N_IN:2 * N_IN + N_OUT], sc[2 * N_IN + N_OUT:]
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    np.testing.assert_allclose(a, xd.mean(0), rtol=1e-5, atol=1e-4)
    np.testing.assert_allclose(1.0 / m_in, xd.std(0), rtol=1e-4)
    np.testing.assert_allclose(b, yd.mean(0), rtol=1e-5, atol=1e-4)
    np.testing.assert_allclose(m_out, yd.std(0), rtol=1e-4)
    scaling = (a, m_in, b, m_out)
    p = s.params()
    out = s.forward(xt).cpu().numpy().astype(np.float64)
    ref, _ = omlp.forward(p, xd, N_IN, N_OUT, WIDTH, bf16=True, scaling=scaling)
    assert np.abs(out - ref).max() <= 1e-2 * np.abs(ref).max()
    loss, g = s.gradients(xt, yt)
    rloss, rg = omlp.loss_and_grads(p, xd, yd, N_IN, N_OUT, WIDTH, bf16=True, scaling=scaling)
    assert abs(loss - rloss) <= 1e-3 * rloss
    assert np.linalg.norm(g.astype(np.float64) - rg) <= 2e-2 * np.linalg.norm(rg)
    gx = s.input_grad(xt[:50].contiguous(), 3).cpu().numpy().astype(np.float64)
    h = 1e-4 * np.abs(xd[:50]).max()
    fd = np.zeros((50, N_IN))
    for i in range(N_IN):
        e = np.zeros(N_IN); e[i] = h
        up, _ = omlp.forward(p, xd[:50] + e, N_IN, N_OUT, WIDTH, scaling=scaling)
        dn, _ = omlp.forward(p, xd[:50] - e, N_IN, N_OUT, WIDTH, scaling=scaling)
        fd[:, i] = (up[:, 3] - dn[:, 3]) / (2 * h)
    assert np.linalg.norm(gx - fd) <= 3e-2 * np.linalg.norm(fd)
    s2 = _sur(seed=6)
    s2.set_scaling(s.scaling())
    np.testing.assert_array_equal(s2.scaling(), s.scaling())
    s2.close()
    s.close()


def test_save_and_load_reproduce_predictions(tmp_path):
    """A trained network with fitted standardisation, written by save() and read by load(),
    predicts the same values bit for bit."""
    from paper_2605_18566_gb300 import Surrogate
    s = _sur(seed=4)
    rng = np.random.default_rng(6)
    x = rng.uniform(-50, 50, size=(4096, N_IN)).astype(np.float32)
    y = rng.normal(size=(4096, N_OUT)).astype(np.float32) * 3 + 1
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    s.fit(xt, yt, epochs=2, batch=1024)
    path = str(tmp_path / "net.npz")
    s.save(path)
    t = Surrogate.load(path)
    assert (t.n_in, t.n_out, t.width) == (N_IN, N_OUT, WIDTH)
    np.testing.assert_array_equal(t.params(), s.params())
    np.testing.assert_array_equal(t.scaling(), s.scaling())
    np.testing.assert_array_equal(t.forward(xt).cpu().numpy(), s.forward(xt).cpu().numpy())
    s.close(); t.close()


def test_gradients_after_an_in_stream_producer():
    """The training kernels are launched as programmatic dependents of the kernel before
    them and wait before their first global read: inputs written by a kernel queued on the
    same stream just before the step give the same gradients, bit for bit, as inputs that
    were complete (synchronised) beforehand."""
    s = _sur(seed=6)
    rng = np.random.default_rng(8)
    x0 = torch.from_numpy(hjg_inputs.random_states(1000, N_IN, 1.5, seed=9)).cuda()
    y0 = torch.from_numpy(rng.normal(size=(1000, N_OUT)).astype(np.float32)).cuda()
    torch.cuda.synchronize()
    loss_ref, g_ref = s.gradients(x0, y0)
    for _ in range(3):
        x = x0 * 1.0 + 0.0        # kernels on the current stream, not waited for on the host
        y = (y0 * 2.0) * 0.5
        loss, g = s.gradients(x, y)
        assert loss == loss_ref
        np.testing.assert_array_equal(g, g_ref)
    s.close()
