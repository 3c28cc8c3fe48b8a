"""Pins for the FP64 surrogate-network reference: finite differences of its loss match its
hand-written backward pass, and the bfloat16 rounding helper matches exact references."""
import numpy as np

from oracle import mlp


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2**-8, 1.0 + 2**-7, 1.0 + 3 * 2**-8, -2.5, 0.0, 3.14159265])
    r = mlp.to_bf16(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0                     # halfway, ties to even (mantissa 0)
    assert r[2] == 1.0 + 2**-7
    assert r[3] == 1.0 + 2 * 2**-7         # halfway, ties to even (odd -> even up)
    assert r[4] == -2.5 and r[5] == 0.0
    assert abs(r[6] - 3.140625) < 1e-12


def test_backward_matches_finite_differences():
    n_in, n_out, width = 3, 4, 16
    lay, total = mlp.layout(n_in, n_out, width)
    rng = np.random.default_rng(0)
    params = rng.normal(0, 0.3, size=total)
    # padded rows/cols carry no information: zero them as the GPU initialisation does
    for (w, o, i, b) in lay:
        W = params[w:w + o * i].reshape(o, i)
        if i == mlp.pad16(n_in):
            W[:, n_in:] = 0.0
        if o == mlp.pad16(n_out):
            W[n_out:, :] = 0.0
            params[b + n_out:b + o] = 0.0
    x = rng.normal(size=(7, n_in)); y = rng.normal(size=(7, n_out))
    loss, g = mlp.loss_and_grads(params, x, y, n_in, n_out, width)
    h = 1e-6
    for k in rng.choice(total, size=60, replace=False):
        e = np.zeros(total); e[k] = h
        lp, _ = mlp.loss_and_grads(params + e, x, y, n_in, n_out, width)
        lm, _ = mlp.loss_and_grads(params - e, x, y, n_in, n_out, width)
        assert abs((lp - lm) / (2 * h) - g[k]) < 1e-6 * (1 + abs(g[k])), k


def test_scaling_is_a_change_of_units():
    """With standardisation (x - a) m_in and outputs o m_out + b, the network's outputs and
    loss equal those of an unscaled network fed the standardised inputs and compared with
    the standardised targets; the backward pass still matches finite differences."""
    n_in, n_out, width = 3, 4, 16
    lay, total = mlp.layout(n_in, n_out, width)
    rng = np.random.default_rng(1)
    params = rng.normal(0, 0.3, size=total)
    for (w, o, i, b) in lay:
        W = params[w:w + o * i].reshape(o, i)
        if i == mlp.pad16(n_in):
            W[:, n_in:] = 0.0
        if o == mlp.pad16(n_out):
            W[n_out:, :] = 0.0
            params[b + n_out:b + o] = 0.0
    sc = (rng.normal(size=n_in), rng.uniform(0.1, 2.0, n_in), rng.normal(size=n_out), rng.uniform(0.5, 20, n_out))
    x = rng.normal(size=(9, n_in)) * 30
    y = rng.normal(size=(9, n_out)) * 10
    out, _ = mlp.forward(params, x, n_in, n_out, width, scaling=sc)
    raw, _ = mlp.forward(params, (x - sc[0]) * sc[1], n_in, n_out, width)
    np.testing.assert_allclose(out, raw * sc[3] + sc[2], rtol=1e-12, atol=1e-12)
    loss, g = mlp.loss_and_grads(params, x, y, n_in, n_out, width, scaling=sc)
    loss_raw, g_raw = mlp.loss_and_grads(params, (x - sc[0]) * sc[1], (y - sc[2]) / sc[3], n_in, n_out, width)
    assert abs(loss - loss_raw) < 1e-12 * (1 + loss)
    np.testing.assert_allclose(g, g_raw, rtol=1e-10, atol=1e-14)
    h = 1e-6
    for k in rng.choice(total, size=30, replace=False):
        e = np.zeros(total); e[k] = h
        lp, _ = mlp.loss_and_grads(params + e, x, y, n_in, n_out, width, scaling=sc)
        lm, _ = mlp.loss_and_grads(params - e, x, y, n_in, n_out, width, scaling=sc)
        assert abs((lp - lm) / (2 * h) - g[k]) < 1e-6 * (1 + abs(g[k])), k
