"""GPU sampler against the oracle: Philox blocks bit-exact, FP32 normals within the error
of the approximate transcendental instructions."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_philox_bit_exact():
    from paper_2605_18566_gb300 import philox_blocks
    r = np.random.default_rng(3)
    K = 100003
    ctr = r.integers(0, 2**32, size=(K, 4), dtype=np.uint64).astype(np.uint32)
    key = r.integers(0, 2**32, size=(K, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 0, 0, 0], [0, 0, 0, 1]]
    key[:4] = [[0, 0], [0xFFFFFFFF] * 2, [0, 0], [0, 0]]
    out = philox_blocks(torch.from_numpy(ctr.view(np.int32)).cuda(),
                        torch.from_numpy(key.view(np.int32)).cuda())
    got = out.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(got, oracle.philox4x32_10(ctr, key))


@pytest.mark.parametrize("n", [3, 6, 45])
def test_normals_match_oracle(n):
    from paper_2605_18566_gb300 import sample_normals
    seed, inst, point, sweep = 0xDEADBEEF12345, 2, 77, 5
    ns = 20000
    z = sample_normals(n, seed, inst, point, sweep, ns).cpu().numpy().astype(np.float64)
    ref = np.array([oracle.normals(n, seed, inst, i, point, sweep) for i in range(ns)])
    err = np.abs(z - ref)
    # radius sqrt(-2 ln u) from an approximate log2: absolute error ~1e-7 in ln u, which
    # the square root amplifies only where u is within ~1e-5 of 1 (radius near 0)
    assert np.quantile(err, 0.999) < 5e-6, np.quantile(err, 0.999)
    assert err.max() < 2e-3, err.max()
    assert np.all(np.isfinite(z))
