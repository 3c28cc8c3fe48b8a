"""Topology markers on the GPU (hjg_topology) against the oracle (scipy labelling).

The smoothed field is compared with the oracle's smoothing; the markers, events and the
partition into components are compared exactly, with the oracle labelling the GPU's own
smoothed field (both threshold in FP64, so only the summation order of the filter could
move a cell across zero; such cells are excluded from nothing because none lie within
1e-12 of zero in these fields, which the test checks)."""
import numpy as np
import pytest

import hjg_inputs
from helpers import solver_for

torch = pytest.importorskip("torch")
pytest.importorskip("scipy")
from oracle import topology as otopo  # noqa: E402

pytestmark = pytest.mark.gpu


def _check(v, cells):
    from paper_2605_18566_gb300 import topology
    from scipy import ndimage
    vt = torch.from_numpy(np.ascontiguousarray(v)).cuda()
    mk, ev, sm, lab = topology(vt, cells)
    sm = sm.cpu().numpy(); lab = lab.cpu().numpy()
    ref_sm = otopo.smooth(v, cells)
    np.testing.assert_allclose(sm, ref_sm, rtol=1e-12, atol=1e-12 * np.abs(v).max())
    assert np.all(np.abs(sm) > 1e-12 * np.abs(v).max())   # no cell decided by rounding
    mk_ref, ev_ref, _ = otopo.markers(sm, cells=0.0)
    np.testing.assert_array_equal(mk, mk_ref)
    np.testing.assert_array_equal(ev, ev_ref)
    for h in range(v.shape[0]):   # the same partition of the set cells
        fg = sm[h] <= 0
        sl, n = ndimage.label(fg, structure=otopo._CROSS)
        pairs = {(int(a), int(b)) for a, b in zip(lab[h][fg], sl[fg])}
        assert len(pairs) == n == len({a for a, _ in pairs})
    return mk, ev


def test_known_shapes_and_events():
    m = 96
    I, J = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    d = np.hypot(I - 48.3, J - 47.7)
    seq = np.stack([d - 15.2, np.maximum(9.1 - d, d - 24.6), np.maximum(9.1 - d, d - 24.6),
                    np.minimum(np.hypot(I - 20.4, J - 20.1) - 7.3, np.hypot(I - 70.2, J - 71.6) - 7.7),
                    d - 15.2])
    mk, ev = _check(seq, 0.0)
    assert [tuple(x) for x in mk] == [(1, 0, 1), (1, 1, 0), (1, 1, 0), (2, 0, 2), (1, 0, 1)]
    assert list(ev) == [0, 3, 0, 4, 1]


@pytest.mark.parametrize("H,m,cells", [(18, 128, 1.5), (5, 37, 1.5), (3, 64, 0.0), (2, 200, 3.0)])
def test_random_fields(H, m, cells):
    rng = np.random.default_rng(H * m)
    v = rng.normal(size=(H, m, m)) + rng.uniform(-0.3, 0.3, size=(H, 1, 1))
    _check(v, cells)


def test_value_slices_at_several_horizons():
    """A 64 x 64 slice of the Dubins game (x3 = 0.4) solved at 6 horizons in one solve."""
    w = hjg_inputs.DUBINS3
    m, times = 64, [0.2, 0.5, 0.8, 1.2, 1.6, 2.0]
    a = np.linspace(-2.0, 2.0, m)
    X = np.stack(np.meshgrid(a, a, indexing="ij"), -1).reshape(-1, 2)
    x = np.concatenate([X, np.full((m * m, 1), 0.4)], 1).astype(np.float32)
    s = solver_for(w, N=2048, K=4)
    s.set_horizons(times)
    s.set_points(torch.from_numpy(x).cuda())
    s.picard_sweep(4)
    v = s.get_state()["v"].reshape(len(times), m, m)
    s.close()
    mk, ev = _check(v.cpu().numpy(), 1.5)
    assert np.all(mk[:, 0] >= 1)
