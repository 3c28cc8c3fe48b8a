"""The seeded synthetic workloads follow their stated recipes: sizes, sample counts, sweeps,
viscosities and horizons of each workload; grid layouts and index order; the ranges and
moments of the scattered states; FP32 values; determinism in the seed."""
import math

import numpy as np

import hjg_inputs as I


def test_workload_table():
    expect = {   # name: (game, n, nu, T, M, N, K)
        "dubins3_grid16": ("dubins3", 3, 0.1, 1.0, 4096, 4096, 10),
        "rockets6_uniform": ("rockets6", 6, 0.05, 2.0, 65536, 65536, 20),
        "rockets45_gauss": ("rockets45", 45, 0.05, 2.0, 262144, 131072, 30),
        "flock_murmuration": ("flock4", 4, 0.02, 1.0, 100000, 16384, 15),
        "rockets_rel3_grid25": ("rockets_rel3", 3, 0.04, 1.0, 15625, 14000, 12),
        "double_int2_grid64": ("double_int2", 2, 0.04, 0.8, 4096, 8000, 15),
    }
    assert set(I.WORKLOADS) == set(expect)
    for name, (game, n, nu, T, M, N, K) in expect.items():
        w = I.WORKLOADS[name]
        assert (w.game, w.n, w.nu, w.T, w.M, w.N, w.K) == (game, n, nu, T, M, N, K), name
        assert w.delta == 2 * nu and math.isclose(w.sigma2, 2 * nu * T)
    for w, states in I.MIXED:   # every mixed-batch instance at nu = 0.02, T = 1, N = 16,384, 15 sweeps
        assert w.name in I.WORKLOADS and states > 0


def test_grids_and_index_order():
    g = I.points(I.DUBINS3)
    assert g.shape == (4096, 3) and g.dtype == np.float32
    a = np.linspace(-2, 2, 16).astype(np.float32)
    th = np.linspace(-math.pi, math.pi, 16).astype(np.float32)
    for i1, i2, i3 in ((0, 0, 0), (3, 7, 11), (15, 15, 15)):
        np.testing.assert_array_equal(g[(i1 * 16 + i2) * 16 + i3], [a[i1], a[i2], th[i3]])
    r = I.points(I.ROCKETS_REL3)
    assert r.shape == (15625, 3)
    np.testing.assert_allclose(r.min(0), [-100, -100, -math.pi / 2], rtol=1e-6)
    np.testing.assert_allclose(r.max(0), [100, 100, math.pi / 2], rtol=1e-6)
    d = I.points(I.DOUBLE_INT2)
    assert d.shape == (4096, 2) and len(np.unique(d[:, 0])) == 64
    np.testing.assert_allclose(d[1] - d[0], [0, 4 / 63], rtol=1e-6)   # last axis fastest


def test_scattered_states_follow_their_distributions():
    x = I.points(I.ROCKETS6)
    assert x.shape == (65536, 6) and x.dtype == np.float32
    assert np.all(np.abs(x[:, :4]) <= 3) and np.all(np.abs(x[:, 4:]) <= math.pi)
    np.testing.assert_allclose(x[:, :4].std(0), 6 / math.sqrt(12), rtol=0.02)
    np.testing.assert_allclose(x[:, 4:].std(0), 2 * math.pi / math.sqrt(12), rtol=0.02)
    y = I.rockets45_points(20000, 0).reshape(-1, 15, 3)
    np.testing.assert_allclose(y[:, :, :2].std(), 2.0, rtol=0.01)
    assert abs(y[:, :, :2].mean()) < 0.02
    assert np.all(np.abs(y[:, :, 2]) <= math.pi)
    np.testing.assert_allclose(y[:, :, 2].std(), 2 * math.pi / math.sqrt(12), rtol=0.01)
    z = I.rockets45_wide_points(20000, 0).reshape(-1, 15, 3)
    assert np.all(np.abs(z[:, :, :2]) <= 100) and z[:, :, :2].std() > 50
    f = I.flock_states(6000, 0)
    k = np.arange(6000) % 6
    for c in range(6):   # six clusters on a ring of radius 40, headings along its tangent
        ang = 2 * math.pi * c / 6
        np.testing.assert_allclose(f[k == c, :2].mean(0), [40 * math.cos(ang), 40 * math.sin(ang)], atol=0.3)
        dpsi = np.angle(np.exp(1j * (f[k == c, 3] - (ang + math.pi / 2))))
        assert abs(dpsi.mean()) < 0.03 and abs(dpsi.std() - 0.3) < 0.03


def test_seeded_and_keyed():
    a = I.rockets6_points(100, seed=3)
    np.testing.assert_array_equal(a, I.rockets6_points(100, seed=3))
    assert not np.array_equal(a, I.rockets6_points(100, seed=4))
    # the state stream is keyed apart from an unkeyed Philox stream of the same seed
    plain = np.random.Generator(np.random.Philox(key=3)).uniform(-3.0, 3.0, size=(100, 4))
    assert not np.allclose(a[:, :4], plain.astype(np.float32))
    # grid workloads: the first M states of the grid; scattered ones: M states of the recipe
    np.testing.assert_array_equal(I.points(I.DUBINS3, M=10), I.points(I.DUBINS3)[:10])
    np.testing.assert_array_equal(I.points(I.ROCKETS6, M=10), I.rockets6_points(10))
