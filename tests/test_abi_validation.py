"""Argument validation at the C boundary, without a GPU: hjg_create and the allocation-free
entry point check their arguments before touching the device, so every refusal below is
the status the header documents (and no context is created)."""
import ctypes as C

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2605_18566_gb300 import build as B, _lib
    B.build()
    return _lib.load(), _lib


def _args(_lib, game="dubins3", n=3, N=1024, K=2):
    dyn = _lib.Dynamics(); dyn.game = _lib.GAMES[game]; dyn.n = n; dyn.h_sign = 1.0
    tgt = _lib.Target(); tgt.radius = 0.5
    opt = _lib.Options(); opt.N = N; opt.K = K; opt.eta = -1.0
    return dyn, tgt, opt


def _create(L, dyn, tgt, opt, nu=0.1, T=1.0):
    ctx = C.c_void_p()
    st = L.hjg_create(C.byref(dyn), C.byref(tgt), nu, T, C.byref(opt), C.byref(ctx))
    assert not ctx.value or st == 0
    return st


def test_refusals_before_any_device_work(lib):
    L, _lib = lib
    # obstacle on a game without a position plane
    dyn, tgt, opt = _args(_lib, "rockets6", 6)
    tgt.obstacle_radius = 1.0
    assert _create(L, dyn, tgt, opt) == _lib.HJG_EUNSUPPORTED
    # negative obstacle radius
    dyn, tgt, opt = _args(_lib)
    tgt.obstacle_radius = -1.0
    assert _create(L, dyn, tgt, opt) == _lib.HJG_EUNSUPPORTED
    # unknown precision; FP64 sweep for the 45-D game
    dyn, tgt, opt = _args(_lib)
    opt.precision = 2
    assert _create(L, dyn, tgt, opt) == _lib.HJG_EINVAL
    dyn, tgt, opt = _args(_lib, "rockets45", 45)
    opt.precision = 1
    assert _create(L, dyn, tgt, opt) == _lib.HJG_EUNSUPPORTED
    # a state dimension the game does not have
    dyn, tgt, opt = _args(_lib, "dubins3", 4)
    assert _create(L, dyn, tgt, opt) == _lib.HJG_EINVAL
    # sample counts: zero, 2^32, and past the 2^32-block stream of the 45-D game
    for N in (0, 1 << 32):
        dyn, tgt, opt = _args(_lib, N=N)
        assert _create(L, dyn, tgt, opt) == _lib.HJG_EINVAL
    dyn, tgt, opt = _args(_lib, "rockets45", 45, N=(1 << 32) // 6 + 1)   # 6 blocks per sample
    assert _create(L, dyn, tgt, opt) == _lib.HJG_EINVAL
    # viscosity and horizon must be positive and finite
    dyn, tgt, opt = _args(_lib)
    assert _create(L, dyn, tgt, opt, nu=0.0) == _lib.HJG_EINVAL
    assert _create(L, dyn, tgt, opt, T=float("inf")) == _lib.HJG_EINVAL
    # clip bounds out of order
    dyn, tgt, opt = _args(_lib)
    opt.c_min, opt.c_max = 10.0, 1.0
    assert _create(L, dyn, tgt, opt) == _lib.HJG_EINVAL


def test_noalloc_refusals_before_any_device_work(lib):
    L, _lib = lib
    dyn, tgt, opt = _args(_lib, "rockets6", 6)
    tgt.obstacle_radius = 1.0

    def call(dyn, tgt, opt, M=4):
        return L.hjg_value_grad_noalloc(C.byref(dyn), C.byref(tgt), 0.1, 1.0, C.byref(opt), None, M, 8,
                                        None, None, 8, None, None)
    assert call(dyn, tgt, opt) == _lib.HJG_EUNSUPPORTED
    dyn, tgt, opt = _args(_lib)
    opt.point_offset = 0xFFFFFFFF
    assert call(dyn, tgt, opt, M=2) == _lib.HJG_EINVAL
    dyn, tgt, opt = _args(_lib)
    opt.precision = 3
    assert call(dyn, tgt, opt) == _lib.HJG_EINVAL
    # the option checks come before the pointer checks: an FP64 sweep of the 45-D game is
    # refused as unsupported even though no buffers are given
    dyn, tgt, opt = _args(_lib, "rockets45", 45)
    opt.precision = 1
    assert call(dyn, tgt, opt) == _lib.HJG_EUNSUPPORTED
    # the flock's neighbour data needs per-agent storage: not on the allocation-free path
    dyn, tgt, opt = _args(_lib, "flock4", 4)
    assert call(dyn, tgt, opt) == _lib.HJG_EINVAL
    # no sweeps requested
    dyn, tgt, opt = _args(_lib, K=0)
    assert call(dyn, tgt, opt) == _lib.HJG_EINVAL
    # a CTA size the game has no launch variant for (the 6-D game has 128 and 256)
    dyn, tgt, opt = _args(_lib, "rockets6", 6)
    opt.block_threads = 96
    assert call(dyn, tgt, opt) == _lib.HJG_EINVAL


def test_mlp_refusals_before_any_device_work(lib):
    """hjg_mlp_create rejects shapes outside its documented range, and hjg_mlp_fit refuses a
    missing network or a non-positive epoch count, batch or learning rate before it launches
    anything."""
    L, _lib = lib
    m = C.c_void_p()
    assert L.hjg_mlp_create(0, 4, 256, 0, C.byref(m)) == _lib.HJG_EINVAL and not m.value
    assert L.hjg_mlp_create(3, 4, 250, 0, C.byref(m)) == _lib.HJG_EINVAL and not m.value
    hist = (C.c_double * 2)()
    buf = C.c_void_p(8)   # never dereferenced: every call below fails its argument check
    assert L.hjg_mlp_fit(None, buf, 3, buf, 4, 16, 2, 8, 1e-3, 1e-4, 0, hist) == _lib.HJG_EINVAL
