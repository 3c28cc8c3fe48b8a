"""The allocation-free solve, hjg_value_grad_noalloc, against hjg_value_grad.

hjg_value_grad_noalloc exists for callers that cannot allocate device memory once they
are running (hard real-time loops, processes whose device memory is owned by another
runtime's allocator, services that reserve everything up front).  It keeps its working
memory in one fixed array inside the library; this test calls it through the C ABI twice
in a row (the second call reuses that array with the first call's contents still in it)
and checks both results against the context-based entry point, state by state, within
the parity tolerance used everywhere else.  The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

import hjg_inputs
from helpers import assert_parity, solver_for

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _structs(w, N, K):
    from paper_2605_18566_gb300 import _lib
    dyn = _lib.Dynamics(); dyn.game = _lib.GAMES[w.game]; dyn.n = w.n; dyn.h_sign = 1.0
    tgt = _lib.Target(); tgt.radius = w.radius
    opt = _lib.Options(); opt.N = N; opt.K = K; opt.eta = -1.0; opt.seed = 0
    return dyn, tgt, opt


def _noalloc(lib, dyn, tgt, nu, T, opt, x, v, g, r, stream):
    return lib.hjg_value_grad_noalloc(C.byref(dyn), C.byref(tgt), nu, T, C.byref(opt),
                                      C.c_void_p(x.data_ptr()), x.shape[0], x.stride(0),
                                      C.c_void_p(v.data_ptr()), C.c_void_p(g.data_ptr()),
                                      g.stride(0), C.c_void_p(r.data_ptr()), stream)


@pytest.mark.parametrize("game", ["dubins3", "rockets6"])
def test_noalloc_matches_value_grad_twice(game):
    from paper_2605_18566_gb300 import Solver, _lib
    lib = _lib.load()
    w = {"dubins3": hjg_inputs.DUBINS3, "rockets6": hjg_inputs.ROCKETS6}[game]
    N, K, M = 8192, 6, 3000
    x = torch.from_numpy(hjg_inputs.points(w, M=M)).cuda()
    s = Solver(w.game, w.nu, w.T, N, K, radius=w.radius, seed=0)
    v_ref, g_ref, r_ref = s.value_grad(x)
    s.close()
    v_ref = v_ref.cpu().numpy(); g_ref = g_ref.cpu().numpy()

    dyn, tgt, opt = _structs(w, N, K)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        v = torch.full((M,), float("nan"), dtype=torch.float64, device="cuda")
        g = torch.full((M, w.n), float("nan"), dtype=torch.float32, device="cuda")
        r = torch.full((2 * K,), float("nan"), dtype=torch.float64, device="cuda")
        st = _noalloc(lib, dyn, tgt, w.nu, w.T, opt, x, v, g, r, stream)
        assert st == 0, _lib.status_string(st)
        torch.cuda.synchronize()
        assert_parity(v.cpu().numpy(), g.cpu().numpy(), v_ref, g_ref,
                      what="noalloc call %d" % call)
        res = r.cpu().numpy().reshape(K, 2)[:, 0]
        np.testing.assert_allclose(res, r_ref, rtol=1e-6, atol=1e-12)


# Options passed both to the context (Solver keywords) and to the allocation-free call
# (hjg_options fields): the 45-D four-lanes-per-sample kernel on its default and on a
# software-pipelined variant, the control variate in the tilted frame, a shard's point
# offset (the Philox counter of every state moves with it), and a CTA size chosen by
# block_threads instead of a variant index.
OPTION_CASES = [
    ("rockets45", dict(), 300, 2048, 3),
    ("rockets45", dict(variant=8), 300, 2048, 3),
    ("rockets45", dict(tilt=True, cv=True), 200, 2048, 2),
    ("dubins3", dict(tilt=True, cv=True), 800, 4096, 3),
    ("rockets6", dict(point_offset=12345), 1000, 4096, 3),
    ("rockets45", dict(point_offset=777), 200, 2048, 2),
    ("dubins3", dict(block_threads=256), 800, 4096, 3),
]


@pytest.mark.parametrize("game,kw,M,N,K", OPTION_CASES,
                         ids=["r45", "r45-pipelined", "r45-cv-tilt", "dubins3-cv-tilt",
                              "rockets6-offset", "r45-offset", "dubins3-block256"])
def test_noalloc_options_match_value_grad(game, kw, M, N, K):
    from paper_2605_18566_gb300 import _lib
    lib = _lib.load()
    w = {"dubins3": hjg_inputs.DUBINS3, "rockets6": hjg_inputs.ROCKETS6,
         "rockets45": hjg_inputs.ROCKETS45}[game]
    x = torch.from_numpy(hjg_inputs.points(w, M=M)).cuda()
    s = solver_for(w, N=N, K=K, seed=0, **kw)
    v_ref, g_ref, r_ref = s.value_grad(x)
    s.close()
    v_ref = v_ref.cpu().numpy(); g_ref = g_ref.cpu().numpy()
    dyn, tgt, opt = _structs(w, N, K)
    for i, a in enumerate(w.speed or []):
        dyn.speed[i] = a
    opt.tilt = 1 if kw.get("tilt") else 0
    opt.cv = 1 if kw.get("cv") else 0
    opt.point_offset = kw.get("point_offset", 0)
    opt.block_threads = kw.get("block_threads", 0)
    opt.variant = kw["variant"] + 1 if "variant" in kw else 0
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        v = torch.full((M,), float("nan"), dtype=torch.float64, device="cuda")
        g = torch.full((M, w.n), float("nan"), dtype=torch.float32, device="cuda")
        r = torch.full((2 * K,), float("nan"), dtype=torch.float64, device="cuda")
        st = _noalloc(lib, dyn, tgt, w.nu, w.T, opt, x, v, g, r, stream)
        assert st == 0, _lib.status_string(st)
        torch.cuda.synchronize()
        assert_parity(v.cpu().numpy(), g.cpu().numpy(), v_ref, g_ref,
                      what="noalloc %s %s call %d" % (game, kw, call))
        res = r.cpu().numpy().reshape(K, 2)[:, 0]
        np.testing.assert_allclose(res, r_ref, rtol=1e-5, atol=1e-12)


def test_noalloc_point_offset_draws_the_shard_samples():
    """A shard [a, b) of a state set, solved with point_offset = a, reproduces those rows
    of the solve of the whole set (the same Philox counters), bit for bit."""
    from paper_2605_18566_gb300 import _lib
    lib = _lib.load()
    w = hjg_inputs.ROCKETS6
    N, K, M, a, b = 4096, 3, 1200, 500, 900
    x = torch.from_numpy(hjg_inputs.points(w, M=M)).cuda()
    dyn, tgt, opt = _structs(w, N, K)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = []
    for lo, hi in ((0, M), (a, b)):
        opt.point_offset = lo
        xs = x[lo:hi].contiguous()
        v = torch.full((hi - lo,), float("nan"), dtype=torch.float64, device="cuda")
        g = torch.full((hi - lo, w.n), float("nan"), dtype=torch.float32, device="cuda")
        r = torch.full((2 * K,), float("nan"), dtype=torch.float64, device="cuda")
        st = _noalloc(lib, dyn, tgt, w.nu, w.T, opt, xs, v, g, r, stream)
        assert st == 0, _lib.status_string(st)
        torch.cuda.synchronize()
        out.append((v.cpu().numpy(), g.cpu().numpy()))
    np.testing.assert_array_equal(out[1][0], out[0][0][a:b])
    np.testing.assert_array_equal(out[1][1], out[0][1][a:b])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2605_18566_gb300 import _lib
    lib = _lib.load()
    w = hjg_inputs.ROCKETS6
    K = 20
    dyn, tgt, opt = _structs(w, 64, K)
    M = 120_000                    # (8K + 16) M bytes = 21 MB > 16 MiB
    x = torch.zeros(M, w.n, device="cuda")
    v = torch.empty(M, dtype=torch.float64, device="cuda")
    g = torch.empty(M, w.n, device="cuda")
    r = torch.empty(2 * K, dtype=torch.float64, device="cuda")
    st = _noalloc(lib, dyn, tgt, w.nu, w.T, opt, x, v, g, r, None)
    assert st == _lib.HJG_EINVAL


def test_noalloc_fp64_and_obstacle_match_value_grad():
    """The FP64 sweep and the reach-avoid obstacle through the allocation-free entry point:
    the same kernel as the context path, so the results agree bit for bit."""
    from paper_2605_18566_gb300 import Solver, _lib
    lib = _lib.load()
    w = hjg_inputs.DUBINS3
    N, K, M = 2048, 4, 1000
    obst = (0.8, 0.3, 0.6)
    x = torch.from_numpy(hjg_inputs.points(w, M=M)).cuda()
    s = Solver(w.game, w.nu, w.T, N, K, radius=w.radius, seed=0, precision="fp64", obstacle=obst)
    v_ref, g_ref, r_ref = s.value_grad(x)
    s.close()
    dyn, tgt, opt = _structs(w, N, K)
    opt.precision = 1
    tgt.obstacle_radius = obst[2]
    tgt.obstacle_center[0], tgt.obstacle_center[1] = obst[0], obst[1]
    v = torch.full((M,), float("nan"), dtype=torch.float64, device="cuda")
    g = torch.full((M, w.n), float("nan"), dtype=torch.float32, device="cuda")
    r = torch.full((2 * K,), float("nan"), dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = _noalloc(lib, dyn, tgt, w.nu, w.T, opt, x, v, g, r, stream)
    assert st == 0, _lib.status_string(st)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(v.cpu().numpy(), v_ref.cpu().numpy())
    np.testing.assert_array_equal(g.cpu().numpy(), g_ref.cpu().numpy())
