"""Failure detection without a GPU fault: a device wait that nothing satisfies gives up
after its iteration limit, reports HJG_ETIMEOUT through the host status, and leaves the
context usable (the next tensor-core GEMM and solve run normally)."""
import ctypes as C

import numpy as np
import pytest

import hjg_inputs
from helpers import solver_for

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_device_stays_usable():
    from paper_2605_18566_gb300 import _lib
    lib = _lib.load()
    assert lib.hjg_selftest_bounded_wait(0, 2000, None) == _lib.HJG_ETIMEOUT
    assert lib.hjg_selftest_bounded_wait(1, 2000, None) == _lib.HJG_OK
    # the same process keeps working: a GEMM on the tensor cores and a sweep
    a = torch.randn(256, 64, device="cuda").to(torch.bfloat16)
    b = torch.randn(128, 64, device="cuda").to(torch.bfloat16)
    c = torch.zeros(256, 128, device="cuda")
    flag = C.c_int(0)
    st = lib.hjg_gemm_bf16(C.c_void_p(a.data_ptr()), 64, 1, C.c_void_p(b.data_ptr()), 1, 64, 256, 128, 64,
                           C.c_void_p(c.data_ptr()), 128, C.byref(flag), None)
    assert st == 0 and flag.value == 0
    ref = a.float() @ b.float().T
    assert torch.allclose(c, ref, rtol=1e-3, atol=1e-3)
    s = solver_for(hjg_inputs.DUBINS3, N=512, K=2)
    s.set_points(torch.from_numpy(hjg_inputs.points(hjg_inputs.DUBINS3, M=64)).cuda())
    r, _ = s.picard_sweep(2)
    assert np.all(np.isfinite(r))
    s.close()
    assert lib.hjg_selftest_bounded_wait(0, 0, None) == _lib.HJG_EINVAL
